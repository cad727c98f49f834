"""GB300-native fluctuating lattice Boltzmann (arXiv 1012.3632).

The compute path is the CUDA library ``libflb.so`` (C ABI in
``include/flb.h``); :mod:`.flb` is its ctypes binding and :mod:`.inputs` holds
the seeded synthetic input generators.
"""
from .flb import (BF16, D2Q9, D3Q19, FP32, FP64, MODE_VAR, MODES, RHO, U, Batch, Context, FLBError,  # noqa: F401
                  interface_fit, landau_free_energy, landau_width, lib, options)
