"""The oracle's Philox4x32-10 against cuRAND's (a library generator) on the GPU:
a second pin of the noise generator, independent of the Triton one on the
CPU.  The helper tests/curand_philox.cu is compiled here with nvcc and maps a
counter (c0, c1, c2, c3) and key (k0, k1) onto curand_init's seed,
subsequence and offset (see its header)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    so = str(tmp_path_factory.mktemp("curand") / "libcurandphilox.so")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler",
                           "-fPIC", os.path.join(HERE, "curand_philox.cu"), "-o", so])
    lib = ctypes.CDLL(so)
    lib.curand_philox_words.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.c_ulonglong, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_uint32)]
    lib.curand_philox_words.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("seed", [0, 1, 0x1234567890ABCDEF, 2 ** 64 - 1])
def test_oracle_philox_equals_curand(orc, curand_lib, seed):
    rng = np.random.default_rng(seed % 1000 + 3)
    n = 512
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] &= (1 << 30) - 1          # c1 < 2^30 (the offset of curand_init is 4 (c0 | c1 << 32))
    ctr[0] = [0, 0, 0, 0]
    ctr[1] = [0xFFFFFFFF, (1 << 30) - 1, 0xFFFFFFFF, 0xFFFFFFFF]
    ctr[2] = [7, 100, 1 | (1 << 8), 5]  # a noise counter: site, step, call | tag << 8, replica
    out = np.zeros((n, 4), dtype=np.uint32)
    c = np.ascontiguousarray(ctr)
    rc = curand_lib.curand_philox_words(c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), seed, n,
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    assert rc == 0
    key = [seed & 0xFFFFFFFF, seed >> 32]
    mine = np.array([orc.philox4x32_10(list(map(int, ci)), key) for ci in ctr], dtype=np.uint32)
    assert np.array_equal(mine, out)
