"""flb_structure_factor_noalloc: the structure factor for callers that cannot
allocate device memory while they run (allocators that forbid cudaMalloc after
start-up, fixed-budget real-time loops).

It reads populations from a device buffer the caller owns, writes S_a(k) into
another caller-owned device buffer and uses a static device work array, so it
must give what flb_structure_factor gives on the same state.  Device buffers
here come from PyTorch (plumbing only); the call itself goes through the C ABI.
This file is collected last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

from paper_1012_3632_gb300 import Context, flb

pytestmark = pytest.mark.gpu


def _noalloc(torch, lattice, dims, f_host, mode):
    L = flb.lib()
    V = dims[0] * dims[1] * dims[2]
    f_dev = torch.from_numpy(np.ascontiguousarray(f_host)).to("cuda")
    S_dev = torch.full((V,), float("nan"), dtype=torch.float64, device="cuda")
    d = (ctypes.c_int * 3)(*dims)
    stream = torch.cuda.current_stream()
    rc = L.flb_structure_factor_noalloc(lattice, d, ctypes.c_void_p(f_dev.data_ptr()), mode,
                                        ctypes.c_void_p(S_dev.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, L.flb_last_error()
    torch.cuda.synchronize()
    return S_dev.cpu().numpy()


@pytest.mark.parametrize("lattice,dims,modes", [(19, (12, 10, 9), (0, 7)), (9, (20, 15, 1), (0, 8))])
def test_noalloc_matches_structure_factor_on_two_calls(lattice, dims, modes):
    torch = pytest.importorskip("torch")
    with Context(lattice, dims, precision="fp64", kT=1e-4, omega_shear=1.2, seed=3) as ctx:
        ctx.init(thermal=True)
        for mode in modes:  # two calls in a row, the second on a later state
            ctx.step(3)
            want = ctx.structure_factor(mode)
            got = _noalloc(torch, lattice, dims, ctx.get_populations(), mode)
            assert np.allclose(got, want, rtol=1e-10, atol=1e-18)


@pytest.mark.parametrize("mode", [0, 18])
def test_noalloc_at_the_maximum_size(mode):
    """D3Q19 128x128x64 = FLB_NOALLOC_MAX_SITES sites, the one size that fills
    the static work array: element by element equal to flb_structure_factor."""
    torch = pytest.importorskip("torch")
    dims = (128, 128, 64)
    assert dims[0] * dims[1] * dims[2] == 1 << 20
    with Context(19, dims, precision="fp64", kT=1e-4, omega_shear=1.2, omega_bulk=0.9, omega_ghost=1.4,
                 seed=5) as ctx:
        ctx.init(thermal=True)
        ctx.step(2)
        want = ctx.structure_factor(mode)
        f = ctx.get_populations()
    for _ in range(2):  # two calls in a row on the same state
        got = _noalloc(torch, 19, dims, f, mode)
        assert np.allclose(got, want, rtol=1e-10, atol=1e-18)


def test_noalloc_rejects_unsupported_sizes():
    torch = pytest.importorskip("torch")
    L = flb.lib()
    f_dev = torch.zeros(19, dtype=torch.float64, device="cuda")
    S_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    # too many sites; an edge with a prime factor 7; edges whose product overflows 32 bits
    for dims in ((1024, 1024, 2), (7, 4, 4), (4096, 4096, 4096), (2 ** 30, 2 ** 30, 2 ** 30)):
        d = (ctypes.c_int * 3)(*dims)
        rc = L.flb_structure_factor_noalloc(19, d, ctypes.c_void_p(f_dev.data_ptr()), 0,
                                            ctypes.c_void_p(S_dev.data_ptr()), None)
        assert rc == flb.FLB_EINVAL
        assert len(L.flb_last_error()) > 0
