"""The C-ABI library builds, loads and exports every entry point of include/flb.h;
argument validation answers without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def flb():
    from paper_1012_3632_gb300 import build, flb

    build.build()
    return flb


def _declared():
    src = open(os.path.join(ROOT, "include", "flb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(flb_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(flb):
    L = flb.lib()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert sorted(flb.EXPORTS) == names


def test_error_strings(flb):
    L = flb.lib()
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert len(L.flb_error_string(code)) > 3
    assert L.flb_error_string(-99) == b"unknown error"


@pytest.mark.parametrize("kw", [
    dict(lattice=7),
    dict(dims=(0, 4, 4)),
    dict(lattice=9, dims=(4, 4, 2)),
    dict(omega_shear=2.0),
    dict(omega_bulk=0.0),
    dict(kT=-1e-5),
    dict(kT=0.5),
    dict(dims=(2048, 1024, 1024)),          # V = 2^31: beyond the 32-bit site index
    dict(opts=dict(guard=2)),
    dict(opts=dict(z_chunk=-1)),
    dict(dims=(4, 4, 262140), opts=dict(z_chunk=1)),  # 262140 z-blocks exceed the launch grid
    dict(opts=dict(check_every=-1)),
])
def test_invalid_arguments_rejected_before_any_device_work(flb, kw):
    """flb_create validates its arguments first (FLB_EINVAL, no context)."""
    L = flb.lib()
    args = dict(lattice=19, dims=(4, 4, 4), omega_shear=1.0, omega_bulk=1.0, omega_ghost=1.0, kT=1e-5)
    args.update(kw)
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 3)(*args["dims"])
    o = flb.options(**args.get("opts", {}))
    rc = L.flb_create(ctypes.byref(h), args["lattice"], d, args["omega_shear"], args["omega_bulk"], 1.0,
                      args["kT"], None, 1, ctypes.byref(o))
    assert rc == flb.FLB_EINVAL
    assert not h.value
    assert len(L.flb_last_error()) > 0


def test_default_options(flb):
    o = flb.options()
    assert o.precision == flb.FP32 and o.rho0 == 1.0 and o.noise_rho_local == 1 and o.device == -1
    assert o.check_every == 0 and o.guard == 0 and o.z_chunk == 0


def test_graft_entry_build_compiles_everything():
    import __graft_entry__ as g

    g.build()
    assert os.path.exists(os.path.join(ROOT, "paper_1012_3632_gb300", "libflb.so"))
    assert os.path.exists(os.path.join(ROOT, "oracle", "liborc.so"))


def test_null_context_rejected(flb):
    """Every entry point that takes a context refuses NULL with FLB_EINVAL
    before touching the device."""
    L = flb.lib()
    d = (ctypes.c_double * 64)()
    ll = (ctypes.c_longlong * 2)(0, 1)
    i1, i2 = ctypes.c_int(), ctypes.c_int()
    calls = [
        lambda: L.flb_step(None, 1),
        lambda: L.flb_step_sums(None, 1, d),
        lambda: L.flb_step_sums_async(None, 1, d),
        lambda: L.flb_conservation(None, d),
        lambda: L.flb_get_populations(None, d),
        lambda: L.flb_get_sites(None, ll, 2, d),
        lambda: L.flb_check_guards(None),
        lambda: L.flb_z_chunk(None, ctypes.byref(i1), ctypes.byref(i2)),
        lambda: L.flb_adjoint_step(None, None, 0, None, None, None),
        lambda: L.flb_adjoint_segment(None, None, 0, 1, None, None, None),
        lambda: L.flb_structure_factor(None, d, 0, 0),
    ]
    for k, call in enumerate(calls):
        assert call() == flb.FLB_EINVAL, k
