"""GPU <-> oracle parity through the C ABI (same seeds, same inputs).

Tolerances (on max |df| of the pre-collision populations):
  FP64 path   1e-12 (both sides double; only rounding order differs)
  FP32 path   2e-5 * rho0 after 100 steps (float deviation storage)
  BF16 path   bfloat16 keeps 8 mantissa bits of deviations |g| <~ 0.02:
              ~4e-5 rounding per step; 2e-3 after 20 steps.
"""
import numpy as np
import pytest

import oracle
from paper_1012_3632_gb300 import BF16, D2Q9, D3Q19, FP32, FP64, MODE_VAR, MODES, RHO, U, Context, inputs
from paper_1012_3632_gb300.flb import FLBError

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5, "bf16": 2e-3}
FE = dict(A=-0.01, B=0.1, rho_c=1.0, kappa=0.02)


def _pair(Q, dims, prec, fe=None, **kw):
    ctx = Context(Q, dims, precision=prec, free_energy=fe, **kw)
    p = oracle.Params(Q=Q, dims=dims, nonideal=fe is not None, **(fe or {}), **kw)
    return ctx, p


def _run_both(Q, dims, prec, steps, fe=None, rho=None, u=None, thermal=False, **kw):
    ctx, p = _pair(Q, dims, prec, fe, **kw)
    with ctx:
        ctx.init(rho=rho, u=u, thermal=thermal)
        ctx.step(steps)
        got = ctx.get_populations()
    want = oracle.run(p, oracle.init(p, rho=rho, u=u, thermal=thermal), 0, steps)
    return got, want


def test_d2q9_32x32_fp64_ideal_100_steps():
    """D2Q9 ideal gas 32x32, FP64, rho0 = 1, kT = 1e-4, all rates 1, f = w rho0, seed 1."""
    got, want = _run_both(9, (32, 32, 1), "fp64", 100, kT=1e-4, omega_shear=1.0, omega_bulk=1.0,
                          omega_ghost=1.0, seed=1)
    assert np.abs(got - want).max() <= TOL["fp64"]


@pytest.mark.parametrize("Q,dims", [(9, (17, 13, 1)), (19, (12, 10, 9)), (19, (1, 1, 1)), (19, (2, 3, 5)),
                                    (9, (1, 1, 1)), (19, (33, 5, 3))])
def test_fp64_ideal_ragged(Q, dims):
    D = 2 if Q == 9 else 3
    u = inputs.random_velocity(dims, D, amp=0.02, seed=2)
    got, want = _run_both(Q, dims, "fp64", 60, u=u, thermal=True, kT=1e-4, omega_shear=1.3,
                          omega_bulk=0.8, omega_ghost=1.55, seed=7)
    assert np.abs(got - want).max() <= TOL["fp64"]


@pytest.mark.parametrize("Q,dims", [(9, (24, 19, 1)), (19, (12, 10, 9)), (19, (35, 6, 5)), (19, (3, 2, 2))])
def test_fp64_nonideal(Q, dims):
    rho = inputs.uniform_density(dims, seed=4)
    got, want = _run_both(Q, dims, "fp64", 60, fe=FE, rho=rho, thermal=True, kT=1e-6, omega_shear=1.1,
                          omega_bulk=1.0, omega_ghost=1.2, seed=9)
    assert np.abs(got - want).max() <= TOL["fp64"]


def test_fp64_random_state_noise_rho0():
    """A generic non-equilibrium start, noise with the reference density (noise_rho_local = 0)."""
    dims = (9, 8, 7)
    f0 = inputs.random_populations(19, dims, seed=3)
    kw = dict(kT=1e-4, omega_shear=0.7, omega_bulk=1.6, omega_ghost=1.9, seed=2 ** 40 + 3, replica=5)
    ctx = Context(19, dims, precision="fp64", noise_rho_local=False, **kw)
    p = oracle.Params(Q=19, dims=dims, noise_rho_local=False, **kw)
    with ctx:
        ctx.set_populations(f0)
        assert np.abs(ctx.get_populations() - f0).max() < 1e-15
        ctx.step_count = 1000
        ctx.step(30)
        got = ctx.get_populations()
    want = oracle.run(p, f0, 1000, 30)
    assert np.abs(got - want).max() <= TOL["fp64"]


@pytest.mark.parametrize("dims", [(16, 16, 16), (17, 9, 8), (2, 5, 3)])
def test_fp32_d3q19_ideal_shear_wave_100_steps(dims):
    """D3Q19 ideal, FP32 deviations, kT = 1e-5, rates (1.2, 1, 1), shear wave + thermal start.
    Even X runs the packed two-site kernel, odd X the one-site kernel."""
    u = inputs.shear_wave(dims, amp=1e-3)
    got, want = _run_both(19, dims, "fp32", 100, u=u, thermal=True, kT=1e-5, omega_shear=1.2, omega_bulk=1.0,
                          omega_ghost=1.0, seed=2)
    assert np.abs(got - want).max() <= TOL["fp32"]


@pytest.mark.parametrize("dims", [(16, 14, 12), (15, 12, 10), (2, 3, 4), (34, 6, 5), (72, 10, 6), (4, 5, 3)])
def test_fp32_d3q19_nonideal_100_steps(dims):
    """D3Q19 non-ideal (A=-0.01, B=0.1, rho_c=1, kappa=0.02), FP32, kT = 1e-6, rates 1.
    Even X runs the packed two-site kernel, odd X the one-site kernel."""
    rho = inputs.uniform_density(dims, seed=3)
    got, want = _run_both(19, dims, "fp32", 100, fe=FE, rho=rho, kT=1e-6, omega_shear=1.0, omega_bulk=1.0,
                          omega_ghost=1.0, seed=3)
    assert np.abs(got - want).max() <= TOL["fp32"]


def test_fp32_d2q9_nonideal():
    dims = (40, 33, 1)
    rho = inputs.uniform_density(dims, seed=8)
    got, want = _run_both(9, dims, "fp32", 100, fe=FE, rho=rho, thermal=True, kT=1e-5, omega_shear=1.4,
                          omega_bulk=0.9, omega_ghost=1.0, seed=5)
    assert np.abs(got - want).max() <= TOL["fp32"]


def test_bf16_storage():
    dims = (16, 12, 10)
    got, want = _run_both(19, dims, "bf16", 20, thermal=True, kT=1e-5, omega_shear=1.2, omega_bulk=1.0,
                          omega_ghost=1.0, seed=4)
    assert np.abs(got - want).max() <= TOL["bf16"]


@pytest.mark.parametrize("dims,fe", [((24, 10, 9), FE), ((18, 10, 9), FE), ((17, 10, 9), FE), ((15, 12, 10), None),
                                     ((4, 5, 3), FE)])
def test_bf16_storage_paths(dims, fe):
    """BF16 storage through every D3Q19 step kernel: the two-sites-per-thread
    non-ideal step with quad (X % 4 = 0) and pair gathers, the one-site kernels
    for odd X, ideal and non-ideal, against the FP64 oracle after 20 steps."""
    rho = inputs.uniform_density(dims, seed=3) if fe else None
    got, want = _run_both(19, dims, "bf16", 20, fe=fe, rho=rho, thermal=fe is None, kT=1e-5, omega_shear=1.1,
                          omega_bulk=1.0, omega_ghost=1.2, seed=6)
    assert np.abs(got - want).max() <= TOL["bf16"]


@pytest.mark.parametrize("Q,dims", [(19, (6, 5, 4)), (9, (7, 5, 1))])
def test_init_parity(Q, dims):
    D = 2 if Q == 9 else 3
    rho = inputs.uniform_density(dims, amp=0.05, seed=1)
    u = inputs.random_velocity(dims, D, seed=1)
    kw = dict(kT=1e-4, omega_shear=1.0, seed=12)
    ctx, p = _pair(Q, dims, "fp64", **kw)
    with ctx:
        ctx.init(rho=rho, u=u, thermal=True)
        got = ctx.get_populations()
        assert ctx.step_count == 0
    want = oracle.init(p, rho=rho, u=u, thermal=True)
    assert np.abs(got - want).max() <= 1e-15


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fe", [None, FE])
def test_observables(prec, fe):
    Q, dims = 19, (10, 9, 8)
    rho = inputs.uniform_density(dims, seed=2)
    kw = dict(kT=1e-5, omega_shear=1.2, seed=3)
    ctx, p = _pair(Q, dims, prec, fe, **kw)
    tol = 1e-13 if prec == "fp64" else 1e-6
    with ctx:
        ctx.init(rho=rho, thermal=True)
        ctx.step(5)
        f = ctx.get_populations()
        r = ctx.moments(RHO)
        u = ctx.moments(U)
        m = ctx.moments(MODES)
        cons = ctx.conservation()
    f_or = oracle.run(p, oracle.init(p, rho=rho, thermal=True), 0, 5)
    assert np.abs(f - f_or).max() <= TOL[prec]
    # observables of the GPU state, recomputed by the oracle
    assert np.abs(r - f.sum(axis=0)).max() <= tol
    assert np.abs(u - oracle.velocity(p, f)).max() <= tol
    assert np.abs(m - oracle.modes(p, f)).max() <= tol
    L = oracle.lattice(Q)
    c = L.c.astype(float)
    assert abs(cons[0] - f.sum()) <= 1e-9
    assert np.allclose(cons[1:], (c.T @ f).sum(axis=1), atol=1e-9)


@pytest.mark.parametrize("dims", [(6, 5, 4), (8, 8, 8), (12, 10, 9), (7, 3, 1), (16, 1, 1)])
def test_structure_factor(dims):
    Q = 9 if dims[2] == 1 and dims[1] > 1 and dims[0] == 7 else 19
    if Q == 9:
        dims = (dims[0], dims[1], 1)
    kw = dict(kT=1e-4, omega_shear=1.2, seed=6)
    ctx, p = _pair(Q, dims, "fp64", **kw)
    with ctx:
        ctx.init(thermal=True)
        ctx.step(3)
        f = ctx.get_populations()
        for mode in (0, 1, Q - 1):
            S = ctx.structure_factor(mode)
            want = oracle.structure_factor(p, f, mode)
            assert np.allclose(S, want, rtol=1e-10, atol=1e-18), mode
        # accumulation over snapshots = mean of the snapshots
        s1 = ctx.structure_factor(0, accumulate=True)
        ctx.step(2)
        s2 = ctx.structure_factor(0, accumulate=False)
        mean = ctx.structure_factor(0, accumulate=True)
        assert ctx.snapshot_count(0) == 2
        assert np.allclose(mean, 0.5 * (s1 + s2), rtol=1e-12, atol=1e-20)


@pytest.mark.parametrize("Q,dims,prec", [(19, (12, 10, 9), "fp32"), (19, (16, 15, 8), "bf16"), (9, (20, 14, 1), "fp32"),
                                         (19, (14, 6, 5), "fp32")])
def test_structure_factor_single_precision_state(Q, dims, prec):
    """FP32 and BF16 states are transformed with the FP32 FFT (|F|^2 summed in
    FP64): S_a(k) of the GPU's own state against the oracle's FP64 DFT of the
    same populations, within the FP32 transform's rounding (14 = 2 * 7 takes
    the direct DFT)."""
    kw = dict(kT=1e-4, omega_shear=1.2, seed=6)
    ctx, p = _pair(Q, dims, prec, **kw)
    with ctx:
        ctx.init(thermal=True)
        ctx.step(3)
        f = ctx.get_populations()
        for mode in (0, 1, Q - 1):
            S = ctx.structure_factor(mode)
            want = oracle.structure_factor(p, f, mode)
            assert np.allclose(S, want, rtol=1e-4, atol=1e-5 * want.max()), mode


def test_mode_variance_accumulator():
    Q, dims = 19, (8, 7, 6)
    kw = dict(kT=1e-4, omega_shear=1.2, seed=6)
    ctx, p = _pair(Q, dims, "fp64", **kw)
    with ctx:
        ctx.init(thermal=True)
        v1 = ctx.moments(MODE_VAR)
        f1 = ctx.get_populations()
        ctx.step(4)
        v2 = ctx.moments(MODE_VAR)
        f2 = ctx.get_populations()
        assert ctx.snapshot_count(-1) == 2
    var = lambda f: oracle.modes(p, f).var(axis=1)
    assert np.allclose(v1, var(f1), rtol=1e-10, atol=1e-20)
    assert np.allclose(v2, 0.5 * (var(f1) + var(f2)), rtol=1e-10, atol=1e-20)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_checkpoint_resume_is_bitwise(tmp_path, prec):
    Q, dims = 19, (9, 8, 7)
    kw = dict(kT=1e-5, omega_shear=1.2, seed=8, free_energy=FE)
    rho = inputs.uniform_density(dims, seed=6)
    with Context(Q, dims, precision=prec, **kw) as a:
        a.init(rho=rho, thermal=True)
        a.step(7)
        a.save(str(tmp_path / "c.flb"))
        a.step(9)
        fa = a.get_populations()
    with Context.load(str(tmp_path / "c.flb")) as b:
        assert b.step_count == 7
        b.step(9)
        fb = b.get_populations()
    assert np.array_equal(fa, fb)


SWIFT_FE = dict(A=-0.025, B=0.4, rho_c=0.75, kappa=0.08, total=True, model=1)


@pytest.mark.parametrize("Q,dims,fe,gathers", [(19, (32, 16, 8), FE, 0), (9, (32, 16, 1), FE, 0),
                                               (9, (32, 16, 1), SWIFT_FE, 5)])
def test_kernel_timing_counts_launches(Q, dims, fe, gathers):
    """The force-model steps gather the density inside the step kernel; the
    modified-equilibrium step reads a density field (and its coloured noise)
    made by a launch before it."""
    with Context(Q, dims, precision="fp32", free_energy=fe, kT=1e-6, omega_shear=1.0) as ctx:
        ctx.init(rho=inputs.uniform_density(dims))
        ctx.kernel_timing(True)
        ctx.step(5)
        ms, n = ctx.kernel_times()
        assert list(n[:2]) == [gathers, 5] and ms[1] > 0 and (ms[0] > 0) == (gathers > 0)


def test_divergence_is_reported():
    """A NaN population (set on the host) makes the next checked step return FLB_EDIVERGED."""
    from paper_1012_3632_gb300 import FLBError

    dims = (6, 6, 6)
    with Context(19, dims, precision="fp32", kT=1e-5, omega_shear=1.0, check_every=1) as ctx:
        f = ctx.get_populations()
        f[3, 17] = np.nan
        ctx.set_populations(f)
        with pytest.raises(FLBError) as e:
            ctx.step(1)
        assert e.value.code == -4


# ---------------------------------------------------------------------------
# Full-size workloads: sampled sites against oracle windows
# ---------------------------------------------------------------------------

def _window_check(Q, dims, prec, steps, fe, rho, u, thermal, kw, centres, tol):
    ctx, p = _pair(Q, dims, prec, fe, **kw)
    with ctx:
        ctx.init(rho=rho, u=u, thermal=thermal)
        ctx.step(steps)
        f = ctx.get_populations()
    D = 2 if Q == 9 else 3
    radius = steps * (3 if fe else 1)  # light cone: streaming 1, force stencils 2 more
    X, Y, Z = dims
    for cen in centres:
        h = radius + 1
        org = tuple(c - h for c in cen)
        win = tuple(2 * h + 1 for _ in cen)
        if D == 2:
            org, win = (org[0], org[1], 0), (win[0], win[1], 1)
        gx = (np.arange(win[0]) + org[0]) % X
        gy = (np.arange(win[1]) + org[1]) % Y
        gz = (np.arange(win[2]) + org[2]) % Z
        sites = (gx[None, None, :] + X * (gy[None, :, None] + Y * gz[:, None, None])).reshape(-1)
        pw = p.with_(origin=org, window=win)
        rw = None if rho is None else rho[sites]
        uw = None if u is None else u[:, sites]
        fw = oracle.run(pw, oracle.init(pw, rho=rw, u=uw, thermal=thermal), 0, steps)
        c_local = (h, h, h if D == 3 else 0)
        s_loc = c_local[0] + win[0] * (c_local[1] + win[1] * c_local[2])
        s_glob = cen[0] + X * (cen[1] + Y * (cen[2] if D == 3 else 0))
        assert np.isfinite(fw[:, s_loc]).all()
        assert np.abs(f[:, s_glob] - fw[:, s_loc]).max() <= tol, cen


def test_full_size_nonideal_256cubed_sampled():
    """256^3 non-ideal FP32 (the benchmark workload): 3 steps, 4 sampled sites."""
    dims = (256, 256, 256)
    rho = inputs.uniform_density(dims, seed=3)
    kw = dict(kT=1e-6, omega_shear=1.0, omega_bulk=1.0, omega_ghost=1.0, seed=3)
    centres = [(0, 0, 0), (255, 17, 128), (100, 255, 3), (37, 200, 255)]
    _window_check(19, dims, "fp32", 3, FE, rho, None, False, kw, centres, TOL["fp32"])


def test_full_size_ideal_128cubed_sampled():
    """128^3 ideal FP32 with shear wave and thermal start: 5 steps, 4 sampled sites."""
    dims = (128, 128, 128)
    u = inputs.shear_wave(dims, amp=1e-3)
    kw = dict(kT=1e-5, omega_shear=1.2, omega_bulk=1.0, omega_ghost=1.0, seed=2)
    centres = [(0, 0, 0), (127, 64, 1), (5, 127, 127), (90, 33, 64)]
    _window_check(19, dims, "fp32", 5, None, None, u, True, kw, centres, TOL["fp32"])


@pytest.mark.parametrize("Q,dims,prec", [
    (19, (72, 70, 64), "fp32"), (19, (72, 70, 64), "bf16"), (9, (613, 517, 1), "fp32"), (19, (5, 3, 2), "fp32"),
])
def test_conservation_sums_are_exact_sums_of_the_state(Q, dims, prec):
    """flb_conservation on single-precision state (compensated single-precision
    sums, several sites per thread, a ragged last block) equals the FP64 sum of
    the populations: mass and momentum, the invariants of the collision (Sec. II)."""
    rho = inputs.uniform_density(dims, seed=5)
    with Context(Q, dims, 1.2, kT=1e-5, seed=6, precision=prec) as ctx:
        ctx.init(rho=rho, thermal=True)
        ctx.step(3)
        f = ctx.get_populations()
        cons = ctx.conservation()
    c = oracle.lattice(Q).c.astype(float)
    V = int(np.prod(dims))
    assert abs(cons[0] - f.sum()) <= 1e-13 * V
    assert np.abs(np.asarray(cons[1:]) - (c.T @ f).sum(axis=1)).max() <= 1e-13 * V


@pytest.mark.parametrize("Q,dims,prec", [(19, (10, 9, 8), "fp64"), (19, (33, 5, 3), "fp32"), (9, (17, 13, 1), "bf16"),
                                         (19, (1, 1, 1), "fp32")])
def test_get_sites_equals_the_full_read(Q, dims, prec):
    """flb_get_sites returns exactly the columns of flb_get_populations (first
    and last site, repeats, random order); bad indices are refused."""
    V = int(np.prod(dims))
    with Context(Q, dims, 1.2, kT=1e-5, seed=4, precision=prec) as ctx:
        ctx.init(rho=inputs.uniform_density(dims, seed=1), thermal=True)
        ctx.step(3)
        f = ctx.get_populations()
        sites = np.r_[0, V - 1, np.random.default_rng(0).integers(0, V, 40), 0]
        assert np.array_equal(ctx.get_sites(sites), f[:, sites])
        assert ctx.get_sites([]).shape == (Q, 0)
        for bad in ([-1], [V], [0, V + 5]):
            with pytest.raises(FLBError):
                ctx.get_sites(bad)


def _sites_window_check(ctx, p, dims, steps, radius, centres, tol):
    """Populations at the centres (read with flb_get_sites) against oracle runs
    on periodic-free windows around them, from the uniform rest state."""
    X, Y, Z = dims
    glob = [c[0] + X * (c[1] + Y * c[2]) for c in centres]
    got = ctx.get_sites(glob)
    h = radius + 1
    for k, cen in enumerate(centres):
        org = tuple(c - h for c in cen)
        win = (2 * h + 1,) * 3
        pw = p.with_(origin=org, window=win)
        fw = oracle.run(pw, oracle.init(pw), 0, steps)
        s_loc = h + win[0] * (h + win[1] * h)
        assert np.isfinite(fw[:, s_loc]).all()
        assert np.abs(got[:, k] - fw[:, s_loc]).max() <= tol, cen


def _free_device_bytes():
    import torch
    return torch.cuda.mem_get_info()[0]


def test_max_size_bf16_ideal_sampled():
    """The largest lattice the API accepts, V = 2048*1024*1023 = 2 145 386 496
    sites (just below 2^31), BF16 storage (163 GB): 2 noisy steps, sampled sites
    against oracle windows, and the total mass."""
    dims = (2048, 1024, 1023)
    V = int(np.prod(dims))
    if _free_device_bytes() < 2 * 19 * 2 * V + 4 * V + 16e9:
        pytest.skip("not enough device memory")
    kw = dict(kT=1e-5, omega_shear=1.2, omega_bulk=1.0, omega_ghost=1.0, seed=11)
    ctx, p = _pair(19, dims, "bf16", None, **kw)
    with ctx:
        ctx.init()
        ctx.step(2)
        centres = [(0, 0, 0), (2047, 1023, 1022), (1000, 511, 700), (5, 1020, 1)]
        _sites_window_check(ctx, p, dims, 2, 2, centres, TOL["bf16"])
        cons = ctx.conservation()
    assert abs(cons[0] / V - 1.0) < 1e-6


def test_max_size_fp32_nonideal_sampled():
    """1024^3 non-ideal FP32 (163 GB, the z-marching fused kernel with plane
    offsets beyond 2^31 elements): 2 steps from the uniform state, sampled
    sites against oracle windows."""
    dims = (1024, 1024, 1024)
    V = int(np.prod(dims))
    if _free_device_bytes() < 2 * 19 * 4 * V + 4 * V + 16e9:
        pytest.skip("not enough device memory")
    kw = dict(kT=1e-6, omega_shear=1.0, omega_bulk=1.0, omega_ghost=1.0, seed=3)
    ctx, p = _pair(19, dims, "fp32", FE, **kw)
    with ctx:
        ctx.init()
        ctx.step(2)
        centres = [(0, 0, 0), (1023, 1023, 1023), (512, 100, 900), (3, 1022, 511)]
        _sites_window_check(ctx, p, dims, 2, 6, centres, TOL["fp32"])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_z_chunk_changes_no_result(prec):
    """Planes of z per block of the z-marching non-ideal step -- fixed (1, 3, 7,
    16, Z) or tuned by flb_step on its first launches (0) -- leave every
    population bitwise the same; the tuned run agrees with the oracle."""
    dims = (24, 20, 70)
    rho = inputs.uniform_density(dims, seed=4)
    kw = dict(kT=1e-6, omega_shear=1.1, omega_bulk=1.0, omega_ghost=1.2, seed=9)
    out = []
    for zc in (0, 1, 3, 7, 16, 70):
        with Context(19, dims, precision=prec, free_energy=FE, z_chunk=zc, **kw) as ctx:
            ctx.init(rho=rho)
            ctx.step(30)
            planes, tuning = ctx.z_chunk()
            assert not tuning and 1 <= planes <= 70
            if zc:
                assert planes == zc
            out.append(ctx.get_populations())
    for f in out[1:]:
        assert np.array_equal(f, out[0])
    p = oracle.Params(Q=19, dims=dims, nonideal=True, **FE, **kw)
    want = oracle.run(p, oracle.init(p, rho=rho), 0, 30)
    assert np.abs(out[0] - want).max() <= TOL[prec]
    with pytest.raises(FLBError):
        Context(19, dims, precision=prec, free_energy=FE, z_chunk=-1, **kw)


@pytest.mark.parametrize("Q,dims,prec,fe", [
    (19, (64, 16, 20), "fp32", FE),   # step kernel's own sums, whole 32 x 8 tiles
    (19, (32, 8, 9), "bf16", FE),     # the same with BF16 storage, one tile per row
    (19, (24, 20, 70), "fp32", FE),   # step kernel's own sums, quad gather
    (19, (18, 12, 9), "bf16", FE),    # pair gather, BF16 storage
    (19, (16, 12, 10), "fp32", None),  # ideal step: reduction before each step
    (19, (9, 8, 7), "fp64", FE),
    (9, (20, 14, 1), "fp32", FE),
])
def test_step_sums_equal_conservation_before_each_step(Q, dims, prec, fe):
    """flb_step_sums reports, for every step, the mass and momentum of the state
    the step starts from (flb_conservation of that state), and steps exactly
    as flb_step does."""
    n = 6
    rho = inputs.uniform_density(dims, seed=7)
    kw = dict(kT=1e-5, omega_shear=1.1, seed=8, precision=prec)
    V = int(np.prod(dims))
    with Context(Q, dims, free_energy=fe, **kw) as a:
        a.init(rho=rho)
        want = []
        for _ in range(n):
            want.append(a.conservation())
            a.step(1)
        fa = a.get_populations()
    with Context(Q, dims, free_energy=fe, **kw) as b:
        b.init(rho=rho)
        got = b.step_sums(n)
        fb = b.get_populations()
    assert np.array_equal(fa, fb)
    want = np.array(want)
    assert np.abs(got[:, 0] - want[:, 0]).max() <= 1e-12 * V + 1e-5
    assert np.abs(got[:, 1:] - want[:, 1:]).max() <= 1e-5
    # the same steps with flb_step_sums_async, one step per call into a
    # page-locked array read after one wait: the same sums and populations
    import torch

    pinned = torch.empty((n, 4), dtype=torch.float64, pin_memory=True).numpy()
    with Context(Q, dims, free_energy=fe, **kw) as c:
        c.init(rho=rho)
        for t in range(n):
            c.step_sums_async(1, pinned[t])
        c.synchronize()
        fc = c.get_populations()
    assert np.array_equal(fc, fb)
    assert np.array_equal(pinned, got)
    # both deliveries: page-locked memory written in place by the reduction
    # (synchronous call), pageable memory through the copy (asynchronous call)
    pinned2 = torch.empty((n, 4), dtype=torch.float64, pin_memory=True).numpy()
    pageable = np.empty((n, 4))
    with Context(Q, dims, free_energy=fe, **kw) as d:
        d.init(rho=rho)
        d.step_sums(n // 2, out=pinned2[: n // 2])
        d.step_sums_async(n - n // 2, pageable[n // 2:])
        d.synchronize()
        fd = d.get_populations()
    assert np.array_equal(fd, fb)
    assert np.array_equal(pinned2[: n // 2], got[: n // 2])
    assert np.array_equal(pageable[n // 2:], got[n // 2:])


# ---------------------------------------------------------------------------
# The D3Q19 force-model step on whole 32 x 8 tiles (X % 32 == 0, Y % 8 == 0,
# the shape of the 256^3 workload): one tile per row or column (the tile its
# own periodic neighbour), one and two planes, column ends.
# ---------------------------------------------------------------------------

TILED = [(32, 8, 12), (64, 16, 9), (32, 24, 5), (96, 8, 3), (32, 8, 1), (64, 8, 2)]


@pytest.mark.parametrize("dims", TILED)
def test_fp32_nonideal_tiled_100_steps(dims):
    """Against the oracle after 100 steps, FP32, thermal start on a random
    density: one tile per row or column (the tile its own neighbour), one and
    two planes, ragged column ends."""
    rho = inputs.uniform_density(dims, seed=3)
    got, want = _run_both(19, dims, "fp32", 100, fe=FE, rho=rho, thermal=True, kT=1e-6, omega_shear=1.1,
                          omega_bulk=0.9, omega_ghost=1.3, seed=3)
    assert np.abs(got - want).max() <= TOL["fp32"]


@pytest.mark.parametrize("dims", [(32, 8, 12), (64, 16, 5)])
def test_bf16_nonideal_tiled(dims):
    rho = inputs.uniform_density(dims, seed=5)
    got, want = _run_both(19, dims, "bf16", 20, fe=FE, rho=rho, thermal=True, kT=1e-6, omega_shear=1.0,
                          omega_bulk=1.0, omega_ghost=1.0, seed=4)
    assert np.abs(got - want).max() <= TOL["bf16"]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_tiled_z_chunk_changes_no_result(prec):
    """Columns of 1, 2, 3, 7, 16 or all 70 planes, or the tuned length, give
    bitwise the same populations on whole tiles."""
    dims = (64, 16, 70)
    rho = inputs.uniform_density(dims, seed=4)
    kw = dict(kT=1e-6, omega_shear=1.1, omega_bulk=1.0, omega_ghost=1.2, seed=9)
    out = []
    for zc in (0, 1, 2, 3, 7, 16, 70):
        with Context(19, dims, precision=prec, free_energy=FE, z_chunk=zc, **kw) as ctx:
            ctx.init(rho=rho)
            ctx.step(30)
            planes, tuning = ctx.z_chunk()
            assert not tuning and (planes == zc or not zc)
            out.append(ctx.get_populations())
    for f in out[1:]:
        assert np.array_equal(f, out[0])
    p = oracle.Params(Q=19, dims=dims, nonideal=True, **FE, **kw)
    want = oracle.run(p, oracle.init(p, rho=rho), 0, 30)
    assert np.abs(out[0] - want).max() <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_tiled_resume_is_bitwise(tmp_path, prec):
    """A run continued from a checkpoint, or from its state written back
    through flb_set_state_device, equals the uninterrupted run bit for bit
    (columns of 7 planes on whole tiles)."""
    import torch

    dims = (64, 16, 20)
    kw = dict(kT=1e-6, omega_shear=1.2, seed=8, free_energy=FE, z_chunk=7)
    rho = inputs.uniform_density(dims, seed=6)
    with Context(19, dims, precision=prec, **kw) as a:
        a.init(rho=rho, thermal=True)
        a.step(7)
        a.save(str(tmp_path / "c.flb"))
        g = torch.empty((19, int(np.prod(dims))), dtype=torch.float32 if prec == "fp32" else torch.bfloat16,
                        device="cuda")
        a.get_state_device(g.data_ptr())
        a.step(9)
        fa = a.get_populations()
        a.set_state_device(g.data_ptr())  # back to the state of step 7
        a.step_count = 7
        a.step(9)
        fa2 = a.get_populations()
    with Context.load(str(tmp_path / "c.flb"), z_chunk=7) as b:
        b.step(9)
        fb = b.get_populations()
    assert np.array_equal(fa, fb)
    assert np.array_equal(fa, fa2)
