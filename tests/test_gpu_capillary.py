"""Capillary-wave workload on the GPU (Sec. VI): the total-free-energy force,
interface heights and height spectrum, against the oracle; and the measured
spectrum of a fluctuating stripe against kT / (sigma (2 - 2 cos k)).

Tolerances: FP64 dynamics 1e-12 and FP32 2e-5 on the populations (as in
test_gpu_parity); heights 1e-9 (FP64 state) and 2e-5 (FP32 state: density
deviations stored in float, |d rho| ~ 1e-7 over a profile slope ~ 0.1).
"""
import numpy as np
import pytest

import oracle
from oracle import capillary as cap
from paper_1012_3632_gb300 import Context, inputs, interface_fit, landau_free_energy
from paper_1012_3632_gb300.flb import FLBError

pytestmark = pytest.mark.gpu

RL, RV, BETA, KAPPA = 1.0, 0.5, 0.1, 0.08
W = cap.width(RL, RV, BETA, KAPPA)
TOL = {"fp64": 1e-12, "fp32": 2e-5}


def _fe():
    fe = landau_free_energy(RL, RV, BETA, KAPPA)
    ref = dict(cap.landau(RL, RV, BETA), kappa=KAPPA, total=True)
    assert all(np.isclose(fe[k], ref[k], rtol=1e-15) for k in ("A", "B", "rho_c", "kappa")) and fe["total"]
    return fe


@pytest.mark.parametrize("Q,dims,prec", [
    (9, (24, 40, 1), "fp64"), (9, (24, 40, 1), "fp32"), (9, (7, 33, 1), "fp32"),
    (19, (8, 28, 4), "fp64"),
    (19, (16, 28, 5), "fp32"), (19, (9, 28, 3), "fp32"),  # one-site z-marching step
])
def test_total_free_energy_parity(Q, dims, prec):
    """Landau double well as total bulk free energy (F = -rho grad mu + cs^2 grad rho):
    a fluctuating stripe, 40 steps, GPU against the oracle."""
    X, Y, Z = dims
    rho = inputs.stripe_density(X, Y, RL, RV, W, 0.25 * Y, 0.75 * Y, amp=0.5, modes=2, seed=4)
    rho = np.broadcast_to(rho, (Z, Y, X)).ravel()
    fe = _fe()
    kw = dict(kT=1e-6, omega_shear=1.1, omega_bulk=1.0, omega_ghost=1.2, seed=9)
    with Context(Q, dims, precision=prec, free_energy=fe, **kw) as ctx:
        ctx.init(rho=rho)
        ctx.step(40)
        got = ctx.get_populations()
    p = oracle.Params(Q=Q, dims=dims, nonideal=True, **{k: fe[k] for k in ("A", "B", "rho_c", "kappa", "total")},
                      **kw)
    want = oracle.run(p, oracle.init(p, rho=rho), 0, 40)
    assert np.abs(got - want).max() <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_interface_heights_parity(prec):
    """flb_interface_heights on a stripe with random per-column heights equals
    the oracle's fit of the same density field."""
    X, Y = 48, 64
    rho = inputs.stripe_density(X, Y, RL, RV, W, 16.3, 47.6, amp=1.5, modes=5, seed=2)
    fit = interface_fit(RL, RV, W, (16.3, 47.6), window=8, iterations=8)
    with Context(9, (X, Y, 1), 1.0, precision=prec, free_energy=_fe()) as ctx:
        ctx.init(rho=rho.ravel())
        got = ctx.interface_heights(fit)
    want = cap.interface_heights(rho, RL, RV, W, (16.3, 47.6), window=8, iterations=8)
    assert np.abs(got - want).max() <= (1e-9 if prec == "fp64" else 2e-5)


def test_height_spectrum_parity_and_accumulation():
    """flb_height_spectrum: one snapshot equals the oracle's spectrum of the
    oracle's heights (X = 60 uses the mixed-radix FFT, X = 14 = 2 * 7 the naive
    DFT); accumulated snapshots of an evolving stripe give the mean of the
    single-snapshot spectra; flb_init and flb_reset_accumulators clear the count."""
    for X in (60, 14):
        Y = 64
        fit = interface_fit(RL, RV, W, (16.0, 48.0), window=8, iterations=8)
        rhos = [inputs.stripe_density(X, Y, RL, RV, W, 16.0, 48.0, amp=1.0, modes=4, seed=s) for s in (1, 2, 3)]
        with Context(9, (X, Y, 1), 1.0, kT=1e-6, precision="fp64", free_energy=_fe()) as ctx:
            for r in rhos:
                ctx.init(rho=r.ravel())
                got = ctx.height_spectrum(fit, accumulate=False)
                want = cap.height_spectrum(cap.interface_heights(r, RL, RV, W, (16.0, 48.0)))
                assert np.allclose(got, want, rtol=1e-9, atol=1e-14)
            one = []
            for _ in range(3):
                ctx.step(5)
                one.append(ctx.height_spectrum(fit, accumulate=False))
                acc = ctx.height_spectrum(fit, accumulate=True)
            assert ctx.snapshot_count(-2) == 3
            assert np.allclose(acc, np.mean(one, axis=0), rtol=1e-12, atol=1e-15)
            ctx.reset_accumulators()
            assert ctx.snapshot_count(-2) == 0


def test_fit_arguments_are_checked():
    fit = interface_fit(RL, RV, W, (16.0, 48.0), window=8, iterations=8)
    with Context(19, (8, 8, 8), 1.0, precision="fp32", free_energy=_fe()) as ctx:
        with pytest.raises(FLBError):
            ctx.interface_heights(fit)  # D3Q19
    with Context(9, (16, 12, 1), 1.0, precision="fp32", free_energy=_fe()) as ctx:
        with pytest.raises(FLBError):
            ctx.interface_heights(fit)  # window 8 needs Y >= 17
        for bad in (interface_fit(RL, RV, 0.0, (3.0, 8.0), window=2), interface_fit(RL, RL, W, (3.0, 8.0), window=2),
                    interface_fit(RL, RV, W, (3.0, 8.0), window=2, iterations=0)):
            with pytest.raises(FLBError):
                ctx.height_spectrum(bad)


def test_stripe_height_spectrum_scales_as_capillary_waves():
    """A fluctuating D2Q9 stripe (256 x 128, thickness 64, the Landau fluid of
    Sec. VI, tau = 1): the height spectrum has the capillary form
    S(k) (2 - 2 cos k) = kT / sigma_eff, flat in k for k <= 0.6 (band means
    agree within 10 %), and it is linear in kT (doubling kT doubles S within
    3 %).  The stiffness sigma_eff of this lattice force model is reported,
    not pinned: see the design notes."""
    from paper_1012_3632_gb300.capillary import run_stripe

    out = {}
    for kT in (1e-7, 2e-7):
        k, S, n, _ = run_stripe(steps=200000, snapshots=800, X=256, Y=128, thickness=64, kT=kT)
        assert n == 800
        out[kT] = S
    k = k[1:129]
    y = out[1e-7][1:129] * (2 - 2 * np.cos(k)) / 1e-7  # 1 / sigma_eff(k)
    lo, hi = y[k <= 0.3].mean(), y[(k > 0.3) & (k <= 0.6)].mean()
    assert abs(lo / hi - 1) < 0.1, (lo, hi)
    assert 0.25 < (1 / lo) / cap.surface_tension(RL, RV, BETA, KAPPA) < 4.0
    ratio = out[2e-7][1:129] / out[1e-7][1:129]
    assert abs(ratio[k <= 1.0].mean() - 2) < 0.06


def test_momentum_equipartition_in_the_landau_fluid():
    """Homogeneous liquid (rho = rho_L) of the Landau fluid as total free energy:
    the momentum fluctuations are at kT, <|j_x(k)|^2> / V = rho kT within 8 %
    for 0 < |k| < 1.5 (Sec. IV.B: momentum is equilibrated at all k)."""
    N, kT = 64, 1e-7
    with Context(9, (N, N, 1), 1.0, kT=kT, free_energy=_fe(), seed=3, precision="fp64") as c:
        c.init(rho=np.full(N * N, RL))
        c.step(5000)
        for _ in range(200):
            c.step(25)
            Sj = c.structure_factor(1, accumulate=True)
    kx = 2 * np.pi * np.fft.fftfreq(N)
    kk = np.hypot(*np.meshgrid(kx, kx)).ravel()
    m = (kk > 0) & (kk < 1.5)
    assert abs(Sj[m].mean() / (RL * kT) - 1) < 0.08
