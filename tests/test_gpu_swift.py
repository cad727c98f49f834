"""Modified-equilibrium model (Sec. IV.C) on the GPU: the non-ideal pressure in
the D2Q9 equilibrium and the k-dependent e/eps noise coloured by FFT.

Parity with the oracle (same Philox draws; the oracle colours the noise with a
direct DFT, the GPU with its mixed-radix FFT): 1e-12 (FP64), 2e-5 (FP32) on the
populations.  Physics: the modes of a homogeneous Landau liquid equilibrate to
G of Eq. (f-correl-yeo) with the noise of Eq. (noise-yeo) (corner from the FDT).
"""
import numpy as np
import pytest

import oracle
from oracle import capillary as cap
from oracle import theory
from paper_1012_3632_gb300 import Context, inputs, landau_free_energy
from paper_1012_3632_gb300.flb import FLBError

pytestmark = pytest.mark.gpu

RL, RV, BETA, KAPPA = 1.0, 0.5, 0.1, 0.08
TOL = {"fp64": 1e-12, "fp32": 2e-5}


def _fe(model=1):
    return dict(landau_free_energy(RL, RV, BETA, KAPPA), model=model)


def _oracle_params(dims, **kw):
    fe = _fe()
    return oracle.Params(Q=9, dims=dims, nonideal=True, A=fe["A"], B=fe["B"], rho_c=fe["rho_c"], kappa=fe["kappa"],
                         total=True, model=1, **kw)


@pytest.mark.parametrize("dims,prec,kT", [
    ((16, 12, 1), "fp64", 1e-6), ((16, 12, 1), "fp32", 1e-6),
    ((15, 10, 1), "fp64", 1e-6),   # mixed-radix lengths 3 * 5 and 2 * 5
    ((14, 9, 1), "fp64", 1e-6),    # 14 = 2 * 7: the direct-DFT path
    ((16, 12, 1), "fp64", 0.0),
])
def test_swift_parity_homogeneous(dims, prec, kT):
    kw = dict(kT=kT, omega_shear=1.1, omega_bulk=0.9, omega_ghost=1.3, seed=8)
    rho = inputs.uniform_density(dims, rho_c=1.0, amp=0.02, seed=2)
    with Context(9, dims, precision=prec, free_energy=_fe(), **kw) as ctx:
        ctx.init(rho=rho)
        ctx.step(40)
        got = ctx.get_populations()
    p = _oracle_params(dims, **kw)
    want = oracle.run(p, oracle.init(p, rho=rho), 0, 40)
    assert np.abs(got - want).max() <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_swift_parity_stripe(prec):
    """An inhomogeneous state (stripe with displaced interfaces): the pressure and
    square-gradient stress of the equilibrium, and the noise, against the oracle."""
    X, Y = 20, 32
    w = cap.width(RL, RV, BETA, KAPPA)
    rho = inputs.stripe_density(X, Y, RL, RV, w, 8.0, 24.0, amp=0.7, modes=3, seed=5).ravel()
    kw = dict(kT=1e-7, omega_shear=1.0, omega_bulk=1.0, omega_ghost=1.0, seed=3)
    with Context(9, (X, Y, 1), precision=prec, free_energy=_fe(), **kw) as ctx:
        ctx.init(rho=rho)
        ctx.step(30)
        got = ctx.get_populations()
    p = _oracle_params((X, Y, 1), **kw)
    want = oracle.run(p, oracle.init(p, rho=rho), 0, 30)
    assert np.abs(got - want).max() <= TOL[prec]


def test_swift_modes_equilibrate():
    """Homogeneous Landau liquid (rho0 = 1, c_s^2 = 0.05), 64 x 64, FP64: every
    mode's <|dm_a(k)|^2>/V averaged over k != 0 equals G_aa(k) of
    Eq. (f-correl-yeo) within 3 %, and within 10 % in each |k| band."""
    N, kT = 64, 1e-6
    L = oracle.lattice(9)
    with Context(9, (N, N, 1), 1.0, 1.1, 1.2, kT=kT, free_energy=_fe(), seed=5, precision="fp64") as c:
        c.init(rho=np.ones(N * N))
        c.step(4000)
        for _ in range(400):
            c.step(20)
            S = [c.structure_factor(a, accumulate=True) for a in range(9)]
    S = np.array(S)
    k1 = 2 * np.pi * np.fft.fftfreq(N)
    G = np.zeros((9, N * N))
    kk = np.zeros(N * N)
    for iy in range(N):
        for ix in range(N):
            k = np.array([k1[ix], k1[iy]])
            _, K2 = theory.stencil_symbols(L, k)
            G[:, ix + N * iy] = np.diag(theory.G_swift(L, 1.0, kT, 0.05 + KAPPA * K2)).real
            kk[ix + N * iy] = np.hypot(*k)
    r = S[:, 1:] / G[:, 1:]
    assert np.all(np.abs(r.mean(axis=1) - 1) < 0.03), r.mean(axis=1)
    for lo, hi in ((0, 1.0), (1.0, 2.0), (2.0, 4.5)):
        m = (kk[1:] > lo) & (kk[1:] <= hi)
        assert np.all(np.abs(r[:, m].mean(axis=1) - 1) < 0.1), (lo, r[:, m].mean(axis=1))


def test_swift_arguments_are_checked():
    with pytest.raises(FLBError):
        Context(19, (8, 8, 8), 1.0, kT=1e-6, free_energy=_fe())  # D2Q9 only
    with pytest.raises(FLBError):
        Context(9, (8, 8, 1), 1.0, kT=1e-6, free_energy=dict(_fe(), model=2))
    # kappa large enough that 2 - 3 c_s^2(k) < 0 at the largest k: no covariance
    with pytest.raises(FLBError):
        Context(9, (8, 8, 1), 1.0, kT=1e-6, free_energy=dict(_fe(), kappa=0.5))


def test_swift_capillary_spectrum_matches_capillary_theory():
    """Fluctuating D2Q9 stripe (256 x 128, thickness 64) of the modified-equilibrium
    Landau fluid, tau = 1, kT = 1e-7: the height spectrum averaged over
    0 < k <= 0.6 equals kT / (sigma (2 - 2 cos k)) of Eq. (capill-static) with
    the mean-field sigma of Eq. (surf-tension) within 15 % (Sec. VI: the
    modified-equilibrium model reproduces the capillary spectrum)."""
    from paper_1012_3632_gb300.capillary import run_stripe

    k, S, n, _ = run_stripe(steps=200000, snapshots=800, X=256, Y=128, thickness=64, kT=1e-7, model=1)
    assert n == 800
    sig = cap.surface_tension(RL, RV, BETA, KAPPA)
    m = (k > 0) & (k <= 0.6)
    ratio = (S[m] / cap.capillary_spectrum(k[m], 1e-7, sig)).mean()
    assert abs(ratio - 1) < 0.15, ratio
