"""Pins of the capillary-wave part of the oracle (Sec. VI and App. A of
arXiv 1012.3632): the total-free-energy force, the Landau double well, the
interface closed forms, the height fit and the height spectrum.  Each test
checks against something other than the oracle's own formula: a numerical
derivative of the printed f0, the paper's second form of a closed form, a
quadrature, the continuum force of Eq. (he-force), a library routine, or the
stationarity of the mean-field stripe under the oracle's own dynamics."""
import numpy as np
import pytest

from oracle import capillary as cap

CS2 = 1.0 / 3.0
RL, RV, BETA, KAPPA = 1.0, 0.5, 0.1, 0.08


def test_landau_mapping_is_derivative_of_f0():
    """A d + B d^3 with the mapped A, B, rho_c equals d f0 / d rho of Eq. (f0-bulk)
    (central differences of the printed double well)."""
    p = cap.landau(RL, RV, BETA)
    rho = np.linspace(0.3, 1.2, 37)
    h = 1e-5
    df = (cap.f0(rho + h, RL, RV, BETA) - cap.f0(rho - h, RL, RV, BETA)) / (2 * h)
    d = rho - p["rho_c"]
    assert np.allclose(p["A"] * d + p["B"] * d ** 3, df, rtol=0, atol=1e-10)
    # the two minima are the coexisting densities
    assert cap.f0(RL, RL, RV, BETA) == 0 and cap.f0(RV, RL, RV, BETA) == 0


def test_width_closed_forms_agree():
    """Eq. (interf-width) gives w twice: sqrt(8 kappa/beta)/(rho_L - rho_V) and
    4 sqrt(rho0 kappa)/c_s with beta = c_s^2 / (2 rho0 (rho_L - rho_V)^2)."""
    for rho0, cs in ((1.0, 0.265), (0.75, 0.2), (0.5, 0.3)):
        beta = cs ** 2 / (2 * rho0 * (RL - RV) ** 2)
        assert np.isclose(cap.width(RL, RV, beta, KAPPA), 4 * np.sqrt(rho0 * KAPPA) / cs, rtol=1e-14)
    assert abs(cap.width(RL, RV, BETA, KAPPA) - 5.06) < 0.01  # "approximately 5 l.u." (Fig. 2 caption)


def test_surface_tension_is_square_gradient_integral():
    """For the mean-field profile, sigma = kappa int (d rho/dy)^2 dy and the
    excess free energy int [f0 + kappa/2 rho'^2] dy are both Eq. (surf-tension)."""
    w = cap.width(RL, RV, BETA, KAPPA)
    y = np.linspace(-60, 60, 200001)
    rho = cap.profile(y, RL, RV, w)
    drho = np.gradient(rho, y)
    sig = cap.surface_tension(RL, RV, BETA, KAPPA)
    assert np.isclose(KAPPA * np.trapezoid(drho ** 2, y), sig, rtol=1e-6)
    assert np.isclose(np.trapezoid(cap.f0(rho, RL, RV, BETA) + 0.5 * KAPPA * drho ** 2, y), sig, rtol=1e-6)


@pytest.mark.parametrize("Q", [9, 19])
def test_total_free_energy_force_is_he_shan_doolen(orc, Q):
    """With psi the total bulk free energy, the oracle's force on a smooth density
    is the continuum force of Eq. (he-force),
      F = kappa rho rho''' - d/dx (p0 - rho cs^2),  p0 = rho f0' - f0,
    i.e. F = kappa rho rho''' - (rho f0''(rho) - cs^2) rho', up to the O(k^2)
    error of the lattice stencils."""
    X = 512
    p = orc.Params(Q=Q, dims=(X, 1, 1), nonideal=True, kappa=KAPPA, total=True, **cap.landau(RL, RV, BETA))
    x = np.arange(X)
    k = 2 * np.pi / X
    rho = 0.75 + 0.2 * np.sin(k * x) + 0.03 * np.cos(3 * k * x)
    d1 = 0.2 * k * np.cos(k * x) - 0.09 * k * np.sin(3 * k * x)
    d3 = -0.2 * k ** 3 * np.cos(k * x) + 0.81 * k ** 3 * np.sin(3 * k * x)
    f0pp = 2 * BETA * ((rho - RL) ** 2 + 4 * (rho - RL) * (rho - RV) + (rho - RV) ** 2)
    F_cont = KAPPA * rho * d3 - (rho * f0pp - CS2) * d1
    _, F = orc.density_force(p, orc.init(p, rho=rho))
    assert np.abs(F[0] - F_cont).max() <= 2e-3 * np.abs(F_cont).max()
    # the ideal-gas term matters: without it the force is off by cs^2 rho'
    p_ex = p.with_(total=False)
    _, F_ex = orc.density_force(p_ex, orc.init(p_ex, rho=rho))
    assert np.abs(F_ex[0] - F_cont).max() > 0.5 * np.abs(F_cont).max()


def test_mean_field_stripe_relaxes_to_a_flat_stationary_stripe(orc):
    """A D2Q9 stripe started from the mean-field profile of Eq. (denprof), with
    the Landau double well as total bulk free energy and kT = 0, relaxes to a
    stationary flat stripe: velocities vanish (no spurious currents at a flat
    interface), the heights stop moving, the bulk densities stay within 1 % of
    rho_L and rho_V and the interfaces within half a site of where they
    started.  (The lattice force model widens the interface from the
    mean-field w = 5.06 to about 8; see the design notes.)"""
    from paper_1012_3632_gb300 import inputs

    X, Y = 4, 64
    w = cap.width(RL, RV, BETA, KAPPA)
    p = orc.Params(Q=9, dims=(X, Y, 1), nonideal=True, kappa=KAPPA, total=True, **cap.landau(RL, RV, BETA))
    rho0 = inputs.stripe_density(X, Y, RL, RV, w, 16.0, 48.0)
    f4 = orc.run(p, orc.init(p, rho=rho0), 0, 4000)
    f6 = orc.run(p, f4, 4000, 2000)
    rho4, rho6 = (f.sum(axis=0).reshape(Y, X) for f in (f4, f6))
    assert abs(rho6[32].mean() - RL) < 0.02 * RL and abs(rho6[0].mean() - RV) < 0.02 * RV
    assert np.abs(rho6 - rho6[:, :1]).max() < 1e-12  # flat
    h4, h6 = (cap.interface_heights(r, RL, RV, w, (16.0, 48.0)) for r in (rho4, rho6))
    assert np.abs(h6 - np.array([[16.0], [48.0]])).max() < 0.5
    assert np.abs(h6 - h4).max() < 1e-4
    assert np.abs(orc.velocity(p, f6)).max() < 1e-6


def test_height_fit_recovers_known_shifts():
    """Noise-free stripe with known per-column heights: the fit returns them."""
    X, Y = 16, 80
    w = cap.width(RL, RV, BETA, KAPPA)
    rng = np.random.default_rng(2)
    h = np.stack([20 + rng.uniform(-2, 2, X), 60 + rng.uniform(-2, 2, X)])
    y = np.arange(Y)[:, None]
    rho = RV + 0.5 * (RL - RV) * (np.tanh(2 * (y - h[0]) / w) - np.tanh(2 * (y - h[1]) / w))
    got = cap.interface_heights(rho, RL, RV, w, (20.0, 60.0), window=8, iterations=12)
    assert np.abs(got - h).max() < 1e-9


def test_height_fit_equals_scipy_least_squares():
    """On a noisy column the Gauss-Newton fit reaches the minimizer that
    scipy.optimize.least_squares finds for the same objective."""
    from scipy.optimize import least_squares

    X, Y = 6, 80
    w = cap.width(RL, RV, BETA, KAPPA)
    rng = np.random.default_rng(5)
    y = np.arange(Y)[:, None]
    rho = RV + 0.5 * (RL - RV) * (np.tanh(2 * (y - 20.7) / w) - np.tanh(2 * (y - 59.2) / w)) * np.ones(X)
    rho = rho + 0.01 * rng.standard_normal(rho.shape)
    got = cap.interface_heights(rho, RL, RV, w, (20.0, 60.0), window=8, iterations=20)
    for i, (c, sign) in enumerate(((20, 1.0), (60, -1.0))):
        ys = np.arange(c - 8, c + 9)
        for x in range(X):
            res = least_squares(lambda hh: rho[ys, x] - cap.profile(ys - hh[0], RL, RV, w, sign), [float(c)],
                                xtol=1e-15, ftol=1e-15, gtol=1e-15)
            assert abs(res.x[0] - got[i, x]) < 5e-8


def test_height_spectrum_matches_numpy_fft():
    rng = np.random.default_rng(3)
    h = rng.standard_normal((2, 24)) + 5.0
    want = sum(np.abs(np.fft.fft(h[i] - h[i].mean())) ** 2 for i in range(2)) / (2 * 24)
    assert np.allclose(cap.height_spectrum(h), want, rtol=1e-12, atol=1e-14)


def test_capillary_spectrum_continuum_limit():
    """kT / (sigma (2 - 2 cos k)) -> kT / (sigma k^2) of Eq. (capill-static) as k -> 0."""
    sig = cap.surface_tension(RL, RV, BETA, KAPPA)
    k = np.array([1e-3, 1e-2])
    assert np.allclose(cap.capillary_spectrum(k, 1e-7, sig), 1e-7 / (sig * k ** 2), rtol=1e-4)


# --------------------------------------------------------------------------
# Modified-equilibrium (Swift) model, Sec. IV.C
# --------------------------------------------------------------------------

def test_swift_stripe_keeps_the_mean_field_interface(orc):
    """With the non-ideal pressure in the equilibrium (Eq. (meq-yeo) plus the
    square-gradient stress) and kT = 0, the D2Q9 stripe started from the
    mean-field profile stays on it: fitted width within 3 % of Eq. (interf-width),
    bulk densities within 1e-3 of rho_L and rho_V, interfaces fixed, velocities
    vanishing (mechanical equilibrium reduces to mu = const, as in the continuum)."""
    from scipy.optimize import least_squares

    from paper_1012_3632_gb300 import inputs

    X, Y = 4, 64
    w = cap.width(RL, RV, BETA, KAPPA)
    p = orc.Params(Q=9, dims=(X, Y, 1), nonideal=True, kappa=KAPPA, total=True, model=1, **cap.landau(RL, RV, BETA))
    f = orc.run(p, orc.init(p, rho=inputs.stripe_density(X, Y, RL, RV, w, 16.0, 48.0)), 0, 4000)
    rho = f.sum(axis=0).reshape(Y, X)[:, 0]
    ys = np.arange(4, 28)
    fit = least_squares(lambda q: rho[ys] - (0.5 * (q[2] + q[3]) + 0.5 * (q[2] - q[3]) * np.tanh(2 * (ys - q[0]) / q[1])),
                        [16.0, 5.0, 1.0, 0.5]).x
    assert abs(fit[1] / w - 1) < 0.03
    assert abs(fit[0] - 16.0) < 0.05
    assert abs(rho[32] - RL) < 1e-3 and abs(rho[0] - RV) < 1e-3
    assert np.abs(orc.velocity(p, f)).max() < 1e-8


def test_swift_modes_equilibrate_to_the_modified_equilibrium_covariance(orc):
    """Homogeneous Landau liquid (rho0 = 1, c_s^2 = 0.05) of the modified-equilibrium
    model with the k-dependent noise: every mode's <|dm_a(k)|^2>/V, averaged over
    k != 0, equals G_aa(k) of Eq. (f-correl-yeo) within 3 % (300 snapshots)."""
    from oracle import theory

    N = 16
    p = orc.Params(Q=9, dims=(N, N, 1), nonideal=True, kappa=KAPPA, total=True, model=1, kT=1e-6,
                   omega_shear=1.0, omega_bulk=1.1, omega_ghost=1.2, seed=5, **cap.landau(RL, RV, BETA))
    L = orc.lattice(9)
    f = orc.run(p, orc.init(p, rho=np.ones(N * N)), 0, 2000)
    acc = np.zeros((9, N * N))
    t = 2000
    for _ in range(300):
        f = orc.run(p, f, t, 10)
        t += 10
        for a in range(9):
            acc[a] += orc.structure_factor(p, f, a)
    acc /= 300
    k1 = 2 * np.pi * np.fft.fftfreq(N)
    G = np.zeros((9, N * N))
    for iy in range(N):
        for ix in range(N):
            _, K2 = theory.stencil_symbols(L, np.array([k1[ix], k1[iy]]))
            G[:, ix + N * iy] = np.diag(theory.G_swift(L, 1.0, 1e-6, 0.05 + KAPPA * K2)).real
    ratio = (acc[:, 1:] / G[:, 1:]).mean(axis=1)
    assert np.all(np.abs(ratio - 1) < 0.03), ratio
