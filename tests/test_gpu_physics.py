"""Statistical and hydrodynamic checks of the GPU path against what the paper fixes.

- Equal-time variance of every mode, ghosts included, equals its ideal-gas FDT
  value rho0 kT N_a / cs^2 (Eqs. (G-ideal), (mu-ideal), (noise-lbe)): mode
  temperatures T_a = cs^2 <dm_a^2> / (rho0 N_a) = kT within 1% over 10^4 steps
  on the 128^3 shear-wave workload.
- Shear-wave amplitude decays as exp(-nu k^2 t), nu = cs^2 (1/omega - 1/2)
  (App. B with the lambda^LB map of Sec. V).
- Ideal gas: S(k) = rho0 kT / cs^2 at every k (Eq. (S-ideal)).
- Force-based non-ideal fluid: momentum and every non-conserved mode keep their
  ideal variances (Eq. (g-mat-forcing)); S(k) follows the Ornstein-Zernike form
  rho0 kT / c_s^2(k), c_s^2(k) = cs^2 + rho0 psi''(rho0) + kappa rho0 k^2
  (Eq. (he-cs2)) at small k.
"""
import numpy as np
import pytest

from paper_1012_3632_gb300 import MODE_VAR, RHO, U, Context, inputs

pytestmark = pytest.mark.gpu

CS2 = 1.0 / 3.0
N19 = np.array([1, 1 / 3, 1 / 3, 1 / 3, 2 / 3, 4 / 3, 4 / 9, 1 / 9, 1 / 9, 1 / 9, 2 / 27, 2 / 27, 2 / 27,
                2 / 9, 2 / 9, 2 / 9, 2 / 9, 1 / 3, 1 / 9])


def _kgrid(dims):
    ks = [2 * np.pi * np.fft.fftfreq(n) for n in dims]  # components in [-pi, pi)
    kz, ky, kx = np.meshgrid(ks[2], ks[1], ks[0], indexing="ij")
    return kx.reshape(-1), ky.reshape(-1), kz.reshape(-1)


@pytest.fixture(scope="module")
def ideal128_run():
    """128^3 D3Q19 ideal gas, FP32, kT = 1e-5, rates (1.2, 1.0, 1.0), shear wave
    u_x = 1e-3 sin(2 pi z / 128) plus thermal start, 10^4 steps; snapshots
    every 100 steps."""
    dims = (128, 128, 128)
    kT, om = 1e-5, 1.2
    u = inputs.shear_wave(dims, amp=1e-3)
    z = np.repeat(np.arange(dims[2]), dims[0] * dims[1])
    sinz = np.sin(2 * np.pi * z / dims[2])
    amps, times = [], []
    with Context(19, dims, om, 1.0, 1.0, kT=kT, seed=2, precision="fp32") as ctx:
        ctx.init(u=u, thermal=True)
        var = None
        for t in range(100, 10001, 100):
            ctx.step(100)
            var = ctx.moments(MODE_VAR)
            ctx.structure_factor(1, accumulate=True, fetch=False)
            ux = ctx.moments(U)[0]
            amps.append(2.0 * (ux @ sinz) / ux.size)
            times.append(t)
        Sjx = ctx.structure_factor(1, accumulate=True)  # one more snapshot, returns the mean
    return dict(dims=dims, kT=kT, om=om, var=var, Sjx=Sjx, amps=np.array(amps), times=np.array(times))


def test_mode_temperatures_within_one_percent(ideal128_run):
    r = ideal128_run
    V = np.prod(r["dims"])
    T = CS2 * r["var"] / N19 / r["kT"]
    # j_x carries the deterministic wave: take its variance from the spectrum
    # without k = 0 and the wave's two wavevectors (0, 0, +-1)
    kx, ky, kz = _kgrid(r["dims"])
    wave = (kx == 0) & (ky == 0) & (np.abs(np.abs(kz) - 2 * np.pi / r["dims"][2]) < 1e-12)
    keep = ~wave
    keep[0] = False
    var_jx = r["Sjx"][keep].sum() / V * V / keep.sum()
    T[1] = CS2 * var_jx / N19[1] / r["kT"]
    assert np.all(np.abs(T - 1.0) < 0.01), T


def test_shear_wave_decay_rate(ideal128_run):
    r = ideal128_run
    k = 2 * np.pi / r["dims"][2]
    nu = CS2 * (1.0 / r["om"] - 0.5)
    # the thermal fluctuation of the same Fourier mode (~3e-6, correlated over
    # ~1/(nu k^2) = 3700 steps) rides on the amplitude: fit while the wave is
    # at least 40% of its initial size
    a = r["amps"]
    sel = a > 0.4 * a[0]
    rate = -np.polyfit(r["times"][sel], np.log(a[sel]), 1)[0]
    assert abs(rate / (nu * k * k) - 1) < 0.01, (rate, nu * k * k)


def test_ideal_gas_structure_factor_flat():
    """S(k) = rho0 kT / cs^2 for every k of a thermalised ideal gas (64^3, 3000 steps)."""
    dims = (64, 64, 64)
    kT = 1e-5
    with Context(19, dims, 1.3, 0.8, 1.5, kT=kT, seed=11, precision="fp32") as ctx:
        ctx.init(thermal=True)
        for _ in range(60):
            ctx.step(50)
            S = ctx.structure_factor(0, accumulate=True)
    ratio = S[1:] / (kT / CS2)
    assert abs(ratio.mean() - 1) < 0.01, ratio.mean()
    kx, ky, kz = _kgrid(dims)
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)[1:]
    for lo, hi in ((0.0, 1.0), (1.0, 2.0), (2.0, 3.0), (3.0, 6.0)):
        m = (kk >= lo) & (kk < hi)
        assert abs(ratio[m].mean() - 1) < 0.03, (lo, hi, ratio[m].mean())


def test_nonideal_fluid_equilibrium():
    """Force-based fluid (A=-0.01, B=0.1, rho_c=1, kappa=0.02) at 64^3, FP32,
    kT = 1e-5, thermal start: momentum and non-conserved modes at kT; density
    structure factor Ornstein-Zernike at |k| < 0.5."""
    dims = (64, 64, 64)
    kT = 1e-5
    A, kappa = -0.01, 0.02
    fe = dict(A=A, B=0.1, rho_c=1.0, kappa=kappa)
    with Context(19, dims, 1.0, 1.0, 1.0, kT=kT, seed=13, precision="fp32", free_energy=fe) as ctx:
        ctx.init(thermal=True)
        ctx.step(2000)
        for _ in range(200):
            ctx.step(100)
            S = ctx.structure_factor(0, accumulate=True, fetch=False)
            var = ctx.moments(MODE_VAR)
        S = ctx.structure_factor(0, accumulate=True)
    T = CS2 * var / N19 / kT
    assert np.all(np.abs(T[1:4] - 1) < 0.01), T[1:4]          # momentum
    assert np.all(np.abs(T[4:] - 1) < 0.02), T[4:]            # stress and ghost modes
    kx, ky, kz = _kgrid(dims)
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    small = (k2 > 0) & (k2 < 0.25)
    oz = kT / (CS2 + A + kappa * k2[small])
    ratio = S[small] / oz
    assert abs(ratio.mean() - 1) < 0.02, ratio.mean()


def test_sound_wave_attenuation_128():
    """D3Q19 ideal gas 128^3, FP32, kT = 0, rates (shear 1.3, bulk 0.8, ghost 1.7):
    a density wave 1e-4 cos(2 pi x / 128) propagates at cs and decays at the
    rate of the App. B viscosities with the Sec. V map, within 0.5 % (the same
    closed form that pins the oracle; it fixes which mode carries omega_bulk)."""
    from hydro_theory import fit_sound_wave, sound_wave_rates

    dims = (128, 128, 128)
    om = dict(omega_shear=1.3, omega_bulk=0.8, omega_ghost=1.7)
    k = 2 * np.pi / dims[0]
    x = np.tile(np.arange(dims[0]), dims[1] * dims[2])
    e = np.exp(-1j * k * x)
    ts, rk, jk = [], [], []
    with Context(19, dims, om["omega_shear"], om["omega_bulk"], om["omega_ghost"], kT=0.0, seed=5,
                 precision="fp32") as ctx:
        ctx.init(rho=1.0 + 1e-4 * np.cos(k * x))
        ctx.step(100)
        for t in range(100, 1501, 20):
            rho = ctx.moments(RHO)
            jx = ctx.moments(U)[0] * rho
            ts.append(t)
            rk.append((rho - 1.0) @ e)
            jk.append(jx @ e)
            ctx.step(20)
    gamma, omega = fit_sound_wave(np.array(ts), rk, jk)
    gamma_th, omega_th = sound_wave_rates(3, k, om["omega_shear"], om["omega_bulk"])
    assert abs(gamma / gamma_th - 1) < 5e-3, (gamma, gamma_th)
    assert abs(omega / omega_th - 1) < 5e-3, (omega, omega_th)


# --------------------------------------------------------------------------
# BF16 storage: kept only if every mode temperature stays within 1 % of kT
# --------------------------------------------------------------------------

def _mode_temperatures_ideal128(precision):
    """The 128^3 shear-wave workload of ideal128_run (kT = 1e-5, rates
    (1.2, 1, 1), shear wave + thermal start, 10^4 steps, 100 snapshots), with
    the given storage; j_x's variance from its spectrum without the wave."""
    dims = (128, 128, 128)
    kT = 1e-5
    u = inputs.shear_wave(dims, amp=1e-3)
    with Context(19, dims, 1.2, 1.0, 1.0, kT=kT, seed=2, precision=precision) as ctx:
        ctx.init(u=u, thermal=True)
        for _ in range(100):
            ctx.step(100)
            var = ctx.moments(MODE_VAR)
            ctx.structure_factor(1, accumulate=True, fetch=False)
        Sjx = ctx.structure_factor(1, accumulate=True)
    V = np.prod(dims)
    T = CS2 * var / N19 / kT
    kx, ky, kz = _kgrid(dims)
    wave = (kx == 0) & (ky == 0) & (np.abs(np.abs(kz) - 2 * np.pi / dims[2]) < 1e-12)
    keep = ~wave
    keep[0] = False
    T[1] = CS2 * (Sjx[keep].sum() / keep.sum()) / N19[1] / kT
    return T


def test_bf16_mode_temperatures_within_one_percent():
    """BF16 population storage on the 128^3 ideal-gas workload: every mode
    temperature, ghosts included, within 1 % of kT over 10^4 steps -- the
    condition under which the BF16 variant is kept (FDT of Eq. (noise-lbe),
    equal-time variances of Eqs. (G-ideal), (mu-ideal))."""
    T = _mode_temperatures_ideal128("bf16")
    assert np.all(np.abs(T - 1.0) < 0.01), T


def _nonideal64_temperatures(precision, kT):
    dims = (64, 64, 64)
    fe = dict(A=-0.01, B=0.1, rho_c=1.0, kappa=0.02)
    with Context(19, dims, 1.0, 1.0, 1.0, kT=kT, seed=13, precision=precision, free_energy=fe) as ctx:
        ctx.init(thermal=True)
        ctx.step(2000)
        for _ in range(200):
            ctx.step(100)
            var = ctx.moments(MODE_VAR)
    return CS2 * var / N19 / kT


def test_bf16_nonideal_mode_temperatures_at_headline_kT():
    """Force-based fluid at the 256^3 workload's kT = 1e-6 (64^3, same model):
    with BF16 storage the momentum stays within 1 % of kT, every mode
    temperature within 1 % of the FP32-storage run on the same seed (the
    storage rounding is the only difference), and the stress and ghost modes
    within the same 2 % of kT as with FP32 (Eq. (g-mat-forcing))."""
    kT = 1e-6
    T32 = _nonideal64_temperatures("fp32", kT)
    T16 = _nonideal64_temperatures("bf16", kT)
    assert np.all(np.abs(T16[1:4] - 1) < 0.01), T16[1:4]
    assert np.all(np.abs(T16[1:] / T32[1:] - 1) < 0.01), (T16, T32)
    assert np.all(np.abs(T16[4:] - 1) < 0.02), T16[4:]


# --------------------------------------------------------------------------
# The equilibration test of Sec. VI (Fig. 1): ratios <|dm_a(k)|^2> / G_aa(k)
# --------------------------------------------------------------------------

def _d2q9_lattice_k2(kx, ky):
    """Symbol K2(k) of the isotropic D2Q9 Laplacian used by the force stencils."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    c = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
    kc = c[:, 0][:, None, None] * kx + c[:, 1][:, None, None] * ky
    return 2.0 / CS2 * (w[:, None, None] * (1.0 - np.cos(kc))).sum(0)


def test_equilibration_ratios_fig1_protocol():
    """The protocol of the paper's equilibration test: D2Q9 128x128, force-based
    fluid with c_s = 0.265 (psi the excess free energy, psi'' = c_s^2 - cs^2,
    Eq. (he-cs2)), kappa = 0.08, kT = 1e-7, tau = 1, 400 snapshots; the ratio
    of each mode's equal-time variance <|dm_a(k)|^2> to G_aa(k) of
    Eq. (g-mat-forcing), averaged over |k| bands.  What the theory fixes:
    transverse momentum, stress and ghost modes at their ideal-gas values
    (ratio 1) at every k, the density at Ornstein-Zernike S(k) = rho0 kT /
    c_s^2(k) as k -> 0.  What the paper reports for its force model, and what
    this discretisation shows too: the density (and to a lesser extent the
    longitudinal momentum) mis-equilibrates at all but the smallest
    wavenumbers."""
    X = Y = 128
    cs, kappa, kT = 0.265, 0.08, 1e-7
    fe = dict(A=cs * cs - CS2, B=0.0, rho_c=1.0, kappa=kappa)
    N9 = np.array([1, 1 / 3, 1 / 3, 4, 4 / 9, 1 / 9, 2 / 3, 2 / 3, 16])
    ky, kx = np.meshgrid(2 * np.pi * np.fft.fftfreq(Y), 2 * np.pi * np.fft.fftfreq(X), indexing="ij")
    kk = np.sqrt(kx ** 2 + ky ** 2)
    kn = np.where(kk > 0, kk, 1.0)
    nsnap = 400
    jl = np.zeros((Y, X))
    jt = np.zeros((Y, X))
    S = {}
    with Context(9, (X, Y, 1), 1.0, 1.0, 1.0, kT=kT, seed=21, precision="fp32", free_energy=fe) as ctx:
        ctx.init(thermal=True)
        ctx.step(5000)
        for s in range(nsnap):
            ctx.step(100)
            last = s == nsnap - 1
            for a in (0, 3, 4, 5, 6, 7, 8):
                out = ctx.structure_factor(a, accumulate=True, fetch=last)
                if last:
                    S[a] = out.reshape(Y, X)
            rho = ctx.moments(RHO)
            j = (ctx.moments(U) * rho).reshape(2, Y, X)
            fx, fy = np.fft.fft2(j[0]), np.fft.fft2(j[1])
            jl += np.abs((kx * fx + ky * fy) / kn) ** 2 / (X * Y)
            jt += np.abs((-ky * fx + kx * fy) / kn) ** 2 / (X * Y)
    jl /= nsnap
    jt /= nsnap

    def band(r, lo, hi):
        m = (kk > lo) & (kk <= hi)
        return r[m].mean()

    bands = [(0.1, 0.2), (0.2, 0.35), (0.35, 0.5), (0.5, 1.0), (1.0, 1.5), (1.5, 2.0), (2.0, 2.5), (2.5, 3.2),
             (3.2, 4.5)]
    # statistics: 40 000 steps of snapshots; the slowest modes of the two
    # smallest bands (transverse momentum, |k| < 0.35, some 70 wavevectors
    # decorrelating over 1/(nu k^2) ~ 270-1000 steps) carry ~2-3 % errors
    for lo, hi in bands:
        tol = 0.06 if hi <= 0.35 else 0.02
        assert abs(band(jt / kT, lo, hi) - 1) < tol, ("j_t", lo, hi)
        assert abs(band(jl / kT, lo, hi) - 1) < 0.07, ("j_par", lo, hi)
        for a in (3, 4, 5, 6, 7, 8):
            r = band(S[a] / (kT * N9[a] / CS2), lo, hi)
            assert abs(r - 1) < (tol if hi <= 2.5 else 0.06), (a, lo, hi, r)
    oz = S[0] / (kT / (cs * cs + kappa * _d2q9_lattice_k2(kx, ky)))
    assert abs(band(oz, 0.1, 0.2) - 1) < 0.05
    # the density's mis-equilibration away from k -> 0 (Sec. VI, Fig. 1a)
    assert band(oz, 0.5, 1.5) < 0.9
