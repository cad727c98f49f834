"""Linear fluctuation theory of the discrete Boltzmann equation, in numpy.

TEST INFRASTRUCTURE (test aid for pinning the noise formula of the oracle and
for the expected values of the statistical tests).  Every function follows a
numbered equation of Gross, Cates, Varnik & Adhikari (arXiv 1012.3632):

  advection A(k)          Eq. (adv-fourier), App. C; (T^-1)_ib = w_i T_bi / N_b
  relaxation Lambda       Eq. (relax-eigenv); lambda_a = 0 on conserved modes
  ideal-gas G             Eqs. (G-ideal), (mu-ideal): G = mu rho0 diag(N), mu = kT/cs^2
  force operator K(k)     Eqs. (force-mom), (lin-intforce): dF = i k [c_s^2(k) - cs^2] drho
  force-model G           Eqs. (s-nonideal), (g-mat-forcing)
  FDT                     Eq. (dbe-fdt): Xi = L G + G L^dagger, L = A + Lambda - K
  lambda^LB map           Sec. V: lambda^LB = 2 lambda / (2 + lambda)
  lattice noise           Eq. (noise-lbe): rho0 kT (2 - w) w N_a / cs^2
  modified equilibrium    Sec. IV.C (D2Q9, App. B basis): Eqs. (meq-yeo),
                          (f-correl-yeo), the operator L(k) and Eq. (noise-yeo)

The Fourier convention is the paper's, f(r) = int f(k) exp(-i k.r) dk.
"""
from __future__ import annotations

import numpy as np


def advection(L, k) -> np.ndarray:
    """A_ab(k) = -i k . T_aj c_j (T^-1)_jb, Eq. (adv-fourier)."""
    k = np.zeros(3) if k is None else np.pad(np.asarray(k, float), (0, 3 - len(k)))
    kc = L.c @ k
    return -1j * (L.T * kc[None, :]) @ L.Tinv


def relaxation(L, lam_bulk, lam_shear, lam_ghost) -> np.ndarray:
    """diag(lambda_a), zero on the conserved modes (Eq. (relax-eigenv))."""
    rate = {0: 0.0, 1: lam_bulk, 2: lam_shear, 3: lam_ghost}
    return np.diag([rate[int(c)] for c in L.cls]).astype(complex)


def mu_mass(L, kT) -> float:
    """Eq. (mu-ideal)."""
    return kT / L.cs2


def G_ideal(L, rho0, kT) -> np.ndarray:
    """Eq. (G-ideal): G_ab = mu rho0 N_a delta_ab."""
    return np.diag(mu_mass(L, kT) * rho0 * L.N).astype(complex)


def K_force(L, k, cs2k) -> np.ndarray:
    """Linear forcing operator in moment space (Eq. (force-mom) with Eq. (lin-intforce)):
    only the momentum rows pick up i k_alpha [c_s^2(k) - cs^2] times the density."""
    k = np.pad(np.asarray(k, float), (0, 3 - len(k)))
    K = np.zeros((L.Q, L.Q), complex)
    for d in range(L.D):
        K[1 + d, 0] = 1j * k[d] * (cs2k - L.cs2)
    return K


def G_force(L, rho0, kT, cs2k) -> np.ndarray:
    """Eq. (g-mat-forcing) with S(k) = rho0 kT / c_s^2(k) (Eq. (s-nonideal))."""
    G = G_ideal(L, rho0, kT)
    G[0, 0] = rho0 * kT / cs2k
    return G


def fdt_noise(Lmat, G) -> np.ndarray:
    """Eq. (dbe-fdt): Xi = L G + G L^dagger."""
    return Lmat @ G + G @ Lmat.conj().T


def lambda_lb(lam):
    """Sec. V: lambda^LB = 2 lambda / (2 + lambda)."""
    return 2.0 * lam / (2.0 + lam)


def lambda_dbe(omega):
    """Inverse of lambda_lb: the DBE rate whose lattice rate is omega."""
    return 2.0 * omega / (2.0 - omega)


def lattice_noise_variance(L, rho0, kT, omega_a, a) -> float:
    """Eq. (noise-lbe) with Delta V = 1: variance of the lattice noise of mode a."""
    return rho0 * kT / L.cs2 * (2.0 - omega_a) * omega_a * L.N[a]


def shear_viscosity(omega, cs2=1.0 / 3.0):
    """nu = cs^2 / lambda (App. B) with lambda the DBE rate of the lattice rate omega:
    nu = cs^2 (1/omega - 1/2)."""
    return cs2 / lambda_dbe(omega)


def stencil_symbols(L, k):
    """Fourier symbols of the isotropic lattice stencils on exp(i k.r):
    grad -> i g(k), g = (1/cs2) sum_i w_i c_i sin(k.c_i);
    lap  -> -K2(k), K2 = (2/cs2) sum_i w_i (1 - cos(k.c_i))."""
    k = np.pad(np.asarray(k, float), (0, 3 - len(k)))
    kc = L.c @ k
    g = (L.w[:, None] * L.c * np.sin(kc)[:, None]).sum(0) / L.cs2
    K2 = 2.0 / L.cs2 * (L.w * (1 - np.cos(kc))).sum()
    return g, K2


def oz_structure_factor(rho0, kT, cs2_lb, psi2, kappa, k2):
    """Ornstein-Zernike S(k) = rho0 kT / c_s^2(k), c_s^2(k) = cs^2 + rho0 psi'' + kappa rho0 k^2
    (App. A, Eq. (he-cs2), with psi the excess free energy over the ideal LB gas)."""
    return rho0 * kT / (cs2_lb + rho0 * psi2 + kappa * rho0 * k2)


# ---------------------------------------------------------------------------
# Modified-equilibrium (Swift) model, D2Q9 basis of App. B (Sec. IV.C)
# Mode indices (0-based): rho 0, jx 1, jy 2, e 3, pww 4, pxy 5, qx 6, qy 7, eps 8.
# ---------------------------------------------------------------------------

def swift_d(cs2k, cs2=1.0 / 3.0):
    """d(k) = 6 [c_s^2(k) - cs^2] of Eq. (meq-yeo)."""
    return 6.0 * (cs2k - cs2)


def G_swift(L, rho0, kT, cs2k) -> np.ndarray:
    """Eq. (f-correl-yeo): <df_i df_j> = (S / rho0) fbar_i(k) delta_ij with
    S = rho0 kT / c_s^2(k) (Eq. (s-nonideal)) and fbar(k) the rest state of the
    modified equilibrium, whose moments are (rho0, 0, 0, d(k) rho0, 0, 0, 0, 0,
    -d(k) rho0) by Eq. (meq-yeo); in moment space G_ab = (S/rho0) sum_i T_ai fbar_i T_bi."""
    S = rho0 * kT / cs2k
    d = swift_d(cs2k, L.cs2)
    m = np.zeros(9)
    m[0], m[3], m[8] = rho0, d * rho0, -d * rho0
    fbar = L.Tinv @ m
    return ((S / rho0) * (L.T * fbar[None, :]) @ L.T.T).astype(complex)


def L_swift(L, k, lam, cs2k) -> np.ndarray:
    """Time-evolution operator of Eq. (FDBE-yeo) with Eq. (meq-yeo):
    L = A(k) + Lambda - lambda_e d(k) e_e (x) e_rho + lambda_eps d(k) e_eps (x) e_rho."""
    M = advection(L, k) + lam
    d = swift_d(cs2k, L.cs2)
    M[3, 0] -= lam[3, 3] * d
    M[8, 0] += lam[8, 8] * d
    return M


def noise_swift(L, rho0, kT, lam_e, lam_s, lam_q, lam_eps, cs2k) -> np.ndarray:
    """Noise covariance of the modified-equilibrium FDBE, Eq. (noise-yeo):
    2 rho0 kT / cs^2 times the matrix with N_e (2 - 3 c_s^2(k)) lambda_e,
    N_s lambda_s (x2), N_q lambda_q (x2), N_eps (5/4 - 3/4 c_s^2(k)) lambda_eps
    on the diagonal and 6 (c_s^2(k) - cs^2)(lambda_e + lambda_eps) in the
    (e, eps) corners.  The corners are printed with 12; the FDT of
    Eq. (dbe-fdt) with Eqs. (FDBE-yeo), (meq-yeo) and (f-correl-yeo), which
    reproduces every other printed entry, gives 6, the value used here."""
    N = L.N
    X = np.zeros((9, 9))
    X[3, 3] = N[3] * (2.0 - 3.0 * cs2k) * lam_e
    X[4, 4] = N[4] * lam_s
    X[5, 5] = N[5] * lam_s
    X[6, 6] = N[6] * lam_q
    X[7, 7] = N[7] * lam_q
    X[8, 8] = N[8] * (1.25 - 0.75 * cs2k) * lam_eps
    X[3, 8] = X[8, 3] = 6.0 * (cs2k - L.cs2) * (lam_e + lam_eps)
    return 2.0 * rho0 * kT / L.cs2 * X


def swift_lattice_noise(L, rho0, kT, om_e, om_s, om_q, om_eps, cs2k) -> np.ndarray:
    """Covariance per site and step of the lattice noise of the modified-equilibrium
    model, following Sec. V: xi^LB_a = (1 - omega_a / 2) xi_a with the DBE rates
    lambda_a = 2 omega_a / (2 - omega_a) in Eq. (noise-yeo)."""
    om = np.array([0, 0, 0, om_e, om_s, om_s, om_q, om_q, om_eps], float)
    X = noise_swift(L, rho0, kT, lambda_dbe(om_e), lambda_dbe(om_s), lambda_dbe(om_q), lambda_dbe(om_eps), cs2k)
    s = 1.0 - 0.5 * om
    return s[:, None] * X * s[None, :]

