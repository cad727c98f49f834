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
