"""Small-k sound waves from the linearised hydrodynamics of the DBE (test aid).

Shared by the oracle pin and the GPU check of the sound attenuation; it holds
closed forms written from the paper (App. B viscosities, the Sec. V rate map)
and a fit of the measured wave, no lattice arithmetic.
"""
import numpy as np

from oracle import theory

CS2 = 1.0 / 3.0


def sound_wave_rates(D, k, omega_shear, omega_bulk):
    """Decay rate Gamma and frequency Omega of a small-k sound wave.

    Chapman-Enskog on the DBE: the non-equilibrium stress relaxes towards
    -cs^2 (d_a j_b + d_b j_a) / lambda, its traceless part with lambda_s (App. B:
    nu_s = cs^2 / lambda_s) and its trace -- the c^2 (bulk) mode -- with
    lambda_b.  A longitudinal wave then obeys
        d_t j = -i k cs^2 rho - k^2 [2 (1 - 1/D) nu_s + (2/D) cs^2 / lambda_b] j,
    so rho ~ exp(-Gamma t) cos(Omega t) with
        Gamma = (k^2 / 2) [2 (1 - 1/D) cs^2 / lambda_s + (2/D) cs^2 / lambda_b],
        Omega = sqrt(cs^2 k^2 - Gamma^2).
    The lattice rates map by Sec. V, lambda = 2 omega / (2 - omega), so that
    cs^2 / lambda = cs^2 (1/omega - 1/2).  The ghost rate enters at O(k^4) only."""
    nu_s = CS2 / theory.lambda_dbe(omega_shear)
    nu_b = CS2 / theory.lambda_dbe(omega_bulk)
    gamma = 0.5 * k * k * (2.0 * (1.0 - 1.0 / D) * nu_s + (2.0 / D) * nu_b)
    return gamma, np.sqrt(CS2 * k * k - gamma * gamma)


def fit_sound_wave(ts, rho_k, j_k):
    """Decay rate and angular frequency of the right-moving sound amplitude
    a = (rho_k + j_k / cs) / 2, which goes as exp(-(Gamma + i Omega) t) for
    rho_k = sum_x drho(x) exp(-i k x) and j_k likewise."""
    a = 0.5 * (np.asarray(rho_k) + np.asarray(j_k) / np.sqrt(CS2))
    gamma = -np.polyfit(ts, np.log(np.abs(a)), 1)[0]
    omega = -np.polyfit(ts, np.unwrap(np.angle(a)), 1)[0]
    return gamma, omega
