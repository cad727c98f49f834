"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds none of the method's arithmetic: it only draws numbers with
numpy's PCG64 generator (``numpy.random.default_rng(seed)``) and evaluates
plain profiles.  The noise the method itself draws (Philox4x32-10) is
implemented separately on each side.

Field layout: site index s = x + X*(y + Y*z); vector fields are (D, V).
"""
from __future__ import annotations

import numpy as np


def uniform_density(dims, rho_c: float = 1.0, amp: float = 0.01, seed: int = 3) -> np.ndarray:
    """rho = rho_c + U(-amp, amp) per site (non-ideal 256^3 workload: rho_c = 1, amp = 0.01)."""
    X, Y, Z = dims
    rng = np.random.default_rng(seed)
    return rho_c + amp * rng.uniform(-1.0, 1.0, X * Y * Z)


def shear_wave(dims, amp: float = 1e-3, D: int = 3) -> np.ndarray:
    """u_x = amp sin(2 pi z / Z) (D3Q19) or amp sin(2 pi y / Y) (D2Q9); other components 0."""
    X, Y, Z = dims
    u = np.zeros((D, X * Y * Z))
    if D == 3:
        z = np.repeat(np.arange(Z), X * Y)
        u[0] = amp * np.sin(2 * np.pi * z / Z)
    else:
        y = np.repeat(np.arange(Y), X)
        u[0] = amp * np.sin(2 * np.pi * y / Y)
    return u


def random_velocity(dims, D: int, amp: float = 0.02, seed: int = 5) -> np.ndarray:
    X, Y, Z = dims
    rng = np.random.default_rng(seed)
    return amp * rng.standard_normal((D, X * Y * Z))


def random_populations(Q: int, dims, rho0: float = 1.0, rel: float = 0.05, seed: int = 7) -> np.ndarray:
    """Positive populations (Q, V) around rho0/Q with relative spread rel: a
    generic, non-equilibrium state (not the lattice's rest state)."""
    X, Y, Z = dims
    rng = np.random.default_rng(seed)
    return rho0 / Q * (1.0 + rel * rng.uniform(-1.0, 1.0, (Q, X * Y * Z)))


def replica_sizes(n: int = 64, choices=(32, 48, 64, 96, 128), seed: int = 4) -> np.ndarray:
    """Cubic replica edge lengths drawn from `choices` (batched-ensemble workload)."""
    rng = np.random.default_rng(seed)
    return rng.choice(np.asarray(choices), size=n)


def replica_omegas(n: int = 64, lo: float = 0.8, hi: float = 1.6, seed: int = 4) -> np.ndarray:
    rng = np.random.default_rng(seed + 1)
    return rng.uniform(lo, hi, n)


def stripe_density(X: int, Y: int, rho_l: float, rho_v: float, width: float, y_lo: float, y_hi: float,
                   amp: float = 0.0, modes: int = 0, seed: int = 6) -> np.ndarray:
    """(Y, X) density of a liquid stripe between rows y_lo and y_hi: two tanh
    interfaces of width `width` between rho_v and rho_l.  With modes > 0 each
    interface is displaced by a sum of `modes` random long-wave sines of total
    amplitude ~amp (seeded)."""
    rng = np.random.default_rng(seed)
    x = np.arange(X)
    h = np.zeros((2, X))
    for i in range(2):
        for n in range(1, modes + 1):
            h[i] += amp / np.sqrt(modes) * rng.standard_normal() * np.sin(2 * np.pi * n * x / X + rng.uniform(0, 2 * np.pi))
    y = np.arange(Y)[:, None]
    a = 0.5 * (rho_l - rho_v)
    return rho_v + a * (np.tanh(2 * (y - (y_lo + h[0])[None, :]) / width) - np.tanh(2 * (y - (y_hi + h[1])[None, :]) / width))

