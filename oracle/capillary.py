"""Capillary-wave observables and closed forms (Sec. VI of arXiv 1012.3632).

TEST INFRASTRUCTURE (oracle).  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference leg use it; the CUDA library never
does.  Plain numpy, FP64, written for checking by eye:

  landau(rho_L, rho_V, beta)   Eq. (f0-bulk) as the quartic psi of the force
                               model: f0' = A d + B d^3, d = rho - (rho_L + rho_V)/2
  width, surface_tension       Eqs. (interf-width), (surf-tension)
  profile                      Eq. (denprof), mean-field interface profile
  interface_heights            Eq. (height-def): h(x) from a least-squares fit of
                               the mean-field profile to each column
  height_spectrum              |h(k)|^2 / X averaged over the two interfaces
  capillary_spectrum           Eq. (capill-static) with k^2 -> 2 - 2 cos k
"""
from __future__ import annotations

import numpy as np


def landau(rho_l: float, rho_v: float, beta: float) -> dict:
    """beta (rho - rho_V)^2 (rho - rho_L)^2 = beta (d^2 - D^2)^2 with
    d = rho - (rho_L + rho_V)/2, D = (rho_L - rho_V)/2, so
    f0' = 4 beta d^3 - 4 beta D^2 d: A = -4 beta D^2, B = 4 beta."""
    D = 0.5 * (rho_l - rho_v)
    return dict(A=-4.0 * beta * D * D, B=4.0 * beta, rho_c=0.5 * (rho_l + rho_v))


def f0(rho, rho_l: float, rho_v: float, beta: float):
    """Eq. (f0-bulk)."""
    return beta * (rho - rho_v) ** 2 * (rho - rho_l) ** 2


def width(rho_l: float, rho_v: float, beta: float, kappa: float) -> float:
    """Eq. (interf-width): w = sqrt(8 kappa / beta) / (rho_L - rho_V)."""
    return np.sqrt(8.0 * kappa / beta) / (rho_l - rho_v)


def surface_tension(rho_l: float, rho_v: float, beta: float, kappa: float) -> float:
    """Eq. (surf-tension): sigma = (rho_L - rho_V)^3 sqrt(2 kappa beta) / 6."""
    return (rho_l - rho_v) ** 3 * np.sqrt(2.0 * kappa * beta) / 6.0


def profile(s, rho_l: float, rho_v: float, w: float, sign: float = 1.0):
    """Eq. (denprof) at signed distance s from the interface; sign = +1: liquid
    at s > 0, sign = -1: liquid at s < 0."""
    return 0.5 * (rho_l + rho_v) + sign * 0.5 * (rho_l - rho_v) * np.tanh(2.0 * s / w)


def interface_heights(rho, rho_l: float, rho_v: float, w: float, guess, window: int = 8,
                      iterations: int = 8) -> np.ndarray:
    """(2, X) heights of the lower and the upper interface of a stripe.

    rho: (Y, X) density.  For each column x and interface i the height h
    minimizes sum_{y = c-window}^{c+window} (rho(x, y mod Y) - profile(y - h))^2,
    c = round(guess[i]), by `iterations` Gauss-Newton steps from h = guess[i]
    (profile rising with y at the lower interface, falling at the upper one)."""
    rho = np.asarray(rho, dtype=np.float64)
    Y, X = rho.shape
    out = np.empty((2, X))
    for i, sign in ((0, 1.0), (1, -1.0)):
        c = int(np.rint(guess[i]))
        ys = np.arange(c - window, c + window + 1)
        col = rho[np.mod(ys, Y), :]                     # (2W+1, X)
        h = np.full(X, float(guess[i]))
        for _ in range(iterations):
            th = np.tanh(2.0 * (ys[:, None] - h[None, :]) / w)
            r = col - profile(ys[:, None] - h[None, :], rho_l, rho_v, w, sign)
            j = -sign * 0.5 * (rho_l - rho_v) * (2.0 / w) * (1.0 - th * th)
            h = h + (j * r).sum(axis=0) / (j * j).sum(axis=0)
        out[i] = h
    return out


def height_spectrum(h) -> np.ndarray:
    """S(k_n) = mean over the two interfaces of |DFT(h - <h>)|^2 / X."""
    h = np.asarray(h, dtype=np.float64)
    X = h.shape[1]
    n = np.arange(X)
    E = np.exp(-2j * np.pi * np.outer(n, n) / X)       # plain DFT matrix
    S = np.zeros(X)
    for i in range(2):
        d = h[i] - h[i].mean()
        S += np.abs(E @ d) ** 2 / X
    return S / 2.0


def capillary_spectrum(k, kT: float, sigma: float):
    """Eq. (capill-static) on the lattice: kT / (sigma (2 - 2 cos k))."""
    k = np.asarray(k, dtype=np.float64)
    return kT / (sigma * (2.0 - 2.0 * np.cos(k)))
