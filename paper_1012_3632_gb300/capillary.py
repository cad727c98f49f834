"""Capillary fluctuations of a liquid stripe (Sec. VI of arXiv 1012.3632).

A D2Q9 box of X x Y sites holds a liquid stripe of the Landau double-well
fluid (rho_L, rho_V, beta, kappa, taken as the total bulk free energy) between
two flat interfaces normal to y.  The run equilibrates for `burn` steps, then
takes a snapshot every `every` steps: the interface heights of every column
(fitted on the GPU to the mean-field profile) and their spectrum, accumulated
in FP64 on the GPU.  The paper's run: 1024 x 400, stripe 200 thick,
rho_L = 1, rho_V = 0.5, beta = 0.1, kappa = 0.08, kT = 1e-7, tau = 1,
10^6 steps, 2000 snapshots.
"""
from __future__ import annotations

import numpy as np

from . import inputs
from .flb import D2Q9, Context, interface_fit, landau_free_energy, landau_width


def stripe_context(X=1024, Y=400, thickness=200, rho_l=1.0, rho_v=0.5, beta=0.1, kappa=0.08, kT=1e-7,
                   omega=1.0, seed=11, precision="fp32", stream=None, model=0):
    """Context holding the mean-field stripe centred in y; returns (ctx, fit).
    model 0: force-based fluid (App. A); model 1: modified equilibrium (Sec. IV.C)."""
    w = landau_width(rho_l, rho_v, beta, kappa)
    y_lo, y_hi = 0.5 * (Y - thickness), 0.5 * (Y + thickness)
    fe = dict(landau_free_energy(rho_l, rho_v, beta, kappa), model=model)
    ctx = Context(D2Q9, (X, Y, 1), omega, omega, omega, kT=kT, free_energy=fe, seed=seed, precision=precision,
                  stream=stream)
    ctx.init(rho=inputs.stripe_density(X, Y, rho_l, rho_v, w, y_lo, y_hi).ravel())
    return ctx, interface_fit(rho_l, rho_v, w, (y_lo, y_hi))


def run_stripe(steps=10**6, snapshots=2000, burn=None, **kw):
    """Run the stripe and return (k, S(k), snapshots taken, final guesses): S is
    the mean over snapshots of the height spectrum of flb_height_spectrum,
    k = 2 pi n / X.  Without `burn`, one tenth of the snapshot interval count
    is spent equilibrating first.  The fit window follows the mean height of
    each interface."""
    X = kw.get("X", 1024)
    every = max(1, steps // (snapshots + (snapshots // 10 if burn is None else 0)))
    burn = steps - every * snapshots if burn is None else burn
    ctx, fit = stripe_context(**kw)
    try:
        ctx.step(burn)
        S = None
        for i in range(snapshots):
            ctx.step(every)
            h = ctx.interface_heights(fit)
            fit.guess[0], fit.guess[1] = float(h[0].mean()), float(h[1].mean())
            S = ctx.height_spectrum(fit, accumulate=True, fetch=(i == snapshots - 1))
        n = ctx.snapshot_count(-2)
    finally:
        ctx.close()
    return 2 * np.pi * np.arange(X) / X, S, n, (fit.guess[0], fit.guess[1])
