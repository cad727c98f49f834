"""Differentiable FP64 reference of the fluctuating LB update in plain PyTorch.

TEST INFRASTRUCTURE (gradient oracle).  Only ``tests/`` use it.  It restates
the update of Gross, Cates, Varnik & Adhikari (arXiv 1012.3632) in whole-lattice
tensor operations so that torch.autograd can differentiate it:

  moments            Eq. (moments), T and N_a of the oracle's lattice tables
  equilibrium        Eq. (feq)
  forcing            Eq. (forcing-term), Guo reading (as in flb_oracle.c)
  update             Eq. (lbe-mom) with the lattice noise of Eq. (noise-lbe)
  force              App. A: F = -rho grad mu, mu = psi'(rho) - kappa lap rho
  streaming          Eq. (lbe-gen): f(r + c_i, t+1) = f*(r, t)

Parameters theta = (omega_shear, omega_bulk, omega_ghost, kappa, A, B) are a
tensor so that their gradients come out of autograd.  The Gaussian normals are
inputs (drawn by the C oracle's Philox), so the noise is the same as on the
GPU.  Its forward results are checked against the C oracle in the tests.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

CS2 = 1.0 / 3.0


class Ref:
    def __init__(self, p: "oracle.Params"):
        assert p.Q == 19 and p.window is None
        self.p = p
        L = oracle.lattice(19)
        self.L = L
        self.T = torch.tensor(L.T, dtype=torch.float64)
        self.Tinv = torch.tensor(L.Tinv, dtype=torch.float64)
        self.N = torch.tensor(L.N, dtype=torch.float64)
        self.w = torch.tensor(L.w, dtype=torch.float64)
        self.c = torch.tensor(L.c.astype(np.float64))
        self.cls = L.cls
        X, Y, Z = p.dims
        self.shape = (Z, Y, X)

    # lattice shifts on (Z, Y, X) fields: phi(r + c)
    def _at(self, phi, c):
        return torch.roll(phi, shifts=(-int(c[2]), -int(c[1]), -int(c[0])), dims=(-3, -2, -1))

    def normals(self, step: int) -> torch.Tensor:
        """(15, Z, Y, X) collision normals of `step` from the C oracle's Philox."""
        X, Y, Z = self.p.dims
        z = np.zeros((15, Z, Y, X))
        for k in range(Z):
            for j in range(Y):
                for i in range(X):
                    site = i + X * (j + Y * k)
                    zz = np.concatenate([oracle.normals4(self.p.seed, site, step, b, 0, self.p.replica)
                                         for b in range(4)])
                    z[:, k, j, i] = zz[:15]
        return torch.tensor(z)

    def rates(self, theta):
        om_s, om_b, om_g = theta[0], theta[1], theta[2]
        zero = theta[0] * 0
        r = []
        for c in self.cls:
            r.append({0: zero, 1: om_b, 2: om_s, 3: om_g}[int(c)])
        return torch.stack(r)

    def force(self, rho, theta):
        if not self.p.nonideal:
            return torch.zeros((3,) + rho.shape, dtype=torch.float64)
        kappa, A, B = theta[3], theta[4], theta[5]
        w, c = self.w, self.c
        lap = sum(w[i] * (self._at(rho, c[i]) - rho) for i in range(1, 19)) * (2.0 / CS2)
        d = rho - self.p.rho_c
        mu = A * d + B * d ** 3 - kappa * lap
        grad = torch.stack([sum(w[i] * c[i, a] * self._at(mu, c[i]) for i in range(1, 19)) / CS2 for a in range(3)])
        F = -rho * grad
        if self.p.total:  # + cs^2 grad rho (ideal-gas pressure of the LB cancelled)
            F = F + torch.stack([sum(w[i] * c[i, a] * self._at(rho, c[i]) for i in range(1, 19)) for a in range(3)])
        return F

    def step(self, g, theta, z):
        """g: (19, Z, Y, X) pre-collision deviations -> next pre-collision deviations."""
        p = self.p
        w, c, T, Tinv, N = self.w, self.c, self.T, self.Tinv, self.N
        f = g + (w * p.rho0)[:, None, None, None]
        rho = f.sum(0)
        F = self.force(rho, theta)
        m = torch.einsum("ai,izyx->azyx", T, f)
        j = torch.einsum("id,izyx->dzyx", c, f)
        u = (j + 0.5 * F) / rho
        cu = torch.einsum("id,dzyx->izyx", c, u)
        cF = torch.einsum("id,dzyx->izyx", c, F)
        uu = (u * u).sum(0)
        uF = (u * F).sum(0)
        feq = w[:, None, None, None] * (rho + rho * cu / CS2 + rho * (cu * cu - CS2 * uu) / (2 * CS2 ** 2))
        phi = w[:, None, None, None] * (cF / CS2 + (2 * cu * cF - 2 * CS2 * uF) / (2 * CS2 ** 2))
        meq = torch.einsum("ai,izyx->azyx", T, feq)
        mF = torch.einsum("ai,izyx->azyx", T, phi)
        om = self.rates(theta)[:, None, None, None]
        rho_n = rho if p.noise_rho_local else torch.full_like(rho, p.rho0)
        nc = torch.tensor([int(cl) != 0 for cl in self.cls])
        xi = torch.zeros_like(m)
        var = rho_n * p.kT * (2.0 - om[nc]) * om[nc] * N[nc][:, None, None, None] / CS2
        xi[nc] = torch.sqrt(var) * z
        ms = m - om * (m - meq) + (1.0 - 0.5 * om) * mF + xi
        fs = torch.einsum("ia,azyx->izyx", Tinv, ms)
        gs = fs - (w * p.rho0)[:, None, None, None]
        return torch.stack([torch.roll(gs[i], shifts=(int(c[i, 2]), int(c[i, 1]), int(c[i, 0])), dims=(0, 1, 2))
                            for i in range(19)])

    def run(self, g0, theta, step0: int, nsteps: int, normals=None):
        g = g0
        for t in range(nsteps):
            z = normals[t] if normals is not None else self.normals(step0 + t)
            g = self.step(g, theta, z)
        return g
