"""Gradients through many fluctuating-LB steps: a ``torch.autograd.Function``
around the C ABI's forward step and hand-written adjoint step.

The forward pass runs ``nsteps`` D3Q19 steps on the GPU (``flb_step``) from a
device tensor of pre-collision deviations g0 = f0 - w rho0 (shape (19, V),
dtype of the storage precision) and keeps a copy of the state every ``every``
steps.  The backward pass walks the segments in reverse: it recomputes the
states of a segment from its checkpoint (the Philox noise is a pure function
of seed, site and step, so the recomputed trajectory is identical) and applies
the adjoint step from the last step of the segment to the first, both in one
``flb_adjoint_segment`` call per segment.  The
parameters theta = (omega_shear, omega_bulk, omega_ghost, kappa, A, B) get
their gradients from the same adjoint steps.

PyTorch provides device memory, the stream and autograd plumbing; every step
and adjoint step runs in the CUDA kernels of libflb.so.
"""
from __future__ import annotations

import torch

from .flb import D3Q19, Context

THETA = ("omega_shear", "omega_bulk", "omega_ghost", "kappa", "A", "B")

# planes per block of the z-marching step, tuned by the first forward pass on a
# lattice shape and reused by later contexts of the same shape (the length
# changes no result)
_ZCHUNK: dict = {}


def _context(dims, theta, cfg):
    th = [float(v) for v in theta.detach().cpu().tolist()]
    fe = None
    if cfg.get("nonideal", True):
        fe = dict(A=th[4], B=th[5], rho_c=cfg.get("rho_c", 1.0), kappa=th[3], total=cfg.get("total", False))
    return Context(D3Q19, dims, th[0], th[1], th[2], kT=cfg["kT"], free_energy=fe, seed=cfg["seed"],
                   precision=cfg["precision"], rho0=cfg.get("rho0", 1.0), replica=cfg.get("replica", 0),
                   noise_rho_local=cfg.get("noise_rho_local", True),
                   stream=torch.cuda.current_stream().cuda_stream,
                   z_chunk=_ZCHUNK.get((tuple(dims), cfg["precision"]), 0))


class FLBRun(torch.autograd.Function):
    """g_N = FLBRun.apply(g0, theta, cfg); differentiable in g0 and theta."""

    @staticmethod
    def forward(fctx, g0, theta, cfg):
        dims = tuple(cfg["dims"])
        nsteps, every = int(cfg["nsteps"]), int(cfg.get("every", 20))
        ctx = _context(dims, theta, cfg)
        g0 = g0.contiguous()
        ctx.set_state_device(g0.data_ptr())
        ctx.step_count = 0
        ckpts = [g0.clone()]
        for start in range(0, nsteps, every):
            ctx.step(min(every, nsteps - start))
            if start + every < nsteps:
                c = torch.empty_like(g0)
                ctx.get_state_device(c.data_ptr())
                ckpts.append(c)
        gN = torch.empty_like(g0)
        ctx.get_state_device(gN.data_ptr())
        planes, tuning = ctx.z_chunk()
        if not tuning:
            _ZCHUNK[(dims, cfg["precision"])] = planes
        fctx.flb = ctx
        fctx.ckpts = ckpts
        fctx.nsteps, fctx.every = nsteps, every
        fctx.theta_meta = (theta.dtype, theta.device)
        return gN

    @staticmethod
    def backward(fctx, lamN):
        ctx = fctx.flb
        nsteps, every = fctx.nsteps, fctx.every
        lam = lamN.contiguous().clone()
        grad = torch.zeros(6, dtype=torch.float64, device=lam.device)
        nseg = (nsteps + every - 1) // every
        states = torch.empty((min(every, nsteps),) + tuple(lam.shape), dtype=lam.dtype, device=lam.device)
        for seg in reversed(range(nseg)):
            start, end = seg * every, min((seg + 1) * every, nsteps)
            # recompute the segment from its checkpoint and run its adjoint steps
            # backwards (flb_adjoint_segment); lam is updated in place
            ctx.adjoint_segment(fctx.ckpts[seg].data_ptr(), start, end - start, states.data_ptr(), lam.data_ptr(),
                                grad.data_ptr())
        ctx.close()
        dtype, device = fctx.theta_meta
        return lam, grad.to(dtype=dtype, device=device), None


def run(g0: torch.Tensor, theta: torch.Tensor, cfg: dict) -> torch.Tensor:
    """Differentiable N-step run; see FLBRun."""
    return FLBRun.apply(g0, theta, cfg)


def density_spectrum_loss(g: torch.Tensor, dims, rho0: float = 1.0, width: float = 0.5) -> torch.Tensor:
    """sum_k |rho_hat(k)|^2 exp(-k^2 / width) with rho_hat the DFT of rho - <rho>,
    k = 2 pi n / L componentwise in (-pi, pi] (the k = 0 term vanishes)."""
    X, Y, Z = dims
    rho = rho0 + g.sum(0).reshape(Z, Y, X).to(torch.float64)
    d = rho - rho.mean()
    rh = torch.fft.fftn(d)
    ks = [2 * torch.pi * torch.fft.fftfreq(n, device=g.device, dtype=torch.float64) for n in (Z, Y, X)]
    kz, ky, kx = torch.meshgrid(*ks, indexing="ij")
    w = torch.exp(-(kx ** 2 + ky ** 2 + kz ** 2) / width)
    return (w * (rh.real ** 2 + rh.imag ** 2)).sum()
