"""Adjoint of the fluctuating LB step (flb_adjoint_step behind FLBRun).

- Gradients equal those of the FP64 PyTorch autograd reference (oracle/torch_ref.py)
  on a small lattice, with checkpoint recomputation in between.
- The 64^3 non-ideal workload (A=-0.01, B=0.1, rho_c=1, kappa=0.02, kT=1e-6,
  omega 1), 200 steps, checkpoints every 20, loss sum_k |rho_hat(k)|^2
  exp(-k^2/0.5) at the last step: gradients w.r.t. omega_shear, omega_bulk,
  kappa, A and the initial populations agree with central finite differences
  (h = 1e-6, FP64).
- The FP32 adjoint agrees with the FP64 one.
"""
import numpy as np
import pytest

import oracle
from paper_1012_3632_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from oracle.torch_ref import Ref  # noqa: E402
from paper_1012_3632_gb300.adjoint import density_spectrum_loss, run  # noqa: E402

FE = dict(A=-0.01, B=0.1, rho_c=1.0, kappa=0.02)


def _g0(dims, seed=3, amp=0.01, thermal=False, kT=1e-6):
    p = oracle.Params(Q=19, dims=dims, kT=kT, seed=seed)
    rho = inputs.uniform_density(dims, amp=amp, seed=seed)
    f0 = oracle.init(p, rho=rho, thermal=thermal)
    return f0 - oracle.lattice(19).w[:, None]


# Landau double well of Sec. VI (rho_L = 1, rho_V = 0.5, beta = 0.1, kappa = 0.08) as total free energy
LANDAU = dict(A=-0.025, B=0.4, rho_c=0.75, kappa=0.08)


@pytest.mark.parametrize("nonideal,total", [(True, False), (False, False), (True, True)])
def test_adjoint_equals_autograd_reference(nonideal, total):
    dims, nsteps = (6, 5, 4), 8
    fe = LANDAU if total else FE
    theta0 = [1.2, 0.9, 1.3, fe["kappa"], fe["A"], fe["B"]]
    kT, seed = 1e-4, 7
    p = oracle.Params(Q=19, dims=dims, omega_shear=theta0[0], omega_bulk=theta0[1], omega_ghost=theta0[2], kT=kT,
                      seed=seed, nonideal=nonideal, total=total, **fe)
    g0 = _g0(dims, seed=2, amp=0.02, thermal=True, kT=kT)
    X, Y, Z = dims
    # reference
    ref = Ref(p)
    gr = torch.tensor(g0.reshape(19, Z, Y, X), requires_grad=True)
    tr = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    gN_ref = ref.run(gr, tr, 0, nsteps)
    density_spectrum_loss(gN_ref.reshape(19, -1), dims).backward()
    # GPU adjoint, checkpoints every 3 steps
    cfg = dict(dims=dims, kT=kT, seed=seed, precision="fp64", nsteps=nsteps, every=3, nonideal=nonideal,
               rho_c=fe["rho_c"], total=total)
    gd = torch.tensor(g0, device="cuda", requires_grad=True)
    td = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    gN = run(gd, td, cfg)
    assert np.abs(gN.detach().cpu().numpy() - gN_ref.detach().reshape(19, -1).numpy()).max() < 1e-12
    density_spectrum_loss(gN, dims).backward()
    lam_ref = gr.grad.reshape(19, -1).numpy()
    assert np.allclose(gd.grad.cpu().numpy(), lam_ref, rtol=1e-8, atol=1e-12 * np.abs(lam_ref).max())
    idx = [0, 1, 2, 3, 4, 5] if nonideal else [0, 1, 2]
    assert np.allclose(td.grad.numpy()[idx], tr.grad.numpy()[idx], rtol=1e-8, atol=1e-14)


def _loss_of(g0_dev, theta, cfg):
    with torch.no_grad():
        return density_spectrum_loss(run(g0_dev, theta, cfg), cfg["dims"]).item()


def test_64cubed_200_steps_gradients_match_finite_differences():
    dims = (64, 64, 64)
    cfg = dict(dims=dims, kT=1e-6, seed=5, precision="fp64", nsteps=200, every=20, nonideal=True,
               rho_c=FE["rho_c"])
    theta0 = torch.tensor([1.0, 1.0, 1.0, FE["kappa"], FE["A"], FE["B"]], dtype=torch.float64)
    g0 = torch.tensor(_g0(dims, seed=5), device="cuda")
    gd = g0.clone().requires_grad_(True)
    td = theta0.clone().requires_grad_(True)
    density_spectrum_loss(run(gd, td, cfg), dims).backward()
    h = 1e-6
    for k in (0, 1, 3, 4):  # omega_shear, omega_bulk, kappa, A
        e = torch.zeros(6, dtype=torch.float64)
        e[k] = h
        fd = (_loss_of(g0, theta0 + e, cfg) - _loss_of(g0, theta0 - e, cfg)) / (2 * h)
        assert abs(td.grad[k].item() - fd) <= 1e-5 * abs(fd) + 1e-12, (k, td.grad[k].item(), fd)
    # initial populations: two single components and one random direction
    lam = gd.grad
    rng = np.random.default_rng(9)
    dirs = []
    for (i, s) in ((3, 1234), (17, 200000)):
        d = torch.zeros_like(g0)
        d[i, s] = 1.0
        dirs.append(d)
    dirs.append(torch.tensor(rng.standard_normal(g0.shape), device="cuda"))
    for d in dirs:
        fd = (_loss_of(g0 + h * d, theta0, cfg) - _loss_of(g0 - h * d, theta0, cfg)) / (2 * h)
        an = (lam * d).sum().item()
        assert abs(an - fd) <= 1e-5 * abs(fd) + 1e-12, (an, fd)


def test_fp32_adjoint_close_to_fp64():
    dims = (32, 32, 32)
    base = dict(dims=dims, kT=1e-6, seed=6, nsteps=50, every=10, nonideal=True, rho_c=FE["rho_c"])
    theta0 = [1.0, 1.0, 1.0, FE["kappa"], FE["A"], FE["B"]]
    g0 = _g0(dims, seed=6)
    out = {}
    for prec, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        gd = torch.tensor(g0, device="cuda", dtype=dt, requires_grad=True)
        td = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
        density_spectrum_loss(run(gd, td, dict(base, precision=prec)), dims).backward()
        out[prec] = (gd.grad.double().cpu().numpy(), td.grad.numpy())
    l64, t64 = out["fp64"]
    l32, t32 = out["fp32"]
    assert np.allclose(t32[[0, 1, 3, 4]], t64[[0, 1, 3, 4]], rtol=2e-3)
    assert np.abs(l32 - l64).max() <= 2e-3 * np.abs(l64).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_segment_equals_single_steps(prec):
    """flb_adjoint_segment (recompute + reverse sweep in one call) gives bitwise
    the lam and gradients of the same segment done with flb_step,
    flb_get_state_device and flb_adjoint_step one step at a time."""
    from paper_1012_3632_gb300 import Context
    from paper_1012_3632_gb300.flb import FLBError

    dims, start, n = (12, 10, 9), 5, 7
    dt = torch.float64 if prec == "fp64" else torch.float32
    g0 = torch.tensor(_g0(dims, seed=4, amp=0.02), dtype=dt, device="cuda").contiguous()
    lam0 = torch.randn(g0.shape, dtype=dt, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    kw = dict(kT=1e-5, free_energy=FE, seed=6, precision=prec)
    outs = []
    with Context(19, dims, 1.1, 0.9, 1.2, **kw) as c:
        lam, grad = lam0.clone(), torch.zeros(6, dtype=torch.float64, device="cuda")
        states = torch.empty((n,) + tuple(g0.shape), dtype=dt, device="cuda")
        c.adjoint_segment(g0.data_ptr(), start, n, states.data_ptr(), lam.data_ptr(), grad.data_ptr())
        torch.cuda.synchronize()
        outs.append((lam.cpu(), grad.cpu(), states.cpu()))
        with pytest.raises(FLBError):
            c.adjoint_segment(g0.data_ptr(), start, 0, states.data_ptr(), lam.data_ptr(), grad.data_ptr())
    with Context(19, dims, 1.1, 0.9, 1.2, **kw) as c:
        st = [g0.clone()]
        c.set_state_device(g0.data_ptr())
        c.step_count = start
        for _ in range(n - 1):
            c.step(1)
            s = torch.empty_like(g0)
            c.get_state_device(s.data_ptr())
            st.append(s)
        lam, grad = lam0.clone(), torch.zeros(6, dtype=torch.float64, device="cuda")
        for k in reversed(range(n)):
            nxt = torch.empty_like(lam)
            c.adjoint_step(st[k].data_ptr(), start + k, lam.data_ptr(), nxt.data_ptr(), grad.data_ptr())
            lam = nxt
        torch.cuda.synchronize()
        outs.append((lam.cpu(), grad.cpu(), torch.stack(st).cpu()))
    (l1, g1, s1), (l2, g2, s2) = outs
    assert torch.equal(s1, s2)
    assert torch.equal(l1, l2)
    assert torch.equal(g1, g2)
