"""The differentiable PyTorch reference (gradient oracle for the adjoint)
reproduces the C oracle's trajectory, and its autograd gradients match central
finite differences of itself."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
from oracle.torch_ref import Ref  # noqa: E402

FE = dict(A=-0.01, B=0.1, rho_c=1.0, kappa=0.02)


def _setup(nonideal, dims=(5, 4, 3), kT=1e-5):
    kw = dict(omega_shear=1.2, omega_bulk=0.9, omega_ghost=1.3, kT=kT, seed=5)
    p = oracle.Params(Q=19, dims=dims, nonideal=nonideal, **(FE if nonideal else {}), **kw)
    rng = np.random.default_rng(1)
    rho = 1 + 0.01 * rng.uniform(-1, 1, p.V)
    f0 = oracle.init(p, rho=rho, thermal=True)
    theta = torch.tensor([1.2, 0.9, 1.3, FE["kappa"], FE["A"], FE["B"]], dtype=torch.float64)
    return p, f0, theta


@pytest.mark.parametrize("nonideal", [False, True])
def test_forward_matches_c_oracle(nonideal):
    p, f0, theta = _setup(nonideal)
    ref = Ref(p)
    X, Y, Z = p.dims
    w = oracle.lattice(19).w
    g0 = torch.tensor((f0 - w[:, None] * p.rho0).reshape(19, Z, Y, X))
    g = ref.run(g0, theta, 0, 6)
    want = oracle.run(p, f0, 0, 6) - w[:, None] * p.rho0
    assert np.abs(g.reshape(19, -1).numpy() - want).max() < 1e-13


def test_autograd_matches_finite_differences():
    p, f0, theta = _setup(True, dims=(4, 3, 3), kT=1e-4)
    ref = Ref(p)
    X, Y, Z = p.dims
    w = oracle.lattice(19).w
    g0 = torch.tensor((f0 - w[:, None] * p.rho0).reshape(19, Z, Y, X))
    normals = [ref.normals(t) for t in range(3)]
    c = torch.tensor(np.random.default_rng(2).standard_normal((19, Z, Y, X)))

    def J(g, th):
        return (c * ref.run(g, th, 0, 3, normals)).sum()

    gg = g0.clone().requires_grad_(True)
    tt = theta.clone().requires_grad_(True)
    J(gg, tt).backward()
    h = 1e-6
    for k in range(6):
        e = torch.zeros(6, dtype=torch.float64)
        e[k] = h
        fd = (J(g0, theta + e) - J(g0, theta - e)) / (2 * h)
        assert abs(fd.item() - tt.grad[k].item()) <= 1e-6 * (abs(fd.item()) + 1e-3), k
    d = torch.tensor(np.random.default_rng(3).standard_normal(g0.shape))
    fd = (J(g0 + h * d, theta) - J(g0 - h * d, theta)) / (2 * h)
    assert abs(fd.item() - (gg.grad * d).sum().item()) <= 1e-6 * abs(fd.item())
