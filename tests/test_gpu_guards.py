"""Bounds check of the kernels' writes.  compute-sanitizer is not available on
the GPU pool, so contexts created with guard zones (opt.guard = 1: 64 KiB of a
fixed byte pattern before and after both population buffers and the density
field) run every step path and every observable on tiny, odd and ragged
lattices -- where the periodic wrap and the partial tiles are most exposed --
and flb_check_guards confirms that no zone was written.
"""
import numpy as np
import pytest

from paper_1012_3632_gb300 import Context, inputs, landau_free_energy
from paper_1012_3632_gb300.flb import FLB_EINVAL, MODES, RHO, U, FLBError

pytestmark = pytest.mark.gpu

EXCESS = dict(A=-0.01, B=0.1, rho_c=1.0, kappa=0.02)
TOTAL = landau_free_energy(1.0, 0.5, 0.1, 0.08)
SWIFT = dict(TOTAL, model=1)

# (32, 8, 1), (32, 16, 7), (64, 8, 18): whole 32 x 8 tiles of the force-model
# step (one-tile periodic wrap, single-plane lattice, columns of several planes)
D3 = [(1, 1, 1), (2, 3, 5), (4, 4, 4), (6, 5, 7), (8, 9, 17), (36, 10, 3), (34, 9, 18), (32, 8, 1), (32, 16, 7),
      (64, 8, 18)]
D2 = [(1, 1, 1), (5, 3, 1), (32, 7, 1), (20, 12, 1)]
CASES = ([(19, d, fe) for d in D3 for fe in (None, EXCESS, TOTAL)] +
         [(9, d, fe) for d in D2 for fe in (None, EXCESS, TOTAL, SWIFT)])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("Q,dims,fe", CASES)
def test_no_write_outside_the_buffers(Q, dims, fe, prec):
    V = int(np.prod(dims))
    with Context(Q, dims, 1.1, 0.9, 1.2, kT=1e-6, free_energy=fe, seed=5, precision=prec, guard=True) as ctx:
        ctx.init(rho=inputs.uniform_density(dims, seed=1), thermal=fe is None)
        ctx.step(4)
        for which in (RHO, U, MODES):
            ctx.moments(which)
        ctx.structure_factor(0, accumulate=True)
        ctx.conservation()
        f = ctx.get_populations()
        ctx.set_populations(f)
        ctx.get_sites([0, V - 1])
        ctx.step(2)
        ctx.check_guards()


def test_guard_arguments():
    with Context(19, (4, 4, 4), 1.0) as ctx:
        with pytest.raises(FLBError) as e:
            ctx.check_guards()  # created without guard zones
        assert e.value.code == FLB_EINVAL
    with pytest.raises(FLBError):
        Context(19, (4, 4, 4), 1.0, guard=2)
