"""Batched replicas (flb_batch_*): many independent D3Q19 ideal-gas lattices of
uneven sizes in one persistent launch per step, replayed from a CUDA graph.

Each replica must evolve exactly like a single lattice with the same
parameters, Philox key and replica word: checked against the FP64 oracle and
against a single-lattice context (bit for bit where X is even)."""
import numpy as np
import pytest

import oracle
from paper_1012_3632_gb300 import Batch, Context

pytestmark = pytest.mark.gpu

# even X: two-site packed path; odd X: one-site path
DIMS = [(8, 8, 8), (12, 10, 9), (6, 5, 4), (32, 16, 8), (7, 6, 5)]
OMS = [1.2, 0.9, 1.55, 1.0, 1.3]
KTS = [1e-5, 2e-5, 1e-4, 1e-5, 3e-5]
SEEDS = [11, 2 ** 33 + 5, 7, 99, 3]
OMB = [1.0, 1.1, 0.8, 1.0, 1.2]
OMG = [1.0, 1.3, 1.2, 0.7, 1.5]


def test_batch_replicas_match_oracle_and_single_lattice():
    steps = 100
    with Batch(DIMS, OMS, KTS, SEEDS, omega_bulk=OMB, omega_ghost=OMG) as b:
        b.init(thermal=True)
        b.step(steps)
        for r, dims in enumerate(DIMS):
            got = b.get_populations(r)
            kw = dict(omega_shear=OMS[r], omega_bulk=OMB[r], omega_ghost=OMG[r], kT=KTS[r], seed=SEEDS[r])
            p = oracle.Params(Q=19, dims=dims, replica=r, **kw)
            want = oracle.run(p, oracle.init(p, thermal=True), 0, steps)
            assert np.abs(got - want).max() <= 2e-5, r
            with Context(19, dims, precision="fp32", replica=r, **kw) as c:
                c.init(thermal=True)
                c.step(steps)
                if dims[0] % 2 == 0:
                    # the two-site path: packed FP32 with the same operations
                    # in the same order as the single-lattice step
                    assert np.array_equal(got, c.get_populations()), r
                else:
                    assert np.abs(got - c.get_populations()).max() <= 1e-6, r


def test_graph_replays_equal_single_steps():
    with Batch(DIMS, OMS, KTS, SEEDS) as a, Batch(DIMS, OMS, KTS, SEEDS) as b:
        a.init(thermal=True)
        b.init(thermal=True)
        a.step(7)  # three graph replays and one direct launch
        for _ in range(7):
            b.step(1)
        a.step(4)
        b.step(3)
        b.step(1)
        for r in range(len(DIMS)):
            assert np.array_equal(a.get_populations(r), b.get_populations(r))
        assert a.info()[2] == b.info()[2] == 11


def test_autotune_keeps_state():
    with Batch(DIMS, OMS, KTS, SEEDS) as b:
        b.init(thermal=True)
        b.step(3)
        before = [b.get_populations(r) for r in range(len(DIMS))]
        shapes = b.autotune()
        assert shapes.shape == (len(DIMS), 3) and np.all(np.prod(shapes, axis=1) == 256)
        for r in range(len(DIMS)):
            assert np.array_equal(before[r], b.get_populations(r))
        assert b.info()[2] == 3


def test_ensemble_mode_temperatures():
    """Every replica's modes equilibrate at its own kT (ensemble of 8 replicas)."""
    dims = [(32, 32, 32), (24, 24, 24)] * 4
    kts = [1e-5, 2e-5] * 4
    oms = list(np.linspace(0.8, 1.6, 8))
    N = np.array([1, 1 / 3, 1 / 3, 1 / 3, 2 / 3, 4 / 3, 4 / 9, 1 / 9, 1 / 9, 1 / 9, 2 / 27, 2 / 27, 2 / 27,
                  2 / 9, 2 / 9, 2 / 9, 2 / 9, 1 / 3, 1 / 9])
    with Batch(dims, oms, kts, list(range(100, 108))) as b:
        b.init(thermal=True)
        for _ in range(40):
            b.step(25)
            var = b.mode_variance()
    T = (var / N / 3.0) / np.array(kts)[:, None]
    V = np.array([np.prod(d) for d in dims])
    T[:, :4] *= (V / (V - 1.0))[:, None]  # the site mean removes k = 0 of the conserved modes
    assert np.all(np.abs(T.mean(axis=0) - 1) < 0.02), T.mean(axis=0)


def test_batch_structure_factor_matches_oracle():
    """flb_batch_structure_factor of each replica (FP32 transform, |F|^2 summed in
    FP64) against the oracle's FP64 DFT of the replica's populations; the
    accumulated mean of two snapshots is their average."""
    with Batch(DIMS, OMS, KTS, SEEDS, omega_bulk=OMB, omega_ghost=OMG) as b:
        b.init(thermal=True)
        b.step(4)
        for r, dims in enumerate(DIMS):
            f = b.get_populations(r)
            p = oracle.Params(Q=19, dims=dims, replica=r, omega_shear=OMS[r], kT=KTS[r], seed=SEEDS[r])
            for mode in (0, 3, 18):
                S = b.structure_factor(r, mode)
                want = oracle.structure_factor(p, f, mode)
                assert np.allclose(S, want, rtol=1e-4, atol=1e-5 * want.max()), (r, mode)
        s1 = b.structure_factor(1, 0, accumulate=True)
        b.step(3)
        s2 = b.structure_factor(1, 0)
        mean = b.structure_factor(1, 0, accumulate=True)
        assert np.allclose(mean, 0.5 * (s1 + s2), rtol=1e-12, atol=1e-20)
