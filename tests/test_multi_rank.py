"""The N > 1 path of bench.py (one replica per rank, no data-path collective)
checked on the CPU with two gloo ranks: the max of the per-rank times over the
process group, the whole-job throughput and the per-rank Philox replica word;
and, on the oracle, that replicas with distinct words evolve independently
while equal words reproduce each other."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + 5.0 * rank, world, device="cpu")
        q.put((rank, t, bench.whole_job_mlups(world, 1000, 50, t), bench.replica_word(rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]            # max over ranks on every rank
    assert out[0][2] == out[1][2] == 2 * 1000 * 50 / 15.0 / 1e6
    assert [o[3] for o in out] == [0, 1]                   # distinct replica words


def test_replica_words_give_independent_noise():
    p0 = oracle.Params(Q=19, dims=(4, 3, 3), kT=1e-5, seed=7, replica=0)
    f0 = oracle.init(p0, thermal=True)
    a = oracle.run(p0, f0, 0, 5)
    b = oracle.run(p0.with_(replica=1), f0, 0, 5)
    c = oracle.run(p0, f0, 0, 5)
    assert np.array_equal(a, c)
    d = (a - b).ravel()
    assert np.abs(d).max() > 1e-4 and abs(np.corrcoef(a.ravel() - f0.ravel(), b.ravel() - f0.ravel())[0, 1]) < 0.9
