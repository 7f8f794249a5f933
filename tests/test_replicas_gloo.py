"""Multi-GPU is "replicas only" (independent bond updates, no data-path collective): the
host logic of bench.py's N > 1 path - distinct per-rank workloads, the max-over-ranks
time and the whole-job throughput - on two gloo ranks on CPU."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        from paper_2212_09782_b300 import workloads as W
        seed = bench.replica_seed(W.BASE_SEED, rank)
        theta00 = complex(W.bond_microbench(8, 2, seed=seed)["theta"].ravel()[0])
        local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        t_max = bench.max_over_ranks(local_ms, dist, "cpu")
        value = bench.job_throughput(10, ws, t_max)
        q.put((rank, seed, theta00, t_max, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    (r0, s0, th0, t0, v0), (r1, s1, th1, t1, v1) = res
    assert s0 != s1 and th0 != th1            # each replica updates its own bond
    assert t0 == t1 == 150.0                  # every rank reports the slowest time
    assert v0 == v1 == pytest.approx(2 * 10 / 0.150)   # units of all ranks / that time


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_throughput(20, 1, 1000.0) == pytest.approx(20.0)
