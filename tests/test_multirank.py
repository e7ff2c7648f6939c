"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2): every rank
builds its own batch of the same distribution, and the reported time is the maximum over
ranks. No GPU and no collective on the data path are involved."""
from __future__ import annotations

import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2602_20826_gb300 import workloads as wl
        t = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5 * rank], dist, "cpu")
        b = wl.config(2, n_dags=3, seed=bench.rank_seed(rank))
        q.put((rank, t, int(b.wcet.sum()), int(b.total_edges())))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_distinct_batches():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, w0, e0), (r1, t1, w1, e1) = res
    assert t0 == t1 == [2.0, 10.0, 0.5]  # element-wise max over ranks, same on both
    assert (w0, e0) != (w1, e1)  # each rank has its own batch ...
    import bench
    from paper_2602_20826_gb300 import workloads as wl
    b = wl.config(2, n_dags=3, seed=bench.rank_seed(1))
    assert (int(b.wcet.sum()), int(b.total_edges())) == (w1, e1)  # ... built deterministically


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks([3, 4.5], None, "cpu") == [3.0, 4.5]
    assert bench.rank_seed(0) != bench.rank_seed(1)
