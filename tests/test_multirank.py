"""Sharding one batch over several ranks, on CPU ranks (gloo, world size 2): the DAGs are
split by the LPT partition, every rank evaluates only its own DAGs (here with the CPU
oracle, since the ranks have no GPU), and the per-DAG bounds gathered on rank 0 equal the
bounds of the whole batch evaluated by one rank, DAG for DAG. The benchmark's time is the
maximum over ranks. No collective is used on the data path: only the gather afterwards."""
from __future__ import annotations

import os

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        from paper_2602_20826_gb300 import shard, workloads as wl
        n = 60
        parts = shard.partition(wl.er_sizes(n, 20, 200, wl.BASE_SEED + 2), world)
        mine = wl.config(2, ids=parts[rank])  # only this rank's DAGs are generated
        bounds, status = oracle.schedule_batch(mine)
        got = shard.gather_over_ranks(dist, parts, bounds, n)
        t = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5 * rank], dist, "cpu")
        q.put((rank, t, None if got is None else got.tolist(), [p.tolist() for p in parts],
               int(mine.total_nodes())))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_one_batch_and_gather():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, got0, parts0, nodes0), (r1, t1, got1, parts1, nodes1) = res
    assert t0 == t1 == [2.0, 10.0, 0.5]  # element-wise max over ranks, same on both
    assert parts0 == parts1  # both ranks computed the same split
    assert got1 is None
    import oracle
    from paper_2602_20826_gb300 import workloads as wl
    whole = wl.config(2, n_dags=60)
    want, st = oracle.schedule_batch(whole)
    assert (st == 0).all() and got0 == want.tolist()
    # balanced by node count: the two shards differ by at most one DAG's nodes
    assert abs(nodes0 - nodes1) <= 200


def test_partition_is_a_balanced_split():
    from paper_2602_20826_gb300 import shard
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        costs = rng.integers(1, 1000, size=int(rng.integers(0, 300)))
        parts = shard.partition(costs, world)
        assert len(parts) == world
        allids = np.sort(np.concatenate(parts)) if len(costs) else np.zeros(0)
        assert np.array_equal(allids, np.arange(len(costs)))  # every DAG exactly once
        loads = [int(costs[p].sum()) for p in parts]
        if len(costs):
            assert max(loads) - min(loads) <= int(costs.max())  # LPT: within one job
        assert [p.tolist() for p in shard.partition(costs, world)] == [p.tolist() for p in parts]
        vals = [np.asarray(p) * 10 for p in parts]
        assert np.array_equal(shard.gather(parts, vals, len(costs)), np.arange(len(costs)) * 10)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks([3, 4.5], None, "cpu") == [3.0, 4.5]
