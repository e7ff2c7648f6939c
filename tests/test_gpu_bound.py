"""GPU parity of candidate-allocation bounds and the argmin against the CPU oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2602_20826_gb300 import workloads as wl
from tests.gpu_helpers import context
from tests.oracle_checks import random_small_dag

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    return context()


def _run(ctx, batch, variants, n_alloc, alloc, stride, dags=None):
    lb = ctx.load(batch)
    for v in sorted(set(variants)):
        lb.schedule(v, fields=("status",))
    ob, bb, bc = lb.bound(variants, n_alloc, alloc, stride)
    for d in (range(batch.n_dags) if dags is None else dags):
        ref, rb, rc = oracle.search_dag(batch, d, alloc, stride, len(variants), n_alloc, variants)
        assert np.array_equal(ob[d], ref), (d, np.nonzero(ob[d] != ref)[0][:5])
        assert bb[d] == rb and bc[d] == rc, (d, bb[d], rb, bc[d], rc)
    lb.free()
    return ob, bb, bc


def test_config1_full(ctx):
    """One 20-node DAG, M = 8: the paper's own allocation plus 4,096 random ones from
    {1, 2, 4, 8}."""
    b = wl.config(1)
    alloc, stride = wl.candidate_allocations(b, 1, 4097, [1, 2, 4, 8], seed=wl.BASE_SEED + 11)
    ob, bb, bc = _run(ctx, b, [0], 4097, alloc, stride)
    rc, ref = oracle.schedule_dag_of(b, 0)
    assert ob[0, 0] == ref["bound"]  # candidate 0 keeps the scheduled allocation


def test_config3_sampled_all_variants(ctx):
    b = wl.config(3, n_dags=60)
    alloc, stride = wl.candidate_allocations(b, 4, 64, [1, 2, 4, 8, 16, 32], seed=wl.BASE_SEED + 13)
    _run(ctx, b, [0, 1, 2, 3], 64, alloc, stride)


def test_arbitrary_allocations_and_M(ctx):
    """Any byte value (non powers of two, above M) exercises every division path."""
    rng = np.random.default_rng(17)
    for M in (1, 3, 8, 100, 148, 4096):
        dags = [random_small_dag(rng, int(rng.integers(1, 60)), 0.15, int(rng.choice([10, 10**4, 2**32 - 1])))
                for _ in range(30)]
        b = wl.from_dags(dags, M)
        alloc, stride = wl.candidate_allocations(b, 2, 40, list(range(0, 256)), seed=M, keep_scheduled=True)
        _run(ctx, b, [0, 3], 40, alloc, stride)


def test_device_path_and_stride(ctx):
    import torch
    b = wl.small_config(3, n_dags=50, v_lo=20, v_hi=300)
    alloc, stride = wl.candidate_allocations(b, 2, 24, [1, 2, 4, 8, 16, 32], seed=5, cand_stride=64)
    lb = ctx.load(b)
    lb.schedule(0, fields=("status",))
    lb.schedule(2, fields=("status",))
    ob_h, bb_h, bc_h = lb.bound([0, 2], 24, alloc, stride)
    da = torch.from_numpy(alloc).cuda()
    ob = torch.zeros(b.n_dags * 48, dtype=torch.int64, device="cuda")
    bb = torch.zeros(b.n_dags, dtype=torch.int64, device="cuda")
    bc = torch.zeros(b.n_dags, dtype=torch.int32, device="cuda")
    lb.bound([0, 2], 24, da, stride, ob, bb, bc)
    torch.cuda.synchronize()
    assert np.array_equal(ob.cpu().numpy().reshape(b.n_dags, 48), ob_h)
    assert np.array_equal(bb.cpu().numpy(), bb_h) and np.array_equal(bc.cpu().numpy(), bc_h)
    for d in range(0, b.n_dags, 7):
        ref, rb, rc = oracle.search_dag(b, d, alloc, stride, 2, 24, [0, 2])
        assert np.array_equal(ob_h[d], ref)


def test_unscheduled_variant_is_rejected(ctx):
    from paper_2602_20826_gb300.dagrt import DagrtError
    b = wl.small_config(2, n_dags=4, v_lo=5, v_hi=20)
    alloc, stride = wl.candidate_allocations(b, 1, 4, [1, 2], seed=1)
    lb = ctx.load(b)
    with pytest.raises(DagrtError):
        lb.bound([1], 4, alloc, stride)


def test_work_item_path_arbitrary_bytes(ctx):
    """n_alloc a multiple of 64 takes the balanced work-item kernel (chunks of plan rows cut
    at group ends): any byte value, M below and above 128 (table entries above M), DAGs
    whose sums need 64 bits mixed in (their items run in 64-bit arithmetic), one-node DAGs,
    and repeated calls on the same scratch."""
    rng = np.random.default_rng(23)
    for M, n_alloc in ((1, 64), (8, 128), (100, 64), (148, 64), (4096, 64)):
        dags = [random_small_dag(rng, int(rng.integers(1, 90)), 0.1, int(rng.choice([10, 10**4, 10**4, 2**32 - 1])))
                for _ in range(40)]
        b = wl.from_dags(dags, M)
        alloc, stride = wl.candidate_allocations(b, 2, n_alloc, list(range(0, 256)), seed=M, keep_scheduled=True)
        _run(ctx, b, [0, 3], n_alloc, alloc, stride)
        pow2, stride2 = wl.candidate_allocations(b, 2, n_alloc, [1, 2, 4, 8, 16, 32, 64, 128], seed=M + 1)
        _run(ctx, b, [3, 0], n_alloc, pow2, stride2)


def test_work_item_path_long_dags_and_reschedule(ctx):
    """DAGs of several hundred plan rows (many chunks, chunks longer than one staging
    phase) and a plan recomputed between two calls (its chunks are rebuilt)."""
    b = wl.config(3, n_dags=24)
    alloc, stride = wl.candidate_allocations(b, 4, 64, [1, 2, 4, 8, 16, 32, 3, 5], seed=99)
    lb = ctx.load(b)
    for v in range(4):
        lb.schedule(v, fields=("status",))
    ob1, bb1, bc1 = lb.bound([0, 1, 2, 3], 64, alloc, stride)
    lb.schedule(1, fields=("status",))
    ob2, bb2, bc2 = lb.bound([0, 1, 2, 3], 64, alloc, stride)
    assert np.array_equal(ob1, ob2) and np.array_equal(bb1, bb2) and np.array_equal(bc1, bc2)
    for d in range(0, 24, 3):
        ref, rb, rc = oracle.search_dag(b, d, alloc, stride, 4, 64, [0, 1, 2, 3])
        assert np.array_equal(ob1[d], ref), (d, np.nonzero(ob1[d] != ref)[0][:5])
        assert bb1[d] == rb and bc1[d] == rc
    lb.free()


def test_work_item_path_with_rejected_dags(ctx):
    """Rejected DAGs (no plan) get -1 bounds and candidate -1 on the work-item path; the
    others are exact."""
    rng = np.random.default_rng(31)
    good = [random_small_dag(rng, int(rng.integers(5, 80)), 0.15, 10**4) for _ in range(6)]
    w, k = good[0][2], good[0][3]
    cyc = (np.array([0, 1, 2, 3], np.int32), np.array([1, 2, 0], np.int32), w[:3], k[:3])
    rng_bad = (np.array([0, 1, 1, 1], np.int32), np.array([7], np.int32), w[:3], k[:3])
    dags = [good[0], cyc, good[1], good[2], rng_bad, good[3], good[4], cyc, good[5]]
    b = wl.from_dags(dags, 148)
    alloc, stride = wl.candidate_allocations(b, 2, 64, [1, 2, 4, 8, 16, 32], seed=3)
    lb = ctx.load(b)
    for v in (0, 1):
        lb.schedule(v, fields=("status",), check=False)
    ob, bb, bc = lb.bound([0, 1], 64, alloc, stride)
    for d in range(b.n_dags):
        if dags[d] is cyc or dags[d] is rng_bad:
            assert (ob[d] == -1).all() and bb[d] == -1 and bc[d] == -1
        else:
            ref, rb, rc = oracle.search_dag(b, d, alloc, stride, 2, 64, [0, 1])
            assert np.array_equal(ob[d], ref) and bb[d] == rb and bc[d] == rc
    lb.free()


def test_work_item_path_empty_dags(ctx):
    """DAGs without nodes (first, middle, last) get bound 0 for every candidate and
    candidate 0 as the argmin; their neighbours are exact; a second call on the same
    scratch gives the same result (the completion counters were left at zero)."""
    rng = np.random.default_rng(5)
    e = (np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64), np.zeros(0, np.uint8))
    good = [random_small_dag(rng, int(rng.integers(2, 60)), 0.1, 10**4) for _ in range(3)]
    dags = [e, good[0], e, good[1], good[2], e]
    b = wl.from_dags(dags, 148)
    alloc, stride = wl.candidate_allocations(b, 2, 64, [1, 2, 4, 8, 16, 32], seed=9)
    lb = ctx.load(b)
    for v in (0, 2):
        lb.schedule(v, fields=("status",))
    first = lb.bound([0, 2], 64, alloc, stride)
    again = lb.bound([0, 2], 64, alloc, stride)
    for x, y in zip(first, again):
        assert np.array_equal(x, y)
    ob, bb, bc = first
    for d in range(b.n_dags):
        if dags[d] is e:
            assert (ob[d] == 0).all() and bb[d] == 0 and bc[d] == 0
        else:
            ref, rb, rc = oracle.search_dag(b, d, alloc, stride, 2, 64, [0, 2])
            assert np.array_equal(ob[d], ref) and bb[d] == rb and bc[d] == rc
    lb.free()
