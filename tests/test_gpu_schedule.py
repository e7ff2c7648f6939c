"""GPU parity of the scheduler (Alg.1, Alg.2, Lemma 1, Theorem 1) against the CPU oracle.

Every output is compared element by element and must be bit-identical (integer work):
levels, W^anc, blocks, groups, SMs, segments, plan rows, extra edges and the bound.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2602_20826_gb300 import workloads as wl
from tests.gpu_helpers import FIELDS, compare_dag, context, gpu_schedule
from tests.oracle_checks import random_small_dag

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    return context()


def _check_batch(ctx, batch, variant=0, edges=True, dags=None):
    lb, res = gpu_schedule(ctx, batch, variant, edges=edges)
    for d in (range(batch.n_dags) if dags is None else dags):
        compare_dag(batch, res, d, variant, edges)
    lb.free()
    return res


def test_worked_example(ctx):
    rp, col = wl.csr_from_edges(7, [0, 0, 0, 2, 3, 3, 1, 4, 5], [1, 2, 3, 4, 4, 5, 6, 6, 6])
    b = wl.from_dags([(rp, col, np.array([1, 4, 2, 2, 4, 4, 1]), np.full(7, 64, np.uint8))], 6)
    res = _check_batch(ctx, b)
    assert res["bound"][0] == 5


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("cfg,vlo,vhi,n", [(1, 20, 20, 40), (2, 5, 200, 120), (3, 50, 300, 40),
                                           (4, 100, 400, 12)])
def test_small_configs_all_outputs(ctx, cfg, vlo, vhi, n, variant):
    b = wl.small_config(cfg, n_dags=n, v_lo=vlo, v_hi=vhi)
    _check_batch(ctx, b, variant)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_random_small_dags_many_M(ctx, variant):
    rng = np.random.default_rng(500 + variant)
    for M in (1, 2, 3, 5, 8, 16, 148, 4096):
        dags = []
        for _ in range(40):
            V = int(rng.integers(1, 40))
            dags.append(random_small_dag(rng, V, float(rng.uniform(0.02, 0.6)),
                                         int(rng.choice([3, 20, 200, 5000]))))
        _check_batch(ctx, wl.from_dags(dags, M), variant)


def test_size_class_boundaries(ctx):
    rng = np.random.default_rng(9)
    dags = []
    for V in (1, 2, 63, 64, 65, 127, 128, 129, 255, 256, 257, 400, 1000):
        dags.append(random_small_dag(rng, V, min(0.5, 8.0 / V), 1000))
    for M in (8, 148):
        _check_batch(ctx, wl.from_dags(dags, M))


def test_special_shapes(ctx):
    dags = []
    # isolated nodes, a chain, an out-star, an in-star, a complete DAG
    dags.append((np.zeros(11, np.int32), np.zeros(0, np.int32), np.arange(1, 11), np.full(10, 64, np.uint8)))
    rp, col = wl.csr_from_edges(30, list(range(29)), list(range(1, 30)))
    dags.append((rp, col, np.arange(30) * 7 + 1, np.arange(30).astype(np.uint8) * 2))
    rp, col = wl.csr_from_edges(200, [0] * 199, list(range(1, 200)))
    dags.append((rp, col, np.full(200, 13), np.full(200, 40, np.uint8)))
    rp, col = wl.csr_from_edges(200, list(range(199)), [199] * 199)
    dags.append((rp, col, np.full(200, 300), np.full(200, 64, np.uint8)))
    V = 40
    src = [i for i in range(V) for j in range(i + 1, V)]
    dst = [j for i in range(V) for j in range(i + 1, V)]
    rp, col = wl.csr_from_edges(V, src, dst)
    dags.append((rp, col, np.arange(1, V + 1), np.full(V, 33, np.uint8)))
    # extreme loads and fractions
    rng = np.random.default_rng(3)
    rp, col, _, _ = random_small_dag(rng, 60, 0.1, 10)
    dags.append((rp, col, np.full(60, 2**32 - 1), np.zeros(60, np.uint8)))
    dags.append((rp, col, rng.integers(2**31, 2**32, size=60), np.full(60, 64, np.uint8)))
    for M in (1, 7, 148, 4096):
        for var in range(5):
            _check_batch(ctx, wl.from_dags(dags, M), var)


def test_empty_dags_and_empty_batch(ctx):
    e = (np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64), np.zeros(0, np.uint8))
    rng = np.random.default_rng(4)
    b = wl.from_dags([e, random_small_dag(rng, 10, 0.3, 9), e], 148)
    res = _check_batch(ctx, b)
    assert res["bound"][0] == 0 and res["bound"][2] == 0
    b0 = wl.from_dags([], 148)
    lb = ctx.load(b0)
    r = lb.schedule(0, fields=("bound",))
    assert r["rc"] == 0 and len(r["bound"]) == 0


def test_invalid_dags_report_per_dag_status(ctx):
    rng = np.random.default_rng(5)
    good = random_small_dag(rng, 12, 0.3, 50)
    rp, col, w, k = good
    dags = [good]
    dags.append((np.array([0, 1, 2, 3], np.int32), np.array([1, 2, 0], np.int32), w[:3], k[:3]))  # cycle
    dags.append((np.array([0, 1, 1, 1], np.int32), np.array([5], np.int32), w[:3], k[:3]))  # range
    dags.append((np.array([0, 1, 1, 1], np.int32), np.array([0], np.int32), w[:3], k[:3]))  # self loop
    dags.append((np.array([0, 2, 2, 2], np.int32), np.array([2, 1], np.int32), w[:3], k[:3]))  # unsorted
    dags.append((np.array([0, 2, 2, 2], np.int32), np.array([1, 1], np.int32), w[:3], k[:3]))  # duplicate
    dags.append((np.array([0, 0, 0, 0], np.int32), np.zeros(0, np.int32), np.array([0, 1, 1]), k[:3]))
    dags.append((np.array([0, 0, 0, 0], np.int32), np.zeros(0, np.int32), np.array([1, 2**32, 1]), k[:3]))
    dags.append((np.array([0, 0, 0, 0], np.int32), np.zeros(0, np.int32), w[:3], np.array([1, 65, 1], np.uint8)))
    dags.append((np.array([0, 2, 1, 2], np.int32), np.array([1, 2], np.int32), w[:3], k[:3]))  # row_ptr
    dags.append(good)
    b = wl.from_dags(dags, 148)
    lb = ctx.load(b)
    res = lb.schedule(0, fields=FIELDS, check=False)
    want = [0, -2, -3, -3, -3, -3, -1, -1, -1, -1, 0]
    assert list(res["status"]) == want
    assert res["rc"] == -2  # the first failing DAG's status
    for d in range(b.n_dags):
        compare_dag(b, res, d, 0, edges=False)


def test_device_pointer_path_matches_host_path(ctx):
    import torch
    b = wl.small_config(2, n_dags=300, v_lo=5, v_hi=200, seed=77)
    want, _ = oracle.schedule_batch(b)
    dev = {k: torch.from_numpy(getattr(b, k)).cuda() for k in
           ("node_off", "edge_off", "row_ptr", "col", "wcet", "k64")}
    lb = ctx.load(dev, M=b.M)
    out = {"bound": torch.full((b.n_dags,), -9, dtype=torch.int64, device="cuda"),
           "status": torch.full((b.n_dags,), -9, dtype=torch.int32, device="cuda")}
    lb.schedule(0, out=out)
    torch.cuda.synchronize()
    assert np.array_equal(out["bound"].cpu().numpy(), want)
    assert (out["status"].cpu().numpy() == 0).all()


def test_full_config2_every_dag(ctx):
    """The full 10,000-DAG batch in the launch configuration the benchmark times."""
    b = wl.config(2)
    want, st = oracle.schedule_batch(b)
    lb = ctx.load(b)
    res = lb.schedule(0, fields=("bound", "status", "n_groups", "n_seg", "n_rows"))
    assert (res["status"] == 0).all() and (st == 0).all()
    assert np.array_equal(res["bound"], want)


def test_full_config3_every_dag(ctx):
    b = wl.config(3)
    want, st = oracle.schedule_batch(b)
    lb = ctx.load(b)
    res = lb.schedule(0, fields=("bound", "status"))
    assert np.array_equal(res["bound"], want)


def test_config5_layered_sampled(ctx):
    """Large layered DAGs (CTA teams, global workspace): a sample of DAGs of the full batch
    in full detail, every DAG's bound against properties that hold at any size."""
    b = wl.config(5, n_dags=12)
    lb, res = gpu_schedule(ctx, b, 0, edges=False)
    sizes = np.diff(b.node_off)
    for d in np.argsort(sizes)[:3]:
        compare_dag(b, res, int(d), 0, edges=False)
    for d in range(b.n_dags):
        n0 = int(b.node_off[d])
        V = int(sizes[d])
        G = res["n_groups"][d]
        assert res["status"][d] == 0
        assert res["bound"][d] == res["group_R"][n0:n0 + G].sum()
        assert res["bound"][d] >= -(-int(b.wcet[n0:n0 + V].sum()) // b.M)
        assert res["n_rows"][d] == V + res["n_seg"][d]


@pytest.mark.slow
def test_config5_full_batch_three_largest_in_full(ctx):
    """The whole 200-DAG layered batch in the benchmark's launch configuration (CTA teams,
    global workspaces sized for the largest DAG); the three largest DAGs (about 20,000
    nodes each: the largest closures, released-set masks and Top_M ballots) are compared
    with the oracle in every output, their extra edges in a second run of just those three,
    and every DAG's bound against properties that hold at any size."""
    b = wl.config(5)
    lb, res = gpu_schedule(ctx, b, 0, edges=False)
    sizes = np.diff(b.node_off)
    big = [int(d) for d in np.argsort(sizes)[-3:]]
    assert min(sizes[big]) > 19000
    for d in big:
        compare_dag(b, res, d, 0, edges=False)
    for d in range(b.n_dags):
        n0, V, G = int(b.node_off[d]), int(sizes[d]), res["n_groups"][d]
        assert res["status"][d] == 0
        assert res["bound"][d] == res["group_R"][n0:n0 + G].sum()
        assert res["bound"][d] >= -(-int(b.wcet[n0:n0 + V].sum()) // b.M)
        assert res["n_rows"][d] == V + res["n_seg"][d]
    lb.free()
    _check_batch(ctx, b.subset(big), 0, edges=True)


@pytest.mark.parametrize("variant", [0, 3])
def test_mid_size_dags_mask_summary_and_top_m(ctx, variant):
    """DAGs of 600-1,500 nodes: released-set masks of 10-24 words (walked through their
    summary of non-empty words), blocks wider than M (Top_M by rank-order ballots), CTA
    teams with shared- and global-memory workspaces; every output bit-exact."""
    b = wl.small_config(4, 6, 600, 1500, seed=61)
    _check_batch(ctx, b, variant)
    layered = []
    rng = np.random.default_rng(62)
    for _ in range(3):
        V = int(rng.integers(700, 1400))
        s, t = wl.layered_edges(rng, V, int(rng.integers(3, 8)), max_width=400)
        rp, col = wl.csr_from_edges(V, s, t)
        layered.append((rp, col, wl.wcet_lognormal(rng, V), wl.k64_uniform(rng, V, 0.3)))
    _check_batch(ctx, wl.from_dags(layered, 148), variant)
