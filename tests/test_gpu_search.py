"""GPU parity of dagrt_search (generated candidates, exact bounds, argmin) against the CPU
oracle's implementation of the same counter-based generator and bound."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2602_20826_gb300 import workloads as wl
from tests.gpu_helpers import context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    return context()


def _want_m(b, d, var, rc, n_alloc, levels, seed, mode):
    """The winning candidate's allocation, row by row, from the oracle's definitions."""
    _, plan = oracle.schedule_dag_of(b, d, var)
    n = plan["n_rows"]
    if mode == oracle.SEARCH_RANDOM:
        return oracle.generated_allocation(seed, d, rc, n, levels, n_alloc)
    a = rc % n_alloc
    out = np.zeros(n, np.uint8)
    if mode == oracle.SEARCH_EXHAUSTIVE:
        B = len(levels) + 1
        for r, u in enumerate(oracle.row_owner(plan)):
            dg = (a // B ** int(u)) % B
            out[r] = 0 if dg == 0 else levels[dg - 1]
        return out
    if a:
        codes = oracle.generated_allocation(seed, d, rc, n, levels, n_alloc)
        out[:] = [oracle.perturbed_m(int(m0), int(c)) for m0, c in zip(plan["row_m0"], codes)]
    return out


def _check(ctx, b, variants, n_alloc, levels, seed, dags, mode=oracle.SEARCH_RANDOM):
    from paper_2602_20826_gb300 import dagrt
    assert (oracle.SEARCH_RANDOM, oracle.SEARCH_EXHAUSTIVE, oracle.SEARCH_PERTURB) == \
        (dagrt.SEARCH_RANDOM, dagrt.SEARCH_EXHAUSTIVE, dagrt.SEARCH_PERTURB)
    lb = ctx.load(b)
    for v in sorted(set(variants)):
        lb.schedule(v, fields=("status",))
    res = lb.search(variants, n_alloc, levels, seed, want_all=True, want_m=True, mode=mode)
    for d in dags:
        ref, rb, rc = oracle.search_dag_generated(b, d, variants, n_alloc, levels, seed, mode)
        assert np.array_equal(res["out_bound"][d], ref), (d, np.nonzero(res["out_bound"][d] != ref)[0][:5])
        assert res["best_bound"][d] == rb and res["best_cand"][d] == rc
        var = variants[rc // n_alloc]
        want_m = _want_m(b, d, var, rc, n_alloc, levels, seed, mode)
        n0 = int(b.node_off[d])
        assert np.array_equal(res["best_m"][2 * n0: 2 * n0 + len(want_m)], want_m)
    lb.free()
    return res


def test_config1_search(ctx):
    """One 20-node DAG, M = 8: the paper's allocation plus 4,096 generated ones."""
    b = wl.config(1)
    _check(ctx, b, [0], 4097, [1, 2, 4, 8], wl.BASE_SEED + 1, [0])


def test_config3_search_sampled(ctx):
    b = wl.config(3, n_dags=40)
    _check(ctx, b, [0, 1, 2, 3], 64, [1, 2, 4, 8, 16, 32], wl.BASE_SEED + 3, [0, 7, 19, 33])


def test_search_odd_levels_and_variants(ctx):
    b = wl.small_config(2, n_dags=30, v_lo=3, v_hi=120, seed=5)
    _check(ctx, b, [3, 0, 3], 7, [3, 5, 148, 200, 1], 12345, range(0, 30, 5))


def _tiny_batch(seed, n, vmax=8):
    from tests.oracle_checks import random_small_dag
    rng = np.random.default_rng(seed)
    dags = [random_small_dag(rng, int(rng.integers(1, vmax + 1)), 0.4, 12) for _ in range(n)]
    return wl.from_dags(dags, 6)


def test_exhaustive_search_matches_oracle():
    """Exhaustive mode on DAGs of at most 8 nodes: every allocation in
    ({schedule's m} + {1, 2, 4})^V of all four structure variants (4^8 = 65,536 per
    variant), each bound, the optimum and the winning allocation bit-exact."""
    import __graft_entry__ as g
    g.build()
    ctx = context()
    b = _tiny_batch(81, 24)
    levels = [1, 2, 4]
    _check(ctx, b, [0, 1, 2, 3], 4 ** 8, levels, 0, range(b.n_dags), mode=oracle.SEARCH_EXHAUSTIVE)


def test_perturbation_search_matches_oracle():
    """Perturbation mode (sparse changes of the schedule's own m: halve, -1, +1, double),
    config 3 sizes and a small M where 255-capping and halving to 1 occur."""
    ctx = context()
    codes = [0] * 12 + [1, 2, 3, 4]
    b = wl.config(3, n_dags=20)
    _check(ctx, b, [0, 1, 2, 3], 64, codes, wl.BASE_SEED + 5, [0, 7, 13, 19], mode=oracle.SEARCH_PERTURB)
    b2 = wl.small_config(2, n_dags=12, v_lo=3, v_hi=60, seed=3)
    b2 = wl.from_dags([b2.dag(d) for d in range(b2.n_dags)], 300)
    _check(ctx, b2, [0, 3], 33, [0, 1, 2, 3, 4], 99, range(12), mode=oracle.SEARCH_PERTURB)


def test_learned_proposals_never_beat_the_exhaustive_optimum():
    """The learned proposer's candidates (the schedule's allocation and per-node level
    assignments from the same levels) lie inside the exhaustive search space of the paper
    structure, so proposal + exact check can at best match the exhaustive optimum."""
    from paper_2602_20826_gb300.dagrt import Model
    ctx = context()
    b = _tiny_batch(82, 40)
    levels = [1, 2, 4]
    lb = ctx.load(b)
    lb.schedule(0, fields=("status",))
    ex = lb.search([0], 4 ** 8, levels, mode=oracle.SEARCH_EXHAUSTIVE)
    for seed in (1, 2):
        model = Model(ctx, levels, seed=seed)
        prop = model.propose(lb, 16)
        assert (prop["best_bound"] >= ex["best_bound"]).all()
        model.free()
    lb.free()
