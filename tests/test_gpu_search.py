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


def _check(ctx, b, variants, n_alloc, levels, seed, dags):
    lb = ctx.load(b)
    for v in sorted(set(variants)):
        lb.schedule(v, fields=("status",))
    res = lb.search(variants, n_alloc, levels, seed, want_all=True, want_m=True)
    plan_rows = {}
    for d in dags:
        ref, rb, rc = oracle.search_dag_generated(b, d, variants, n_alloc, levels, seed)
        assert np.array_equal(res["out_bound"][d], ref), (d, np.nonzero(res["out_bound"][d] != ref)[0][:5])
        assert res["best_bound"][d] == rb and res["best_cand"][d] == rc
        var = variants[rc // n_alloc]
        if var not in plan_rows:
            plan_rows[var] = {}
        _, plan = oracle.schedule_dag_of(b, d, var)
        want_m = oracle.generated_allocation(seed, d, rc, plan["n_rows"], levels, n_alloc)
        n0 = int(b.node_off[d])
        assert np.array_equal(res["best_m"][2 * n0: 2 * n0 + plan["n_rows"]], want_m)
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
