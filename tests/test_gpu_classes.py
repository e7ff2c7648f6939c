"""Size classes of the scheduler at their boundaries: DAGs of 0, 1, 16, 17, 32, 33, 255, 256
and 257 nodes, a dense DAG that stays in a warp class (a large edge capacity for its class),
a dense DAG sent to a CTA team by its edge count, in a scrambled order; every output of every
DAG against the oracle, for several warp cutoffs. Also a batch loaded from host and from
device arrays in turn (the load's staging buffer is reused)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2602_20826_gb300 import workloads as wl
from tests.gpu_helpers import FIELDS, compare_dag, context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    return context()


def _dag(rng, V, p):
    s, t = [], []
    for i in range(V):
        for j in range(i + 1, V):
            if rng.random() < p:
                s.append(i)
                t.append(j)
    rp, col = wl.csr_from_edges(V, s, t)
    w = rng.integers(1, 5000, size=V).astype(np.int64)
    k = rng.integers(20, 65, size=V).astype(np.uint8)
    return rp, col, w, k


def _boundary_batch():
    rng = np.random.default_rng(2026)
    dags = [_dag(rng, V, 0.1) for V in (0, 1, 16, 17, 32, 33, 255, 256, 257)]
    dags.append(_dag(rng, 64, 1.0))  # 2,016 edges: a warp class with a large edge capacity
    dags.append(_dag(rng, 80, 1.0))  # 3,160 edges > 12 x 256: a CTA team
    order = rng.permutation(len(dags))
    return wl.from_dags([dags[i] for i in order], 148, "class-boundaries")


def test_class_boundaries_match_the_oracle(ctx):
    b = _boundary_batch()
    lb = ctx.load(b)
    for w in (256, 128, 0):
        lb.set_tuning(warp_max_v=w, cta_smem=2)
        res = lb.schedule(0, fields=FIELDS, check=False)  # no extra edges written
        for d in range(b.n_dags):
            compare_dag(b, res, d, 0, edges=False)
        cnt = lb.schedule(0, fields=("n_extra",), check=False)["n_extra"]  # and with them
        res = lb.schedule(0, fields=FIELDS, extra_cap=np.maximum(cnt, 0), check=False)
        for d in range(b.n_dags):
            compare_dag(b, res, d, 0, edges=True)
    lb.free()


def test_host_and_device_loads_in_turn(ctx):
    import torch
    b = wl.small_config(2, 40, 5, 200, seed=77)
    keys = ("node_off", "edge_off", "row_ptr", "col", "wcet", "k64")
    dev = {k: torch.from_numpy(getattr(b, k)).cuda() for k in keys}
    ref = [oracle.schedule_dag_of(b, d)[1]["bound"] for d in range(b.n_dags)]
    for i in range(6):
        lb = ctx.load(b) if i % 2 == 0 else ctx.load(dev, M=b.M)
        got = lb.schedule(0, fields=("bound", "status"))
        assert (got["status"] == 0).all() and list(got["bound"]) == ref
        lb.free()
