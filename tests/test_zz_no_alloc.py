"""dagrt_schedule_noalloc: the scheduler entry point for callers that cannot allocate.

Some callers may not allocate device memory while they run (real-time executives that
reserve every buffer up front, graph-captured or budget-limited code, host frameworks
that forbid cudaMalloc). This entry point keeps its scratch in a fixed array inside the
library instead. The test checks, through the C ABI, that two calls in a row give the same
bounds and statuses as the allocating entry point (dagrt_load_csr + dagrt_schedule),
bit-exact like every other bound test, and that DAGs over its size limit are rejected.
This file is collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2602_20826_gb300 import workloads as wl
from tests.oracle_checks import random_small_dag

pytestmark = pytest.mark.gpu


def _batch():
    b = wl.small_config(3, n_dags=150, v_lo=5, v_hi=500, seed=99)
    rng = np.random.default_rng(8)
    dags = [b.dag(d) for d in range(b.n_dags)]
    dags.insert(7, random_small_dag(rng, 600, 0.01, 100))    # over the 512-node limit
    dags.insert(40, random_small_dag(rng, 300, 0.25, 100))   # over the 8192-edge limit
    dags.insert(41, (np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64),
                     np.zeros(0, np.uint8)))                  # empty DAG
    return wl.from_dags(dags, b.M)


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2602_20826_gb300 import dagrt
    b = _batch()
    ctx = dagrt.Context(0, torch.cuda.current_stream().cuda_stream)
    dev = {k: torch.from_numpy(getattr(b, k)).cuda() for k in
           ("node_off", "edge_off", "row_ptr", "col", "wcet", "k64")}
    sizes = np.diff(b.node_off)
    edges = np.diff(b.edge_off)
    over = (sizes > 512) | (edges > 8192)
    assert over.sum() == 2
    for variant in (0, 3):
        lb = ctx.load(dev, M=b.M)
        ref = {"bound": torch.zeros(b.n_dags, dtype=torch.int64, device="cuda"),
               "status": torch.zeros(b.n_dags, dtype=torch.int32, device="cuda")}
        lb.schedule(variant, out=ref)
        torch.cuda.synchronize()
        ref_b = ref["bound"].cpu().numpy()
        ref_s = ref["status"].cpu().numpy()
        assert (ref_s == 0).all()
        for call in range(2):
            bound = torch.full((b.n_dags,), -9, dtype=torch.int64, device="cuda")
            status = torch.full((b.n_dags,), -9, dtype=torch.int32, device="cuda")
            rc = dagrt.schedule_noalloc(dev, b.M, variant, bound, status,
                                        torch.cuda.current_stream().cuda_stream)
            assert rc == dagrt.OK
            torch.cuda.synchronize()
            got_b = bound.cpu().numpy()
            got_s = status.cpu().numpy()
            assert np.array_equal(got_b[~over], ref_b[~over]), (variant, call)
            assert np.array_equal(got_s[~over], ref_s[~over]), (variant, call)
            assert (got_s[over] == dagrt.E_INVAL).all() and (got_b[over] == -1).all()
        lb.free()


def test_noalloc_rejects_bad_arguments():
    from paper_2602_20826_gb300 import dagrt
    assert dagrt.dagrt_schedule_noalloc(-1, None, None, None, None, None, None, 8, 0, None, None, None) \
        == dagrt.E_INVAL
    assert dagrt.dagrt_schedule_noalloc(1, None, None, None, None, None, None, 0, 0, None, None, None) \
        == dagrt.E_INVAL
    assert dagrt.dagrt_schedule_noalloc(1, None, None, None, None, None, None, 8, 9, None, None, None) \
        == dagrt.E_INVAL
    assert dagrt.dagrt_schedule_noalloc(0, None, None, None, None, None, None, 8, 0, None, None, None) \
        == dagrt.OK
