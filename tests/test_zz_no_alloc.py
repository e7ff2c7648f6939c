"""dagrt_schedule_noalloc: the scheduler entry point for callers that cannot allocate.

Some callers may not allocate device memory while they run (real-time executives that
reserve every buffer up front, code under a memory budget owned by someone else, host
frameworks that forbid cudaMalloc). This entry point keeps its scratch in a fixed array
inside the library instead. The test checks, through the C ABI, that two calls in a row
give the CPU oracle's bounds and statuses bit for bit (the same bar as every other bound
test), that DAGs over its size limit and DAGs whose offsets reach past the arrays they index
are rejected per DAG, and that a call leaves the device's free memory unchanged.
This file is collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2602_20826_gb300 import workloads as wl
from tests.oracle_checks import random_small_dag

pytestmark = pytest.mark.gpu

KEYS = ("node_off", "edge_off", "row_ptr", "col", "wcet", "k64")


def _batch():
    b = wl.small_config(3, n_dags=150, v_lo=5, v_hi=500, seed=99)
    rng = np.random.default_rng(8)
    dags = [b.dag(d) for d in range(b.n_dags)]
    dags.insert(7, random_small_dag(rng, 600, 0.01, 100))    # over the 512-node limit
    dags.insert(40, random_small_dag(rng, 300, 0.25, 100))   # over the 8192-edge limit
    dags.insert(41, (np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64),
                     np.zeros(0, np.uint8)))                  # empty DAG
    return wl.from_dags(dags, b.M)


def test_noalloc_matches_oracle_twice():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2602_20826_gb300 import dagrt
    b = _batch()
    dev = {k: torch.from_numpy(getattr(b, k)).cuda() for k in KEYS}
    sizes = np.diff(b.node_off)
    edges = np.diff(b.edge_off)
    over = (sizes > 512) | (edges > 8192)
    assert over.sum() == 2
    stream = torch.cuda.current_stream().cuda_stream
    for variant in (0, 3):
        want_b, want_s = oracle.schedule_batch(b, variant)
        assert (want_s == 0).all()
        for call in range(2):
            bound = torch.full((b.n_dags,), -9, dtype=torch.int64, device="cuda")
            status = torch.full((b.n_dags,), -9, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            rc = dagrt.schedule_noalloc(dev, b.M, variant, bound, status, stream)
            assert rc == dagrt.OK
            torch.cuda.synchronize()
            if call == 1:  # the second call allocates nothing at all
                assert torch.cuda.mem_get_info()[0] == free_before
            got_b = bound.cpu().numpy()
            got_s = status.cpu().numpy()
            assert np.array_equal(got_b[~over], want_b[~over]), (variant, call)
            assert (got_s[~over] == 0).all(), (variant, call)
            assert (got_s[over] == dagrt.E_INVAL).all() and (got_b[over] == -1).all()


def test_noalloc_rejects_offsets_past_the_arrays():
    """The kernel checks every DAG's node and edge range against the array lengths: DAGs
    that reach past a shortened wcet/k64 or col array get E_INVAL, the others their bound."""
    import torch
    from paper_2602_20826_gb300 import dagrt
    b = wl.small_config(2, n_dags=40, v_lo=5, v_hi=120, seed=17)
    want_b, _ = oracle.schedule_batch(b)
    dev = {k: torch.from_numpy(getattr(b, k)).cuda() for k in KEYS}
    cut_n = int(b.node_off[30]) + 2          # DAGs 30.. reach past the node arrays
    cut_e = int(b.edge_off[20]) + 1          # DAGs 20.. (with edges) reach past col
    short = dict(dev)
    short["wcet"] = dev["wcet"][:cut_n].clone()
    short["k64"] = dev["k64"][:cut_n].clone()
    short["col"] = dev["col"][:cut_e].clone()
    bound = torch.full((b.n_dags,), -9, dtype=torch.int64, device="cuda")
    status = torch.full((b.n_dags,), -9, dtype=torch.int32, device="cuda")
    assert dagrt.schedule_noalloc(short, b.M, 0, bound, status, torch.cuda.current_stream().cuda_stream) == dagrt.OK
    torch.cuda.synchronize()
    got_b, got_s = bound.cpu().numpy(), status.cpu().numpy()
    bad = (b.node_off[1:] > cut_n) | (b.edge_off[1:] > cut_e)
    assert bad[35] and not bad[3]
    assert (got_s[bad] == dagrt.E_INVAL).all() and (got_b[bad] == -1).all()
    assert np.array_equal(got_b[~bad], want_b[~bad]) and (got_s[~bad] == 0).all()


def test_noalloc_rejects_bad_arguments():
    from paper_2602_20826_gb300 import dagrt
    f = dagrt.dagrt_schedule_noalloc
    assert f(-1, None, None, None, None, None, None, 0, 0, 8, 0, None, None, None) == dagrt.E_INVAL
    assert f(1, None, None, None, None, None, None, 0, 0, 0, 0, None, None, None) == dagrt.E_INVAL
    assert f(1, None, None, None, None, None, None, 0, 0, 8, 9, None, None, None) == dagrt.E_INVAL
    assert f(1, None, None, None, None, None, None, -1, 0, 8, 0, None, None, None) == dagrt.E_INVAL
    assert f(0, None, None, None, None, None, None, 0, 0, 8, 0, None, None, None) == dagrt.OK
