"""Batching controls and CUDA graphs: every launch-shape setting gives bit-identical
results (checked against the oracle), the autotuner keeps a valid setting, and a captured
graph replays the same work -- on whatever the device buffers hold at replay time."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2602_20826_gb300 import workloads as wl
from tests.gpu_helpers import FIELDS, context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    return context()


def _mixed_batch():
    # small, medium and large DAGs, so every size class and the CTA teams are used
    b1 = wl.small_config(2, 30, 5, 60, seed=41)
    b2 = wl.small_config(3, 12, 150, 420, seed=42)
    dags = [b1.dag(d) for d in range(b1.n_dags)] + [b2.dag(d) for d in range(b2.n_dags)]
    order = np.random.default_rng(3).permutation(len(dags))
    return wl.from_dags([dags[i] for i in order], 148, "mixed")


def test_schedule_identical_for_every_warp_cutoff(ctx):
    b = _mixed_batch()
    lb = ctx.load(b)
    ref = None
    for w, cs in ((256, 1), (256, 0), (0, 1), (0, 0), (64, 2), (128, 3), (192, 4)):
        lb.set_tuning(warp_max_v=w, cta_smem=cs)
        assert lb.tuning()["warp_max_v"] == w and lb.tuning()["cta_smem"] == cs
        res = lb.schedule(0, fields=FIELDS, check=False)
        if ref is None:
            ref = res
            for d in range(0, b.n_dags, 5):
                rc, o = oracle.schedule_dag_of(b, d)
                assert res["status"][d] == rc and res["bound"][d] == o["bound"]
        else:
            for f in FIELDS:
                assert np.array_equal(res[f], ref[f]), (w, f)
    lb.free()


def test_bound_identical_for_every_chunking(ctx):
    b = wl.config(3, n_dags=30)
    alloc, stride = wl.candidate_allocations(b, 2, 128, [1, 2, 4, 8, 16, 32, 3, 0], seed=8)
    lb = ctx.load(b)
    for v in (0, 2):
        lb.schedule(v, fields=("status",))
    ref = None
    for cr, wp in ((24, 4), (8, 1), (100, 8), (16, 2), (256, 3)):
        lb.set_tuning(chunk_rows=cr, item_warps=wp)
        ob, bb, bc = lb.bound([0, 2], 128, alloc, stride)
        if ref is None:
            ref = (ob, bb, bc)
            for d in range(0, 30, 6):
                r, rb, rcand = oracle.search_dag(b, d, alloc, stride, 2, 128, [0, 2])
                assert np.array_equal(ob[d], r) and bb[d] == rb and bc[d] == rcand
        else:
            assert np.array_equal(ob, ref[0]) and np.array_equal(bb, ref[1]) and np.array_equal(bc, ref[2]), (cr, wp)
    lb.free()


def test_tuning_rejects_bad_values(ctx):
    from paper_2602_20826_gb300.dagrt import DagrtError, E_INVAL
    lb = ctx.load(wl.small_config(2, 3, 5, 20, seed=1))
    for kw in ({"warp_max_v": 100}, {"chunk_rows": 4}, {"chunk_rows": 300}, {"item_warps": 0}, {"item_warps": 9},
               {"cta_smem": 5}, {"cta_smem": -1}):
        with pytest.raises(DagrtError) as e:
            lb.set_tuning(**kw)
        assert e.value.code == E_INVAL
    lb.free()


def test_autotuner_keeps_a_valid_setting(ctx):
    import torch
    b = wl.config(3, n_dags=60)
    lb = ctx.load(b)
    t, ms = lb.autotune_schedule(0, reps=2)
    assert t["warp_max_v"] in (64, 128, 192, 256) and ms > 0
    assert lb.tuning() == t
    for v in range(4):
        lb.schedule(v, fields=("status",))
    alloc, stride = wl.candidate_allocations(b, 4, 64, [1, 2, 4, 8, 16, 32], seed=wl.BASE_SEED + 13)
    t2, ms2 = lb.autotune_bound([0, 1, 2, 3], 64, torch.from_numpy(alloc).cuda(), stride, reps=2)
    assert t2["chunk_rows"] in (24, 32, 48, 64) and t2["item_warps"] in (2, 4, 8) and ms2 > 0
    ob, bb, bc = lb.bound([0, 1, 2, 3], 64, alloc, stride)
    for d in (0, 17, 59):
        r, rb, rc = oracle.search_dag(b, d, alloc, stride, 4, 64, [0, 1, 2, 3])
        assert np.array_equal(ob[d], r) and bb[d] == rb and bc[d] == rc
    lb.free()


def test_graph_replays_schedule_and_bound(ctx):
    """Capture schedule (device outputs) + candidate bounds; replay twice; change the WCETs
    in place between replays and compare with the oracle on the new values."""
    import torch
    b = wl.config(3, n_dags=40)
    keys = ("node_off", "edge_off", "row_ptr", "col", "wcet", "k64")
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(b, k))).cuda() for k in keys}
    lb = ctx.load(dev, b.M)
    alloc, stride = wl.candidate_allocations(b, 1, 64, [1, 2, 4, 8, 16, 32], seed=4)
    da = torch.from_numpy(alloc).cuda()
    nd = b.n_dags
    sched = {"bound": torch.zeros(nd, dtype=torch.int64, device="cuda"),
             "status": torch.zeros(nd, dtype=torch.int32, device="cuda")}
    ob = torch.zeros(nd * 64, dtype=torch.int64, device="cuda")
    bb = torch.zeros(nd, dtype=torch.int64, device="cuda")
    bc = torch.zeros(nd, dtype=torch.int32, device="cuda")
    # one eager round first, so that every buffer exists before the capture
    lb.schedule(0, out=sched)
    lb.bound([0], 64, da, stride, ob, bb, bc)
    torch.cuda.synchronize()
    l0 = ctx.launches()
    ctx.graph_begin()
    lb.schedule(0, out=sched)
    lb.bound([0], 64, da, stride, ob, bb, bc)
    g = ctx.graph_end()
    assert ctx.launches() == l0  # recorded, not run
    for trial in range(2):
        if trial == 1:  # new WCETs, same structure
            w = b.wcet.copy()
            w[::3] = np.maximum(1, w[::3] // 2 + 7)
            b.wcet[:] = w
            dev["wcet"].copy_(torch.from_numpy(w))
        sched["bound"].zero_()
        ob.zero_()
        g.launch()
        torch.cuda.synchronize()
        got_s = sched["bound"].cpu().numpy()
        got = ob.cpu().numpy().reshape(nd, 64)
        for d in range(0, nd, 4):
            rc, o = oracle.schedule_dag_of(b, d)
            assert got_s[d] == o["bound"], (trial, d)
            r, rb, rcand = oracle.search_dag(b, d, alloc, stride, 1, 64, [0])
            assert np.array_equal(got[d], r), (trial, d)
            assert bb[d].item() == rb and bc[d].item() == rcand
    assert ctx.launches() > l0
    g.free()
    lb.free()


def test_host_calls_are_refused_during_capture(ctx):
    from paper_2602_20826_gb300.dagrt import DagrtError, E_INVAL
    b = wl.small_config(2, 5, 5, 30, seed=2)
    lb = ctx.load(b)
    lb.schedule(0)
    ctx.graph_begin()
    assert lb.schedule(0)["rc"] == E_INVAL  # host outputs (the binding reports the code)
    with pytest.raises(DagrtError) as e:
        lb.search([0], 4, [1, 2], 1)  # host outputs
    assert e.value.code == E_INVAL
    with pytest.raises(DagrtError):
        ctx.load(b)
    g = ctx.graph_end()  # the capture is still intact (nothing was recorded)
    g.launch()
    g.free()
    assert lb.schedule(0)["status"].tolist() == [0] * 5
    lb.free()
