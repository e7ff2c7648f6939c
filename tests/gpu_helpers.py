"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and compare it
with the CPU oracle element by element."""
from __future__ import annotations

import numpy as np

import oracle

FIELDS = ("bound", "status", "n_groups", "n_seg", "n_rows", "n_extra", "level", "wanc", "block_of",
          "group_of", "exec_group", "m", "group_R", "seg_parent", "seg_load", "seg_m", "seg_group",
          "row_id", "row_group", "row_m0", "row_load", "greedy", "greedy_unaware", "graham_para", "crit_path")


def context():
    import torch
    from paper_2602_20826_gb300.dagrt import Context
    return Context(0, torch.cuda.current_stream().cuda_stream)


def gpu_schedule(ctx, batch, variant=0, fields=FIELDS, edges=True):
    lb = ctx.load(batch)
    cap = None
    if edges:
        # first pass: edge counts; second pass: edges
        cnt = lb.schedule(variant, fields=("n_extra",), check=False)["n_extra"]
        cap = np.maximum(cnt, 0)
    res = lb.schedule(variant, fields=fields, extra_cap=cap, check=False)
    return lb, res


def compare_dag(batch, res, d, variant=0, edges=True):
    """Compare every output of DAG d with the oracle; returns the oracle result."""
    rc, ref = oracle.schedule_dag_of(batch, d, variant, extra_cap=-1 if edges else 0)
    n0 = int(batch.node_off[d])
    V = batch.n_nodes(d)
    assert res["status"][d] == rc, (d, res["status"][d], rc)
    if "greedy" in res:  # the Evaluation section's baselines (-1 for a failed DAG)
        rb, g, u, gr = oracle.baselines(*batch.dag(d), batch.M)
        want = (g, u, gr) if rb == 0 else (-1, -1, -1)
        assert (res["greedy"][d], res["greedy_unaware"][d], res["graham_para"][d]) == want, (d, want)
    if "crit_path" in res:
        want = oracle.crit_path(ref, *batch.dag(d)[:2], batch.M) if rc == 0 else -1
        assert res["crit_path"][d] == want, (d, res["crit_path"][d], want)
    if rc != 0:
        assert res["bound"][d] == -1
        return ref
    assert res["bound"][d] == ref["bound"], (d, res["bound"][d], ref["bound"])
    for f in ("n_groups", "n_seg", "n_rows", "n_extra"):
        if f in res:
            assert res[f][d] == ref[f], (d, f, res[f][d], ref[f])
    for f in ("level", "wanc", "block_of", "group_of", "exec_group", "m"):
        if f in res:
            assert np.array_equal(res[f][n0:n0 + V], ref[f]), (d, f)
    if "group_R" in res:
        G = ref["n_groups"]
        assert np.array_equal(res["group_R"][n0:n0 + G], ref["group_R"]), (d, "group_R")
    if "seg_parent" in res:
        S = ref["n_seg"]
        for f in ("seg_parent", "seg_load", "seg_m", "seg_group"):
            assert np.array_equal(res[f][n0:n0 + S], ref[f]), (d, f)
    if "row_id" in res:
        R = ref["n_rows"]
        for f in ("row_id", "row_group", "row_m0", "row_load"):
            assert np.array_equal(res[f][2 * n0:2 * n0 + R], ref[f]), (d, f)
    if edges and "extra_off" in res:
        eo = res["extra_off"]
        got = np.stack([res["extra_src"][eo[d]:eo[d + 1]], res["extra_dst"][eo[d]:eo[d + 1]]], axis=1)
        assert got.shape == ref["extra"].shape and np.array_equal(got, ref["extra"]), (d, "extra")
    return ref
