"""GPU parity of the Evaluation section's pieces: the baseline bounds (Greedy, Greedy +
unaware, Graham_para) written by the scheduler, the no-repair structure variant, and the
schedulability flags of implicit-deadline tasks, against the CPU oracle, on the paper's
layered DAGs and on the measured workloads' distributions."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2602_20826_gb300 import workloads as wl
from tests.gpu_helpers import compare_dag, context, gpu_schedule

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    return context()


@pytest.mark.parametrize("M", [4, 32, 256])
def test_baselines_and_no_repair_on_paper_layered_dags(ctx, M):
    b = wl.paper_layered_batch(150, 16, M, 20, 7)
    for variant in (0, 4):
        lb, res = gpu_schedule(ctx, b, variant)
        for d in range(b.n_dags):
            compare_dag(b, res, d, variant)
        lb.free()


def test_baselines_extreme_loads(ctx):
    """Loads up to 2^32 - 1 with serial fractions: Greedy + unaware's 128-bit products and
    its saturation at 2^63 - 1."""
    rng = np.random.default_rng(95)
    dags = []
    for V in (1, 3, 40, 200):
        s, t = wl.er_edges(rng, V, 0.1)
        rp, col = wl.csr_from_edges(V, s, t)
        w = rng.integers(2**31, 2**32, size=V).astype(np.int64)
        dags.append((rp, col, w, rng.integers(0, 65, size=V).astype(np.uint8)))
    for M in (1, 148, 4096):
        b = wl.from_dags(dags, M)
        lb, res = gpu_schedule(ctx, b, 0, edges=False)
        for d in range(b.n_dags):
            compare_dag(b, res, d, 0, edges=False)
        assert (res["greedy_unaware"][:b.n_dags] <= 2**63 - 1).all()
        lb.free()


def test_schedulable_flags_match_oracle(ctx):
    import torch
    for b in (wl.paper_layered_batch(200, 16, 32, 20, 9), wl.config(2, n_dags=500)):
        lb = ctx.load(b)
        for variant in (0, 3, 4):
            lb.schedule(variant, fields=("status",))
            want, st = oracle.schedule_batch(b, variant)
            for U in (0.02, 0.3, 0.8):
                dl = wl.implicit_deadlines(b, U)
                ok, n = lb.schedulable(variant, dl)
                ref = ((want <= dl) & (st == 0)).astype(np.int32)
                assert np.array_equal(ok, ref) and n == int(ref.sum())
                # device pointers: flags and count stay on the GPU
                d_dl = torch.from_numpy(dl).cuda()
                d_ok = torch.full((b.n_dags,), -1, dtype=torch.int32, device="cuda")
                d_n = torch.zeros(1, dtype=torch.int64, device="cuda")
                from paper_2602_20826_gb300 import dagrt
                ctx.check(dagrt.dagrt_schedulable(lb.h, variant, d_dl.data_ptr(), d_ok.data_ptr(),
                                                  dagrt.C.cast(d_n.data_ptr(), dagrt.C.POINTER(dagrt.C.c_int64)),
                                                  dagrt.PTR_DEVICE))
                torch.cuda.synchronize()
                assert np.array_equal(d_ok.cpu().numpy(), ref) and int(d_n.item()) == int(ref.sum())
        lb.free()


def test_conditional_dags_match_oracle(ctx):
    """dagrt_cond_bound: every realisation of every conditional DAG bounded in one batched
    call; the adaptive and fixed bounds, the worst realisation and the realisation count
    against the realisation oracle."""
    from oracle import conditional as CD
    from tests.oracle_checks import random_small_dag
    rng = np.random.default_rng(97)
    dags, conds = [], []
    for _ in range(60):
        V = int(rng.integers(1, 14))
        dags.append(random_small_dag(rng, V, float(rng.uniform(0.1, 0.5)), int(rng.choice([5, 50, 400])), kmin=16))
        conds.append((rng.random(V) < 0.3).astype(np.uint8))
    for M in (3, 16, 148):
        b = wl.from_dags(dags, M)
        for variant in (0, 4):
            got = ctx.cond_bound(b, np.concatenate(conds), variant=variant)
            for d in range(b.n_dags):
                rp, col, w, k = b.dag(d)
                a, f, arg, n = CD.cond_bounds(rp, col, w, k, conds[d], M, variant)
                assert (got["adaptive"][d], got["fixed"][d], got["worst_real"][d], got["n_real"][d]) == (a, f, arg, n), d
