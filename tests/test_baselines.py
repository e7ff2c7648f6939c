"""The Evaluation section's baseline bounds (Greedy, Greedy + unaware, Graham_para) in the
oracle, pinned by hand values and closed forms, and the paper's qualitative trends of the
normalised makespan (Figs. 4-6) on its synthetic layered DAGs, recomputed with the oracle.

The figures themselves are missing from the paper and its DAG generator is not available,
so the trends are checked, not numbers; where this implementation's trend differs from the
paper's text, the test records what it finds."""
from __future__ import annotations

import math

import numpy as np

import oracle
from paper_2602_20826_gb300 import workloads as wl
from tests.oracle_checks import amdahl_time, hop_levels, random_small_dag, succ_lists


def test_worked_example_baselines():
    """The 7-node example at M = 6 (loads 1, 4, 2, 2, 4, 4, 1): every kernel fits the GPU,
    so Greedy and Greedy + unaware give each C = 1 and sum to 7; the longest path v1 v3 v5
    v7 has 4 nodes and the loads sum to 18, so Graham_para = 4 + ceil(14 / 6) = 7; the
    proposed bound is 5."""
    rp, col = wl.csr_from_edges(7, [0, 0, 0, 2, 3, 3, 1, 4, 5], [1, 2, 3, 4, 4, 5, 6, 6, 6])
    w = np.array([1, 4, 2, 2, 4, 4, 1])
    k = np.full(7, 64, np.uint8)
    assert oracle.baselines(rp, col, w, k, 6) == (0, 7, 7, 7)
    assert oracle.schedule(rp, col, w, k, 6)[1]["bound"] == 5


def test_baselines_closed_forms():
    rng = np.random.default_rng(91)
    for _ in range(80):
        V = int(rng.integers(1, 30))
        rp, col, w, k = random_small_dag(rng, V, float(rng.uniform(0.05, 0.5)), 300)
        # M = 1: one SM, everything sequential: Greedy = Graham_para = sum of loads;
        # Greedy + unaware runs a kernel on C^ SMs in C^ waves: C^ * C^ (1 - f) + C^ f
        rc, g, u, gr = oracle.baselines(rp, col, w, k, 1)
        assert rc == 0 and g == gr == int(w.sum())
        f = [int(x) for x in k]
        assert u == sum(math.ceil(int(x) * int(x) * (64 - kk) / 64 + int(x) * kk / 64)
                        for x, kk in zip(w, f))
        # any M: Greedy is the sum of Eq.1 times on min(C^, M) SMs; with M >= every load
        # the two greedy variants coincide (all kernels get their maximum parallelism)
        M = int(rng.integers(1, 400))
        rc, g, u, gr = oracle.baselines(rp, col, w, k, M)
        assert g == sum(amdahl_time(int(x), int(kk), min(int(x), M), M) for x, kk in zip(w, k))
        if M >= int(w.max()):
            assert u == g
        L = 1 + max(hop_levels(rp, col))
        assert gr == L + -(-(int(w.sum()) - L) // M)


def test_greedy_variants_coincide_for_fully_parallel_kernels():
    """With whole ticks (Eq.1 rounded up) and f = 1, a kernel on min(C^, M) SMs and one on
    C^ SMs both take ceil(C^ / M) ticks, so Greedy and Greedy + unaware are equal; they
    differ only for kernels with a serial part."""
    rng = np.random.default_rng(92)
    differs = 0
    for _ in range(60):
        rp, col, w, k = random_small_dag(rng, 12, 0.3, 500)
        M = int(rng.integers(1, 64))
        k64 = np.full(12, 64, np.uint8)
        _, g, u, _ = oracle.baselines(rp, col, w, k64, M)
        assert g == u
        _, g, u, _ = oracle.baselines(rp, col, w, k, M)
        differs += u > g
    assert differs > 0


def test_graham_para_bounds_every_list_schedule_of_the_unit_dag():
    """Graham's bound holds for the transformed DAG: a greedy list schedule of the unit
    loads (each node's C^ units become ready when its predecessors' units are done) on M
    processors never takes longer than Graham_para."""
    rng = np.random.default_rng(93)
    for _ in range(80):
        V = int(rng.integers(1, 12))
        M = int(rng.integers(1, 6))
        rp, col, w, k = random_small_dag(rng, V, 0.3, 6)
        succ = succ_lists(rp, col)
        pred = [[u for u in range(V) if v in succ[u]] for v in range(V)]
        left = [int(x) for x in w]
        done_at = [None] * V
        t = 0
        while any(d is None for d in done_at):
            ready = [v for v in range(V) if done_at[v] is None and left[v] > 0 and
                     all(done_at[p] is not None and done_at[p] <= t for p in pred[v])]
            cap = M
            for v in sorted(ready, key=lambda v: (int(rng.integers(0, 100)), v)):
                take = min(cap, left[v])
                left[v] -= take
                cap -= take
                if left[v] == 0:
                    done_at[v] = t + 1
            t += 1
        _, _, _, gr = oracle.baselines(rp, col, w, k, M)
        assert max(done_at) <= gr


def _trend(n, P, M, c_avg, seed, dlo=5, dhi=8):
    b = wl.paper_layered_batch(n, P, M, c_avg, seed, dlo, dhi)
    out = []
    for d in range(n):
        rp, col, w, k = b.dag(d)
        rc, r = oracle.schedule(rp, col, w, k, M, 0, extra_cap=0)
        _, g, u, gr = oracle.baselines(rp, col, w, k, M)
        out.append((r["bound"] / u, g / u, gr / u))
    return np.mean(out, axis=0)


def test_normalised_makespan_trends():
    """Figs. 4-6 of the paper as trends (normalised to Greedy + unaware), loads with mean 20:
      * vs M (P = 16): the gap to Greedy is below 3% for M <= 8 and widens as M grows; at
        M = 128 the proposed bound is 20-35% below Graham_para;
      * vs P (M = 32, P = 4..10): the proposed bound is the lowest of the three;
      * vs depth (P = 32, M = 32): the advantage over Greedy grows with the depth, to about
        a third.
    Findings where this implementation departs from the paper's text (kept as assertions
    so that they stay visible): the gap to Greedy grows with P here (the paper reports it
    shrinking from 23.9% to 13.7%), and Graham_para is below the proposed bound for M <= 32
    and for P = 32 (integer SMs of Eq.5 cost up to a tick per group that Graham's unit-load
    bound does not pay)."""
    by_m = {M: _trend(60, 16, M, 20, 1) for M in (4, 8, 32, 128)}
    gap_g = {M: 1 - v[0] / v[1] for M, v in by_m.items()}
    assert gap_g[4] < 0.03 and gap_g[8] < 0.03
    assert gap_g[4] < gap_g[8] < gap_g[32] < gap_g[128]
    assert 0.20 < 1 - by_m[128][0] / by_m[128][2] < 0.35
    assert by_m[8][2] < by_m[8][0]  # finding: Graham_para lower at small M
    by_p = {P: _trend(60, P, 32, 20, 2) for P in (4, 10)}
    for v in by_p.values():
        assert v[0] < v[1] and v[0] < v[2]
    assert 1 - by_p[4][0] / by_p[4][1] < 1 - by_p[10][0] / by_p[10][1]  # finding: grows with P
    shallow, deep = _trend(30, 32, 32, 20, 3, 4, 4), _trend(30, 32, 32, 20, 3, 32, 32)
    assert 1 - shallow[0] / shallow[1] < 1 - deep[0] / deep[1] < 0.4
    assert deep[2] < deep[0]  # finding: Graham_para lower at P = 32


def test_schedulability_sweep_trends():
    """Schedulable share (R(G) <= D = T, implicit deadlines at normalised utilisation U =
    sum C^ / (M T)) on the paper's layered DAGs (M = 32, P = 16, loads of mean 20): it can
    only fall as U grows; keeping Eq.5's sum within M (the repair) never schedules fewer
    DAGs than leaving the rounded SMs as they are, and at moderate U it schedules many more
    (the unrepaired over-full groups run in sequence)."""
    b = wl.paper_layered_batch(120, 16, 32, 20, 5)
    bounds = {v: oracle.schedule_batch(b, v)[0] for v in (oracle.VAR_PAPER, oracle.VAR_LITERAL, oracle.VAR_NOREPAIR)}
    prev = {v: 1.0 for v in bounds}
    gain = 0.0
    for U in (0.2, 0.4, 0.6, 0.7, 0.8, 0.9, 1.0):
        dl = wl.implicit_deadlines(b, U)
        assert (dl * 32 * U >= np.add.reduceat(b.wcet, b.node_off[:-1]) - 1e-6).all()
        share = {v: float(np.mean(bounds[v] <= dl)) for v in bounds}
        for v in bounds:
            assert share[v] <= prev[v]
        assert share[oracle.VAR_PAPER] >= share[oracle.VAR_NOREPAIR]
        gain = max(gain, share[oracle.VAR_PAPER] - share[oracle.VAR_NOREPAIR])
        prev = share
    assert gain > 0.2
    assert prev[oracle.VAR_PAPER] == 0.0  # at U = 1 no DAG with any serial step fits
