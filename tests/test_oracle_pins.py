"""Pins of the CPU oracle against what the paper and mathematics fix.

Every test here checks the oracle against something other than itself: the paper's
printed worked example, hand-computed values, closed forms of special DAG families,
properties recomputed by brute force (reachability, longest paths) and the paper's
lemma/theorem invariants.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_2602_20826_gb300 import workloads as wl
from tests.oracle_checks import (amdahl_time, ancestors_by_search, hop_levels,
                                 longest_weighted_path, random_small_dag, succ_lists)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt")


def _golden():
    kv = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    return kv


def _groups_of(res):
    G = res["n_groups"]
    return [sorted(int(v) for v in np.nonzero(res["group_of"] == j)[0]) for j in range(G)]


# ------------------------------------------------------------ worked example

def test_worked_example_every_printed_value():
    g = _golden()
    edges = [tuple(int(x) - 1 for x in e.split(">")) for e in g["edges"].split()]
    V = 7
    rp, col = wl.csr_from_edges(V, [a for a, _ in edges], [b for _, b in edges])
    w = np.array([int(x) for x in g["wcet"].split()], np.int64)
    k = np.array([int(x) for x in g["k64"].split()], np.uint8)
    M = int(g["M"])
    rc, r = oracle.schedule(rp, col, w, k, M)
    assert rc == oracle.OK
    # Theta (Sec. 3.1/3.2 example): v5 then v7
    assert [t + 1 for t in r["theta"]] == [int(x) for x in g["theta"].split()]
    # blocks B1..B3
    blocks = [sorted(int(x) for x in b.split(",")) for b in g["blocks"].split("|")]
    got = [sorted(int(v) + 1 for v in np.nonzero(r["block_of"] == b)[0]) for b in range(3)]
    assert got == blocks
    # local complete paths of B1 and B2 (from the in-block forest of the oracle's blocks)
    succ = succ_lists(rp, col)
    for bi, key in ((0, "paths_block1"), (1, "paths_block2")):
        members = set(np.nonzero(r["block_of"] == bi)[0].tolist())
        inpred = {v: [u for u in members if v in succ[u]] for v in members}
        paths = []

        def walk(v, acc):
            kids = [s for s in succ[v] if s in members]
            if not kids:
                paths.append(tuple(x + 1 for x in acc + [v]))
            for s in kids:
                walk(s, acc + [v])
        for v in sorted(members):
            if not inpred[v]:
                walk(v, [])
        want = sorted(tuple(int(x) for x in p.split(",")) for p in g[key].split("|"))
        assert sorted(paths) == want
    # Pi
    want_groups = [sorted(int(x) for x in grp.split(",")) for grp in g["groups"].split("|")]
    assert [[v + 1 for v in grp] for grp in _groups_of(r)] == want_groups
    # Sec. 4.1: m3 = m4 = 2 in pi_2; para(pi_2) = {v2}; WS_2 = 2; split of v2 into 2 + 2
    rows2 = [i for i in range(r["n_rows"]) if r["row_group"][i] == 1]
    m_of = {int(r["row_id"][i]): int(r["row_m0"][i]) for i in rows2}
    assert m_of[2] == int(g["m_3"]) and m_of[3] == int(g["m_4"])
    S2 = M - (m_of[2] + m_of[3])
    assert int(r["group_R"][1]) * S2 == int(g["ws_group2"])
    assert r["n_seg"] == 1
    assert int(r["seg_parent"][0]) + 1 == int(g["segment_parent"]) == int(g["para_group2"])
    p, rest = (int(x) for x in g["segment_loads"].split())
    assert int(r["seg_load"][0]) == p
    resid = [i for i in range(r["n_rows"]) if r["row_id"][i] == 1]
    assert len(resid) == 1 and int(r["row_load"][resid[0]]) == rest and r["row_group"][resid[0]] == 2
    assert int(r["seg_m"][0]) == int(g["segment_m"])
    # extra dependencies (v_{2,1}, v5) and (v3, v_{2,2})
    want_e = set()
    for e in g["extra_edges"].split():
        a, b = e.split(">")
        want_e.add((V if a == "seg" else int(a) - 1, int(b) - 1))
    assert set(map(tuple, r["extra"].tolist())) == want_e
    # Sec. 4.2: R(G) <= 5
    assert r["bound"] == int(g["bound"])


# ------------------------------------------------------------------- Eq.1

@pytest.mark.parametrize("load,k,m,M,want", [
    (4, 64, 2, 6, 2),      # ceil(4/2)
    (7, 64, 3, 6, 3),      # ceil(7/3)
    (10, 64, 8, 6, 3),     # two waves: ceil(2*10/8)
    (10, 0, 4, 8, 10),     # no parallel part: no speed-up
    (100, 32, 4, 8, 63),   # 100*(1/2 + 1/8) = 62.5
    (1, 64, 5, 8, 1),      # t_min = 1
    (3, 64, 12, 4, 1),     # three waves: 3*3/12 = 0.75, raised to t_min
    (9, 48, 3, 148, 5),    # 9*(1/4 + 3/12) = 4.5
    (2**32 - 1, 64, 4096, 1, (2**32 - 1)),  # 4096 waves of 1/4096 each
])
def test_exec_time_hand_values(load, k, m, M, want):
    assert oracle.exec_time(load, k, m, M) == want


def test_exec_time_against_amdahl_rationals():
    rng = np.random.default_rng(5)
    for _ in range(4000):
        M = int(rng.integers(1, 300))
        m = int(rng.integers(1, 4 * M + 1))
        load = int(rng.integers(1, 10**6))
        k = int(rng.integers(0, 65))
        assert oracle.exec_time(load, k, m, M) == amdahl_time(load, k, m, M)
    # extreme magnitudes
    for load in (1, 2**31, 2**32 - 1):
        for m in (1, 3, 255, 4096):
            for M in (1, 148, 4096):
                for k in (0, 19, 64):
                    assert oracle.exec_time(load, k, m, M) == amdahl_time(load, k, m, M)


def test_exec_time_full_fraction_is_eq1():
    """k = 64 (f = 1) reduces to Eq.1 itself: max(t_min, ceil(m/M) * C^/m), rounded up."""
    from fractions import Fraction
    import math
    for load in range(1, 40):
        for M in (1, 3, 6, 8):
            for m in range(1, 3 * M + 2):
                eq1 = max(1, math.ceil(math.ceil(Fraction(m, M)) * Fraction(load, m)))
                assert oracle.exec_time(load, 64, m, M) == eq1


# ----------------------------------------------------------- closed forms

def test_single_sm_bound_is_total_load():
    """M = 1: every group is one node on one SM, so R(G) = sum of C^ (any fraction)."""
    rng = np.random.default_rng(11)
    for _ in range(60):
        V = int(rng.integers(1, 25))
        rp, col, w, k = random_small_dag(rng, V, 0.3, 50)
        for var in range(4):
            rc, r = oracle.schedule(rp, col, w, k, 1, var)
            assert rc == 0 and r["bound"] == int(w.sum())


def test_chain_bound_is_greedy_sum():
    """A chain has no join and one local path: groups are single nodes with
    m = min(C^, M), and R(G) is the Greedy sequential sum."""
    rng = np.random.default_rng(12)
    for _ in range(60):
        V = int(rng.integers(1, 30))
        M = int(rng.integers(1, 200))
        rp, col = wl.csr_from_edges(V, list(range(V - 1)), list(range(1, V)))
        w = rng.integers(1, 500, size=V)
        k = rng.integers(0, 65, size=V).astype(np.uint8)
        rc, r = oracle.schedule(rp, col, w, k, M)
        want = sum(amdahl_time(int(w[i]), int(k[i]), min(int(w[i]), M), M) for i in range(V))
        assert rc == 0 and r["bound"] == want
        assert r["n_groups"] == V and r["n_seg"] == 0


def test_abundant_sms_bound_is_hop_depth():
    """M >= sum C^ with f = 1: every node gets m = C^ and C = 1, every released node
    fits as a parallel node, so the groups run the DAG level by level and R(G) is the
    number of nodes on the longest path. Without parallel launches R(G) = |Pi|."""
    rng = np.random.default_rng(13)
    for _ in range(80):
        V = int(rng.integers(1, 30))
        rp, col, w, _ = random_small_dag(rng, V, float(rng.uniform(0.05, 0.5)), 20)
        k = np.full(V, 64, np.uint8)
        M = int(w.sum()) + int(rng.integers(0, 10))
        rc, r = oracle.schedule(rp, col, w, k, M)
        assert rc == 0 and r["bound"] == 1 + max(hop_levels(rp, col))
        rc, r1 = oracle.schedule(rp, col, w, k, M, oracle.VAR_NOPARA)
        assert rc == 0 and r1["bound"] == r1["n_groups"]


def test_fork_join_closed_form():
    """s -> n equal children (load c < M) -> t: Pi = <{s}, children, {t}>, children get
    round(M/n) SMs (one fewer for the children trimmed to keep the sum <= M)."""
    import math
    for M in (4, 6, 8, 13, 32, 148):
        for n in range(1, min(M, 12) + 1):
            for c in (1, 2, 3, 5, M - 1):
                if c < 1 or c >= M:
                    continue
                for cs, ct in ((1, 1), (3, 7), (M + 5, 2 * M)):
                    V = n + 2
                    src = [0] * n + list(range(1, n + 1))
                    dst = list(range(1, n + 1)) + [n + 1] * n
                    rp, col = wl.csr_from_edges(V, src, dst)
                    w = np.array([cs] + [c] * n + [ct], np.int64)
                    k = np.full(V, 64, np.uint8)
                    rc, r = oracle.schedule(rp, col, w, k, M)
                    assert rc == 0
                    q = min(c, (2 * M + n) // (2 * n))  # round half up of M/n, capped at c
                    q = max(q, 1)
                    if n * q > M:
                        q -= 1  # at least one child is trimmed to q - 1
                    Cx = lambda x: math.ceil(x / min(x, M))
                    want = Cx(cs) + math.ceil(c / q) + Cx(ct)
                    assert r["bound"] == want, (M, n, c, cs, ct)
                    assert _groups_of(r) == [[0], list(range(1, n + 1)), [n + 1]]


# ------------------------------------------------- brute-force structure pins

def _check_structure(rp, col, w, k, M, var, r):
    V = len(w)
    succ = succ_lists(rp, col)
    anc = ancestors_by_search(rp, col)
    # Kahn levels and Eq.2 from plain graph search
    assert list(r["level"]) == hop_levels(rp, col)
    assert [int(x) for x in r["wanc"]] == [int(w[v]) + sum(int(w[u]) for u in anc[v]) for v in range(V)]
    W = r["wanc"]
    # Theta: join nodes, ascending W^anc, ties by id
    indeg = [0] * V
    for ss in succ:
        for s in ss:
            indeg[s] += 1
    joins = sorted((v for v in range(V) if indeg[v] >= 2), key=lambda v: (int(W[v]), v))
    assert list(r["theta"]) == joins
    # Eq.3 blocks
    assigned = [-1] * V
    for kk, th in enumerate(joins):
        for u in anc[th]:
            if assigned[u] < 0:
                assigned[u] = kk
    assigned = [len(joins) if b < 0 else b for b in assigned]
    assert list(r["block_of"]) == assigned
    # each block is an out-forest
    for v in range(V):
        inb = [u for u in range(V) if v in succ[u] and assigned[u] == assigned[v]]
        assert len(inb) <= 1
    # groups partition V, respect precedence, hold concurrent nodes, obey Rules 1-2,
    # and follow the block order
    groups = _groups_of(r)
    assert sorted(sum(groups, [])) == list(range(V))
    for u in range(V):
        for s in succ[u]:
            assert r["group_of"][u] < r["group_of"][s]
    last_block = -1
    for grp in groups:
        assert 1 <= len(grp) <= M
        if len(grp) > 1:
            assert all(w[v] < M for v in grp)
        for a in grp:
            for b in grp:
                assert a == b or (a not in anc[b] and b not in anc[a])
        bl = {assigned[v] for v in grp}
        assert len(bl) == 1
        assert min(bl) >= last_block
        last_block = min(bl)
    # plan rows: every node's final part and every segment, loads add up to C^
    nr = r["n_rows"]
    tot = {}
    for i in range(nr):
        rid = int(r["row_id"][i])
        owner = int(r["seg_parent"][rid - V]) if rid >= V else rid
        tot[owner] = tot.get(owner, 0) + int(r["row_load"][i])
    assert tot == {v: int(w[v]) for v in range(V)}
    assert all(r["row_group"][i] <= r["row_group"][i + 1] for i in range(nr - 1))
    # per executed group: SMs fit (except the literal variant), launched parts finish
    # within R, R is the largest member time, and the bound is the sum of R
    gR = r["group_R"]
    total = 0
    for j in range(r["n_groups"]):
        rows = [i for i in range(nr) if r["row_group"][i] == j]
        if not rows:
            assert gR[j] == 0
            continue
        times = [amdahl_time(int(r["row_load"][i]), int(r["row_k"][i]), int(r["row_m0"][i]), M)
                 for i in range(nr) if r["row_group"][i] == j]
        is_member = [r["row_id"][i] < V and r["group_of"][r["row_id"][i]] == j for i in rows]
        assert any(is_member)
        assert gR[j] == max(t for t, mb in zip(times, is_member) if mb)
        if var != oracle.VAR_LITERAL:
            assert sum(int(r["row_m0"][i]) for i in rows) <= M
            assert max(times) == gR[j]
        total += int(gR[j])
    assert r["bound"] == total
    # execution order: every original edge runs forward in groups; a para node ran
    # only after all its predecessors finished
    eg = r["exec_group"]
    for u in range(V):
        for s in succ[u]:
            assert eg[u] < eg[s]
        seg_groups = [int(r["seg_group"][x]) for x in range(r["n_seg"]) if r["seg_parent"][x] == u]
        for sg in seg_groups:
            assert sg < eg[u]
            assert all(eg[p] < sg for p in anc[u] if u in succ[p])
    # Theorem 1 lower bounds: bound >= critical path of G' with weights C, >= work / M
    n_exp = V + r["n_seg"]
    weight = [0] * n_exp
    for i in range(nr):
        weight[int(r["row_id"][i])] = amdahl_time(int(r["row_load"][i]), int(r["row_k"][i]),
                                                  int(r["row_m0"][i]), M)
    edges = [(u, s) for u in range(V) for s in succ[u]]
    preds = [[u for u in range(V) if v in succ[u]] for v in range(V)]
    for x in range(r["n_seg"]):
        par = int(r["seg_parent"][x])
        edges.append((V + x, par))
        edges += [(p, V + x) for p in preds[par]]
    edges += [tuple(map(int, e)) for e in r["extra"]]
    if var != oracle.VAR_LITERAL:
        assert r["bound"] >= longest_weighted_path(n_exp, edges, weight)
    assert r["bound"] >= -(-int(w.sum()) // M)
    # the candidate bound with the scheduled allocation equals the paper bound
    if var != oracle.VAR_LITERAL:
        assert oracle.bound_plan(r, M) == r["bound"]


@pytest.mark.parametrize("var", [0, 1, 2, 3])
def test_structure_on_random_small_dags(var):
    rng = np.random.default_rng(100 + var)
    for it in range(150):
        V = int(rng.integers(1, 22))
        M = int(rng.choice([1, 2, 3, 4, 6, 8, 16, 148]))
        rp, col, w, k = random_small_dag(rng, V, float(rng.uniform(0.05, 0.6)),
                                         int(rng.choice([3, 20, 200])))
        rc, r = oracle.schedule(rp, col, w, k, M, var)
        assert rc == 0
        _check_structure(rp, col, w, k, M, var, r)


def test_bound_monotone_in_load_for_fixed_structure():
    """For a fixed schedule structure and allocation, raising any row's load never
    lowers the bound (Eq.1 is non-decreasing in C^; max and sum are monotone)."""
    rng = np.random.default_rng(21)
    for _ in range(100):
        V = int(rng.integers(2, 20))
        M = int(rng.choice([4, 8, 148]))
        rp, col, w, k = random_small_dag(rng, V, 0.3, 100)
        rc, r = oracle.schedule(rp, col, w, k, M)
        alloc = rng.choice([0, 1, 2, 4, 8], size=r["n_rows"]).astype(np.uint8)
        b0 = oracle.bound_plan(r, M, alloc)
        i = int(rng.integers(0, r["n_rows"]))
        r2 = dict(r)
        r2["row_load"] = r["row_load"].copy()
        r2["row_load"][i] += int(rng.integers(1, 50))
        assert oracle.bound_plan(r2, M, alloc) >= b0


# --------------------------------------------- gang-scheduling brute force

def _simulate_barrier(r, M, durations):
    """Discrete-event run of the schedule with group barriers: the parts of group j
    start together when group j-1 has finished and each holds its SMs until it ends."""
    t = 0
    nr = r["n_rows"]
    for j in range(r["n_groups"]):
        rows = [i for i in range(nr) if r["row_group"][i] == j]
        if not rows:
            continue
        assert sum(int(r["row_m0"][i]) for i in rows) <= M
        t += max(durations[i] for i in rows)
    return t


def test_sustainability_by_enumerating_early_completion():
    """Sustainability: actual times anywhere in [1, C_i] never push the makespan of the
    scheduled DAG past R(G). All combinations are enumerated on DAGs of <= 8 nodes."""
    import itertools
    rng = np.random.default_rng(31)
    for _ in range(40):
        V = int(rng.integers(1, 9))
        M = int(rng.choice([2, 3, 4, 6]))
        rp, col, w, k = random_small_dag(rng, V, 0.4, 8)
        rc, r = oracle.schedule(rp, col, w, k, M)
        C = [amdahl_time(int(r["row_load"][i]), int(r["row_k"][i]), int(r["row_m0"][i]), M)
             for i in range(r["n_rows"])]
        choices = [sorted({1, c}) if c > 3 else list(range(1, c + 1)) for c in C]
        n = 0
        for durs in itertools.product(*choices):
            assert _simulate_barrier(r, M, durs) <= r["bound"]
            n += 1
            if n > 20000:
                break


def test_exhaustive_allocation_search_lower_than_paper():
    """On tiny DAGs the best allocation over all of L^rows (L = {1,2,4}) plus the
    scheduled one, for the paper's structure, is <= the paper's bound, and every
    candidate bound is >= the critical-path and work lower bounds."""
    import itertools
    rng = np.random.default_rng(41)
    for _ in range(25):
        V = int(rng.integers(1, 6))
        M = int(rng.choice([2, 4, 8]))
        rp, col, w, k = random_small_dag(rng, V, 0.4, 12)
        rc, r = oracle.schedule(rp, col, w, k, M)
        best = r["bound"]
        for combo in itertools.product([0, 1, 2, 4], repeat=r["n_rows"]):
            b = oracle.bound_plan(r, M, np.array(combo, np.uint8))
            best = min(best, b)
            assert b >= -(-int(w.sum()) // M)
        assert best <= r["bound"]


# --------------------------------------------------------------- validation

def test_validation_error_codes():
    rp, col = wl.csr_from_edges(3, [0, 1], [1, 2])
    w = np.array([1, 2, 3]); k = np.array([64, 64, 64], np.uint8)
    assert oracle.schedule(rp, col, w, k, 4)[0] == oracle.OK
    assert oracle.schedule(rp, col, w, k, 0)[0] == oracle.E_INVAL
    assert oracle.schedule(rp, col, w, k, 4097)[0] == oracle.E_INVAL
    assert oracle.schedule(rp, col, np.array([0, 2, 3]), k, 4)[0] == oracle.E_INVAL
    assert oracle.schedule(rp, col, np.array([1, 2, 2**32]), k, 4)[0] == oracle.E_INVAL
    assert oracle.schedule(rp, col, w, np.array([64, 65, 0], np.uint8), 4)[0] == oracle.E_INVAL
    assert oracle.schedule(rp, np.array([1, 3], np.int32), w, k, 4)[0] == oracle.E_RANGE
    assert oracle.schedule(rp, np.array([0, 2], np.int32), w, k, 4)[0] == oracle.E_RANGE  # self loop
    rp2 = np.array([0, 2, 2, 2], np.int32)
    assert oracle.schedule(rp2, np.array([2, 1], np.int32), w, k, 4)[0] == oracle.E_RANGE  # unsorted
    assert oracle.schedule(rp2, np.array([1, 1], np.int32), w, k, 4)[0] == oracle.E_RANGE  # duplicate
    rp3 = np.array([0, 1, 2, 3], np.int32)
    assert oracle.schedule(rp3, np.array([1, 2, 0], np.int32), w, k, 4)[0] == oracle.E_CYCLE
    assert oracle.schedule(np.array([0, 1, 1, 2], np.int32), np.array([1, 1], np.int32),
                           w, k, 4)[0] == oracle.OK
    assert oracle.schedule(np.array([0, 2, 1, 2], np.int32), np.array([1, 2], np.int32),
                           w, k, 4)[0] == oracle.E_INVAL  # row_ptr decreases
    # empty DAG
    rc, r = oracle.schedule(np.array([0], np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64),
                            np.zeros(0, np.uint8), 4)
    assert rc == oracle.OK and r["bound"] == 0 and r["n_groups"] == 0


# ------------------------------------------------------- candidate generator

def test_splitmix64_published_outputs():
    """SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) seeded with 0 yields
    0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F as its first outputs; the
    generator advances the state by the golden gamma before mixing."""
    g = 0x9E3779B97F4A7C15
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(g) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64(2 * g) == 0x06C45D188009454F


def test_generated_levels_are_uniform_and_keep_candidate_zero():
    levels = [1, 2, 4, 8, 16, 32]
    counts = np.zeros(len(levels), int)
    for c in range(1, 200):
        a = oracle.generated_allocation(7, 3, c, 50, levels, 200)
        for x in a:
            counts[levels.index(int(x))] += 1
    assert counts.min() > 0.9 * counts.mean() and counts.max() < 1.1 * counts.mean()
    assert not oracle.generated_allocation(7, 3, 0, 50, levels, 200).any()
    assert not oracle.generated_allocation(7, 3, 400, 50, levels, 200).any()
