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
        for var in range(5):
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


# ------------------------------------------------------ Top_M and Rule 2 (Alg.1)

def _eq5_nopara_bound(groups, w, k, M):
    """Sum over groups of max C_i with Eq.5's SMs, written out from Eq.5 in exact
    rationals: m_i = min(C^_i, max(1, round-half-up(C^_i M / W))), then the largest m
    (ties: higher id) trimmed until the group fits in M SMs."""
    from fractions import Fraction
    import math
    total = 0
    for grp in groups:
        W = sum(int(w[v]) for v in grp)
        m = {v: min(int(w[v]), max(1, math.floor(Fraction(int(w[v]) * M, W) + Fraction(1, 2)))) for v in grp}
        while sum(m.values()) > M:
            top = max(grp, key=lambda v: (m[v], v))
            m[top] -= 1
        total += max(amdahl_time(int(w[v]), int(k[v]), m[v], M) for v in grp)
    return total


def test_top_m_isolated_nodes_closed_form():
    """V isolated nodes: one residual block whose every node is a one-node path, so each
    round's heads are all remaining nodes and W^anc = C^. Alg.1 then cuts the nodes, in
    descending C^ order (ties: lower id), into groups: every node with C^ >= M alone
    (Rule 2), then chunks of M (Top_M, Rule 1). Without parallel launches the bound is the
    sum of the groups' largest Eq.5 times."""
    rng = np.random.default_rng(71)
    for _ in range(60):
        V = int(rng.integers(2, 40))
        M = int(rng.integers(2, 12))
        w = rng.integers(1, 2 * M + 3, size=V).astype(np.int64)
        k = rng.integers(0, 65, size=V).astype(np.uint8)
        rp = np.zeros(V + 1, np.int32)
        col = np.zeros(0, np.int32)
        order = sorted(range(V), key=lambda v: (-int(w[v]), v))
        big = [v for v in order if w[v] >= M]
        rest = [v for v in order if w[v] < M]
        want = [[v] for v in big] + [rest[i:i + M] for i in range(0, len(rest), M)]
        rc, r = oracle.schedule(rp, col, w, k, M, oracle.VAR_NOPARA)
        assert rc == 0
        assert _groups_of(r) == [sorted(g) for g in want]
        assert r["bound"] == _eq5_nopara_bound(want, w, k, M)


def test_top_m_follows_ancestor_weight_not_load():
    """Disjoint two-node chains a_i -> b_i, more chains than M: a round's heads are the
    unpicked a's (W^anc = C^(a)) and the b's whose a was picked (W^anc = C^(a) + C^(b)), so
    the M heads with the largest W^anc differ from the M largest loads. The expected groups
    follow from peeling the chains head by head by W^anc (Rule 2 when a picked head has
    C^ >= M)."""
    rng = np.random.default_rng(72)
    differs = 0
    for _ in range(60):
        n = int(rng.integers(3, 9))
        M = int(rng.integers(2, n))
        V = 2 * n
        src, dst = list(range(n)), list(range(n, 2 * n))  # a_i = i, b_i = n + i
        rp, col = wl.csr_from_edges(V, src, dst)
        w = rng.integers(1, M + 3, size=V).astype(np.int64)
        k = np.full(V, 64, np.uint8)
        W = {v: int(w[v]) for v in range(n)}
        W.update({n + i: int(w[i] + w[n + i]) for i in range(n)})
        pos = [0] * n  # next node of chain i: 0 -> a_i, 1 -> b_i, 2 -> done
        want = []
        while any(p < 2 for p in pos):
            heads = [i if pos[i] == 0 else n + i for i in range(n) if pos[i] < 2]
            heads.sort(key=lambda v: (-W[v], v))
            top = heads[:M]
            bigs = [v for v in top if w[v] >= M]
            grp = [max(bigs, key=lambda v: (int(w[v]), -top.index(v)))] if bigs else top
            want.append(sorted(grp))
            for v in grp:
                pos[v % n] += 1
        rc, r = oracle.schedule(rp, col, w, k, M, oracle.VAR_NOPARA)
        assert rc == 0 and _groups_of(r) == want, (M, list(w))
        # the same peeling by load alone (C^ instead of W^anc) picks other groups here
        pos = [0] * n
        by_load = []
        while any(p < 2 for p in pos):
            heads = [i if pos[i] == 0 else n + i for i in range(n) if pos[i] < 2]
            heads.sort(key=lambda v: (-int(w[v]), v))
            top = heads[:M]
            bigs = [v for v in top if w[v] >= M]
            grp = [max(bigs, key=lambda v: (int(w[v]), -top.index(v)))] if bigs else top
            by_load.append(sorted(grp))
            for v in grp:
                pos[v % n] += 1
        differs += by_load != want
    assert differs >= 10


# ------------------------------------------- parallel launches and segmentation (Alg.2)

def test_parallel_launch_order_split_and_extra_edges():
    """x, y -> J and three isolated nodes p, q, r (ids 3, 4, 5) of distinct loads. pi_1 =
    {x, y} leaves S SMs for R(pi_1); p, q, r are released (residual block) and are taken in
    descending W^anc (= load) order, which is neither id order nor its reverse: each is
    launched whole on min(load, S) SMs while it finishes within R, S shrinking by its SMs;
    the first that does not fit is split into the largest load that finishes within R on
    min(load, S) SMs, and the loop stops. Extra edges: every launched part -> succ(v_R),
    v_R -> every released node not launched whole. All expected values are derived here
    from those rules by brute force over the segment size."""
    M = 12
    for (cp, cq, cr, kx, kk) in ((4, 5, 3, 64, 64), (4, 5, 3, 64, 40), (6, 9, 2, 0, 64), (5, 7, 6, 32, 50)):
        # x = 0, y = 1, J = 2, p = 3, q = 4, r = 5
        rp, col = wl.csr_from_edges(6, [0, 1], [2, 2])
        w = np.array([2, 2, 4, cp, cq, cr], np.int64)
        k = np.array([kx, kx, 64, kk, kk, kk], np.uint8)
        rc, r = oracle.schedule(rp, col, w, k, M, oracle.VAR_PAPER)
        assert rc == 0
        assert _groups_of(r)[0] == [0, 1]
        # pi_1 = {x, y}: Eq.5 gives each min(2, round(2 * 12 / 4)) = 2 SMs
        R = max(amdahl_time(2, kx, 2, M), amdahl_time(2, kx, 2, M))
        S = M - 4
        order = sorted([3, 4, 5], key=lambda v: (-int(w[v]), v))
        launched, split = [], None
        for u in order:
            if S == 0:
                break
            mu = min(int(w[u]), S)
            if amdahl_time(int(w[u]), int(k[u]), mu, M) <= R:
                launched.append((u, mu))
                S -= mu
                continue
            x = max(x for x in range(1, int(w[u])) if amdahl_time(x, int(k[u]), min(x, S), M) <= R)
            split = (u, x, min(x, S))
            break
        rows0 = [(int(r["row_id"][i]), int(r["row_load"][i]), int(r["row_m0"][i]))
                 for i in range(r["n_rows"]) if r["row_group"][i] == 0]
        want_rows = [(0, 2, 2), (1, 2, 2)] + [(u, int(w[u]), mu) for u, mu in launched]
        if split:
            want_rows.append((6, split[1], split[2]))  # segment id = V + 0
        assert rows0 == want_rows, (rows0, want_rows)
        assert r["group_R"][0] == R
        if split:
            assert list(r["seg_parent"]) == [split[0]] and list(r["seg_load"]) == [split[1]]
        else:
            assert r["n_seg"] == 0
        vR = 0  # x and y tie on C: the lower id
        parts = [u for u, _ in launched] + ([6] if split else [])
        want_e = [(p_, 2) for p_ in parts]  # succ(v_R) = {J}
        whole = {u for u, _ in launched}
        want_e += [(vR, u) for u in order if u not in whole]
        assert [tuple(e) for e in r["extra"].tolist()] == want_e


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
        sms = sum(int(r["row_m0"][i]) for i in rows)
        if var == oracle.VAR_NOREPAIR and sms > M:
            # Eq.5 left unrepaired over-fills the group: no launches, members in sequence
            assert all(is_member) and gR[j] == sum(times)
        else:
            assert gR[j] == max(t for t, mb in zip(times, is_member) if mb)
        if var not in (oracle.VAR_LITERAL, oracle.VAR_NOREPAIR):
            assert sms <= M
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
    if var != oracle.VAR_LITERAL:  # (unrepaired groups run in sequence: still >= any path)
        assert r["bound"] >= longest_weighted_path(n_exp, edges, weight)
    assert r["bound"] >= -(-int(w.sum()) // M)
    # the candidate bound with the scheduled allocation equals the paper bound
    if var != oracle.VAR_LITERAL:
        assert oracle.bound_plan(r, M) == r["bound"]


@pytest.mark.parametrize("var", [0, 1, 2, 3, 4])
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


def test_critical_path_lower_bound():
    """The schedule's critical-path lower bound (oracle.crit_path) against a longest-path DP
    over the expanded graph (every part a node; a node's parts chained in plan order, i.e.
    by group; an edge of G from the tail's last part to every part of the head) and the work
    bound,
    computed here; it never exceeds R(G) except under the literal Alg.2; on a chain and at
    M = 1 it equals R(G)."""
    rng = np.random.default_rng(47)
    for _ in range(120):
        V = int(rng.integers(1, 20))
        M = int(rng.choice([1, 2, 4, 8, 148]))
        rp, col, w, k = random_small_dag(rng, V, 0.3, 60)
        succ = succ_lists(rp, col)
        for var in range(5):
            rc, r = oracle.schedule(rp, col, w, k, M, var, extra_cap=0)
            n = r["n_rows"]
            rid = [int(x) for x in r["row_id"][:n]]
            own = [x if x < V else int(r["seg_parent"][x - V]) for x in rid]
            wt = [amdahl_time(int(r["row_load"][i]), int(r["row_k"][i]), int(r["row_m0"][i]), M) for i in range(n)]
            last = {x: i for i, x in enumerate(rid) if x < V}
            # a node's parts one after another, in plan order (their groups increase)
            edges = []
            for v in range(V):
                mine = [i for i in range(n) if own[i] == v]
                edges += list(zip(mine, mine[1:]))
            edges += [(last[u], i) for u in range(V) for s in succ[u] for i in range(n) if own[i] == s]
            want = max(longest_weighted_path(n, edges, wt),
                       -(-sum(int(r["row_m0"][i]) * wt[i] for i in range(n)) // M))
            got = oracle.crit_path(r, rp, col, M)
            assert got == want
            if var != oracle.VAR_LITERAL:
                assert got <= r["bound"]
            if M == 1:
                assert got == r["bound"]
    for _ in range(20):
        V = int(rng.integers(1, 12))
        rp, col = wl.csr_from_edges(V, list(range(V - 1)), list(range(1, V)))
        w = rng.integers(1, 90, size=V)
        k = rng.integers(0, 65, size=V).astype(np.uint8)
        rc, r = oracle.schedule(rp, col, w, k, 7)
        assert oracle.crit_path(r, rp, col, 7) == r["bound"]


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

def test_gang_simulator_closed_forms():
    """The simulator against hand-worked executions: SM capacity serialises two
    full-GPU parts; a chain adds up; three 2-SM parts on 4 SMs have worst order 4 (start
    the two short ones, then the long one waits) and best 3."""
    from tests.gang_sim import worst_makespan
    M = 4
    two = [(0, 1, 64, 4, 0), (1, 1, 64, 4, 0)]
    assert worst_makespan(two, [set(), set()], M, "edges", durations=[[2], [3]])[0] == 5
    chain = [(i, 1, 64, 1, i) for i in range(4)]
    pred = [set(), {0}, {1}, {2}]
    assert worst_makespan(chain, pred, M, "edges", durations=[[1], [2], [3], [1]])[0] == 7
    three = [(i, 1, 64, 2, 0) for i in range(3)]
    w, nb = worst_makespan(three, [set(), set(), set()], M, "edges", durations=[[1], [2], [3]])
    assert (w, nb) == (4, 3)  # three maximal first pairs, worst 4
    # barrier mode: group 1 waits for all of group 0 even without edges
    g = [(0, 1, 64, 1, 0), (1, 1, 64, 1, 0), (2, 1, 64, 1, 1)]
    assert worst_makespan(g, [set(), set(), set()], M, "barrier", durations=[[1], [5], [2]])[0] == 7
    assert worst_makespan(g, [set(), set(), set()], M, "edges", durations=[[1], [5], [2]])[0] == 5


def _sim_cases(seed, n):
    from tests.gang_sim import add_extra_edges, parts_of
    rng = np.random.default_rng(seed)
    for _ in range(n):
        V = int(rng.integers(1, 9))
        M = int(rng.choice([2, 3, 4, 6, 8]))
        rp, col, w, k = random_small_dag(rng, V, 0.4, 8)
        succ = succ_lists(rp, col)
        for var in range(5):
            rc, r = oracle.schedule(rp, col, w, k, M, var)
            assert rc == 0
            parts, preds, last = parts_of(r, succ, V)
            add_extra_edges(r, parts, preds, last, V)
            yield var, M, r, parts, preds


def test_sustainability_every_execution_within_bound():
    """Theorem 1 and its sustainability remark, by brute force on DAGs of <= 8 nodes: under
    group-by-group execution, every work-conserving start order and every actual execution
    time in [1, C_i] finishes within R(G); with every part at its full C_i the worst case
    equals R(G) (the groups' SMs fit, so each group takes its largest C). Variants 0-2.
    The literal variant (S_j fixed, WS_j reduced by loads) breaks it in two ways, and only
    in these: a group may be given more SMs than the GPU has, and a parallel node whose
    load fits WS_j may still run longer than R(pi_j) when part of it is serial (WS_j counts
    load, not time) -- the reasons the library's default reads Eq.6 as SMs still free and
    tests a launch by its time."""
    from tests.gang_sim import exec_time, worst_makespan
    over_literal = {"sms": 0, "time": 0}
    for var, M, r, parts, preds in _sim_cases(31, 60):
        worst, _ = worst_makespan(parts, preds, M, "barrier")
        sums, too_long = {}, False
        for (_, load, k, m, g) in parts:
            sums[g] = sums.get(g, 0) + m
            too_long |= exec_time(load, k, m, M) > int(r["group_R"][g])
        if var == oracle.VAR_NOREPAIR and max(sums.values(), default=0) > M:
            assert worst <= r["bound"]  # an over-full group is bounded by its sum
        elif var != oracle.VAR_LITERAL:
            assert worst == r["bound"], (var, worst, r["bound"])
            assert max(sums.values(), default=0) <= M and not too_long
        elif worst > r["bound"]:
            assert max(sums.values()) > M or too_long
            over_literal["sms" if max(sums.values()) > M else "time"] += 1
    # the finding about the literal reading of Alg.2 (fixed sample): parallel nodes that
    # run longer than R(pi_j); the over-subscription case is built by hand below
    assert over_literal["time"] > 0, over_literal


def test_literal_alg2_can_oversubscribe_the_gpu():
    """x, y (serial, load 2) -> J, plus isolated p (load 3) and q (load 1), M = 6: pi_1 =
    {x, y} gets 2 + 2 SMs (Eq.5) and R = 2, so S = 2 and WS = 4. Read literally, Alg.2
    launches p on min(3, S) = 2 SMs (WS -> 1) and q on 1 SM (WS -> 0) without lowering S:
    7 SMs in a 6-SM group. q must wait for p, the group takes 3 ticks instead of 2 and the
    schedule exceeds its bound. With the remaining-SM reading (variant 0), q is split to
    fit, and the bound holds."""
    from tests.gang_sim import add_extra_edges, parts_of, worst_makespan
    rp, col = wl.csr_from_edges(5, [0, 1], [2, 2])  # x=0, y=1 -> J=2; p=3, q=4 isolated
    w = np.array([2, 2, 1, 3, 1], np.int64)
    k = np.array([0, 0, 64, 64, 64], np.uint8)
    M = 6
    succ = succ_lists(rp, col)
    rc, r = oracle.schedule(rp, col, w, k, M, oracle.VAR_LITERAL)
    assert rc == 0 and _groups_of(r)[0] == [0, 1]
    rows0 = [(int(r["row_id"][i]), int(r["row_m0"][i])) for i in range(r["n_rows"]) if r["row_group"][i] == 0]
    assert rows0 == [(0, 2), (1, 2), (3, 2), (4, 1)]  # members, then p and q, 7 SMs
    parts, preds, last = parts_of(r, succ, 5)
    add_extra_edges(r, parts, preds, last, 5)
    assert worst_makespan(parts, preds, M, "barrier")[0] == r["bound"] + 1
    rc, r0 = oracle.schedule(rp, col, w, k, M, oracle.VAR_PAPER)
    parts, preds, last = parts_of(r0, succ, 5)
    add_extra_edges(r0, parts, preds, last, 5)
    assert worst_makespan(parts, preds, M, "barrier")[0] == r0["bound"]


def test_extra_edges_alone_do_not_keep_the_bound():
    """Finding about the paper's claim that the extra dependencies alone run the groups in
    order: with only the DAG's edges, the segment order and Alg.2's extra edges (no group
    barriers), a work-conserving dispatcher can start a later group's part early, take SMs
    a member of the current group needs, and finish past R(G). Recorded on a fixed sample:
    the paper schedule exceeds its bound on 7 of 60 DAGs (by at most a few ticks), the
    variant without parallel launches (no extra edges at all) on 12."""
    from tests.gang_sim import worst_makespan
    over = {0: 0, 1: 0, 2: 0, 3: 0, 4: 0}
    for var, M, r, parts, preds in _sim_cases(31, 60):
        worst, _ = worst_makespan(parts, preds, M, "edges")
        over[var] += worst > r["bound"]
    assert over[0] == 7 and over[1] == 12


def test_exhaustive_search_enumerates_every_node_allocation():
    """The exhaustive search (base-B digits, one per node) evaluates exactly the
    allocations of ({schedule's m} + L)^V, each once: its bounds, as a multiset, equal
    those of an itertools enumeration of per-node choices; its optimum is <= the paper
    bound (allocation 0 is the schedule) and >= the work bound ceil(sum C^ / M)."""
    import itertools
    rng = np.random.default_rng(41)
    levels = [1, 2, 4]
    for _ in range(25):
        V = int(rng.integers(1, 7))
        M = int(rng.choice([2, 4, 8]))
        rp, col, w, k = random_small_dag(rng, V, 0.4, 12)
        for var in range(4):
            rc, r = oracle.schedule(rp, col, w, k, M, var)
            n_alloc = (len(levels) + 1) ** V
            got = oracle.exhaustive_plan(r, M, levels, n_alloc)
            own = oracle.row_owner(r)
            want = []
            for choice in itertools.product([0] + levels, repeat=V):
                alloc = np.array([choice[u] for u in own], np.uint8)
                want.append(oracle.bound_plan(r, M, alloc if r["n_rows"] else None))
            assert sorted(got.tolist()) == sorted(want)
            assert got[0] == oracle.bound_plan(r, M)
            if var != oracle.VAR_LITERAL:
                assert got[0] == r["bound"]
            assert got.min() >= -(-int(w.sum()) // M)


def test_exhaustive_search_on_a_chain_is_separable():
    """On a chain every group is one node, so the bound is a sum of per-node times and the
    exhaustive optimum is the sum over nodes of the best of the schedule's m and the
    levels -- computed here node by node from Eq.1."""
    rng = np.random.default_rng(43)
    levels = [1, 3, 8]
    for _ in range(30):
        V = int(rng.integers(1, 7))
        M = int(rng.integers(2, 12))
        rp, col = wl.csr_from_edges(V, list(range(V - 1)), list(range(1, V)))
        w = rng.integers(1, 40, size=V).astype(np.int64)
        k = rng.integers(0, 65, size=V).astype(np.uint8)
        rc, r = oracle.schedule(rp, col, w, k, M, oracle.VAR_PAPER)
        got = oracle.exhaustive_plan(r, M, levels, (len(levels) + 1) ** V).min()
        want = sum(min(amdahl_time(int(w[i]), int(k[i]), m, M) for m in [min(int(w[i]), M)] + levels)
                   for i in range(V))
        assert got == want


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
