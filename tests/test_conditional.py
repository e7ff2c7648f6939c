"""Conditional DAGs (the paper's future work, in the reading of oracle/conditional.py):
pins of the realisation oracle by hand-worked cases and by the gang simulator."""
from __future__ import annotations

import numpy as np

import oracle
from oracle import conditional as CD
from paper_2602_20826_gb300 import workloads as wl
from tests.oracle_checks import amdahl_time, random_small_dag, succ_lists


def test_no_conditional_node_is_one_realisation():
    rng = np.random.default_rng(61)
    for _ in range(30):
        V = int(rng.integers(1, 15))
        rp, col, w, k = random_small_dag(rng, V, 0.3, 30)
        reals = CD.realisations(rp, col, np.zeros(V, np.uint8))
        assert len(reals) == 1 and reals[0][0] == list(range(V))
        a, f, arg, n = CD.cond_bounds(rp, col, w, k, np.zeros(V, np.uint8), 6)
        assert a == f == oracle.schedule(rp, col, w, k, 6)[1]["bound"] and (arg, n) == (0, 1)


def test_diamond_branches_are_chains():
    """c -> a | b -> j with c conditional: the realisations are the chains c a j and c b j,
    whose bounds are Greedy sums (one node per group); adaptive is the larger one, fixed is
    the bound of the whole diamond."""
    rp, col = wl.csr_from_edges(4, [0, 0, 1, 2], [1, 2, 3, 3])  # c=0, a=1, b=2, j=3
    cond = np.array([1, 0, 0, 0], np.uint8)
    reals = CD.realisations(rp, col, cond)
    assert reals == [([0, 1, 3], [(0, 1), (1, 3)]), ([0, 2, 3], [(0, 2), (2, 3)])]
    for M in (2, 5, 16):
        w = np.array([3, 17, 9, 4], np.int64)
        k = np.array([64, 40, 64, 20], np.uint8)
        chain = lambda ids: sum(amdahl_time(int(w[i]), int(k[i]), min(int(w[i]), M), M) for i in ids)  # noqa: E731
        a, f, arg, n = CD.cond_bounds(rp, col, w, k, cond, M)
        want = [chain([0, 1, 3]), chain([0, 2, 3])]
        assert a == max(want) and arg == int(np.argmax(want)) and n == 2
        assert f == oracle.schedule(rp, col, w, k, M)[1]["bound"]


def test_nested_branches_count_each_realisation_once():
    """c1 -> x | c2, c2 -> y | z: choosing x leaves c2 out, so the two choices of c2 under x
    give one realisation; three in all, in the order (x), (c2, y), (c2, z)."""
    rp, col = wl.csr_from_edges(5, [0, 0, 2, 2], [1, 2, 3, 4])  # c1=0, x=1, c2=2, y=3, z=4
    cond = np.array([1, 0, 1, 0, 0], np.uint8)
    reals = CD.realisations(rp, col, cond)
    assert [r[0] for r in reals] == [[0, 1], [0, 2, 3], [0, 2, 4]]


def test_fixed_schedule_holds_for_every_realisation():
    """The whole DAG's schedule run on a realisation -- the parts of nodes that do not run
    take no time, the others anything in [1, C] -- never finishes after the fixed bound:
    every execution of the gang simulator under group barriers stays within it."""
    from tests.gang_sim import add_extra_edges, parts_of, worst_makespan
    rng = np.random.default_rng(62)
    checked = 0
    for _ in range(40):
        V = int(rng.integers(3, 8))
        rp, col, w, k = random_small_dag(rng, V, 0.4, 6)
        cond = (rng.random(V) < 0.4).astype(np.uint8)
        M = int(rng.choice([2, 4, 6]))
        rc, whole = oracle.schedule(rp, col, w, k, M)
        succ = succ_lists(rp, col)
        parts, preds, last = parts_of(whole, succ, V)
        add_extra_edges(whole, parts, preds, last, V)
        owner = [pid if pid < V else int(whole["seg_parent"][pid - V]) for pid, *_ in parts]
        for nodes, _ in CD.realisations(rp, col, cond):
            run = set(nodes)
            C = [max(1, -(-int(ld) * (64 * m - kk * (m - 1)) // (64 * m))) for _, ld, kk, m, _ in parts]
            durs = [([0] if owner[i] not in run else (list(range(1, c + 1)) if c <= 2 else [1, c]))
                    for i, c in enumerate(C)]
            wst, _ = worst_makespan(parts, preds, M, "barrier", durations=durs)
            assert wst <= whole["bound"]
            checked += 1
    assert checked > 40
