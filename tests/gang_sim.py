"""Discrete-event gang simulator of a schedule: every execution the schedule allows.

Test infrastructure, independent of the oracle's arithmetic: it takes a schedule's plan rows
(the parts that run: each node's last part and each parallel segment, with load, parallel
fraction, SMs and group) and runs them on an M-SM GPU as gangs -- a part holds its m SMs
from its start to its end and starts only when that many SMs are free.

What the simulator enumerates:
  * actual execution times: each part runs for any integer time in [1, C], C its Eq.1 time
    (exhaustively when C <= 3, else the two extremes 1 and C);
  * start orders: whenever parts are ready, a work-conserving dispatcher starts a maximal
    set of them that fits into the free SMs -- every such set is one branch (these are the
    outcomes of every order in which a ready queue can be served).

Precedence: an original edge u -> v makes every part of v wait for u's last part; a node's
parallel segment runs before its residual part; the schedule's extra dependency edges are
respected; in "barrier" mode every part of group j also waits for every part of the groups
before it (the group-by-group execution the bound's proof assumes); in "edges" mode only the
edges order the parts.

It returns the largest makespan over every branch; Theorem 1 (with the sustainability of
the bound) says that in barrier mode no branch may exceed R(G).
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction


def exec_time(load, k, m, M):
    """Eq.1 with t_min = 1 and an Amdahl parallel fraction k/64, in exact rationals."""
    f = Fraction(int(k), 64)
    t = math.ceil(Fraction(int(m), int(M))) * int(load) * ((1 - f) + f / int(m))
    return max(1, math.ceil(t))


def parts_of(plan, succ, V):
    """Parts and their predecessor sets from an oracle schedule result.

    Returns (parts, preds): parts[i] = (row_id, load, k, m, group); preds[i] = set of part
    indices that must finish before part i starts (edges and segment order only)."""
    n = int(plan["n_rows"])
    parts = [(int(plan["row_id"][i]), int(plan["row_load"][i]), int(plan["row_k"][i]),
              int(plan["row_m0"][i]), int(plan["row_group"][i])) for i in range(n)]
    seg_parent = [int(x) for x in plan["seg_parent"]]
    owner = [pid if pid < V else seg_parent[pid - V] for pid, *_ in parts]
    last = {}  # node -> index of its last part (the row with row_id == node)
    for i, (pid, *_) in enumerate(parts):
        if pid < V:
            last[pid] = i
    pred_nodes = [[] for _ in range(V)]
    for u in range(V):
        for s in succ[u]:
            pred_nodes[s].append(u)
    preds = [set() for _ in range(n)]
    for i in range(n):
        v = owner[i]
        for u in pred_nodes[v]:
            preds[i].add(last[u])
        if parts[i][0] < V:  # a node's residual part waits for its segments
            for j in range(n):
                if parts[j][0] >= V and owner[j] == v:
                    preds[i].add(j)
    return parts, preds, last


def add_extra_edges(plan, parts, preds, last, V):
    """The schedule's extra dependencies (v_R, v_n) and (v_n, succ(v_R)) between parts:
    an id below V names the node's last part, an id >= V the segment's part."""
    by_id = {pid: i for i, (pid, *_) in enumerate(parts)}
    for a, b in plan["extra"]:
        a, b = int(a), int(b)
        ia = by_id[a] if a >= V else last[a]
        ib = by_id[b] if b >= V else last[b]
        preds[ib].add(ia)


def worst_makespan(parts, preds, M, mode="barrier", durations=None, limit=200000):
    """Largest makespan over every branch (start orders x execution times).

    durations: per part, the list of times to try (default: 1..C if C <= 3, else {1, C}).
    Returns (worst, n_branches). Raises if a part can never start (m > M)."""
    n = len(parts)
    C = [exec_time(load, k, m, M) for (_, load, k, m, _) in parts]
    if durations is None:
        durations = [list(range(1, c + 1)) if c <= 3 else [1, c] for c in C]
    for (_, _, _, m, _) in parts:
        if m > M:
            raise ValueError("a part needs more SMs than the GPU has")
    group = [g for (*_, g) in parts]
    worst = [0, 0]  # makespan, branches

    def ready(i, done):
        if not preds[i] <= done:
            return False
        if mode == "barrier":
            return all(j in done for j in range(n) if group[j] < group[i])
        return True

    def rec(t, running, done, started):
        # running: tuple of (end, part); done: frozenset; started: frozenset
        if worst[1] > limit:
            raise RuntimeError("too many branches")
        free = M - sum(parts[i][3] for _, i in running)
        cand = [i for i in range(n) if i not in started and ready(i, done)]
        # maximal subsets of the ready parts that fit into the free SMs
        sets = []
        for r in range(len(cand), 0, -1):
            for sub in itertools.combinations(cand, r):
                need = sum(parts[i][3] for i in sub)
                if need > free:
                    continue
                rest = free - need
                if any(parts[i][3] <= rest for i in cand if i not in sub):
                    continue  # not maximal: another ready part still fits
                sets.append(sub)
        if not sets:
            sets = [()]
        for sub in sets:
            if not sub and not running:
                if len(done) == n:
                    worst[0] = max(worst[0], t)
                    worst[1] += 1
                    return
                raise RuntimeError("deadlock: nothing runs and nothing can start")
            for ds in itertools.product(*[durations[i] for i in sub]):
                run2 = tuple(sorted(running + tuple((t + d, i) for d, i in zip(ds, sub))))
                st2 = started | frozenset(sub)
                # advance to the next completion
                t2 = run2[0][0]
                fin = frozenset(i for e, i in run2 if e == t2)
                rest = tuple((e, i) for e, i in run2 if e != t2)
                rec(t2, rest, done | fin, st2)

    rec(0, (), frozenset(), frozenset())
    return worst[0], worst[1]
