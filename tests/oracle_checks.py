"""Independent brute-force helpers the tests use to pin the oracle.

Each helper recomputes a property from its textbook definition (reachability by
search, longest paths by dynamic programming, Amdahl's law with exact rationals),
without calling the oracle, so a mistake inside the oracle shows up as a mismatch.
"""
from __future__ import annotations

from fractions import Fraction
import math

import numpy as np


def succ_lists(row_ptr, col):
    V = len(row_ptr) - 1
    return [list(map(int, col[row_ptr[v]:row_ptr[v + 1]])) for v in range(V)]


def pred_lists(row_ptr, col):
    V = len(row_ptr) - 1
    pred = [[] for _ in range(V)]
    for u, ss in enumerate(succ_lists(row_ptr, col)):
        for s in ss:
            pred[s].append(u)
    return pred


def ancestors_by_search(row_ptr, col):
    """anc[v] = set of nodes with a path to v, by backward depth-first search."""
    pred = pred_lists(row_ptr, col)
    V = len(pred)
    out = []
    for v in range(V):
        seen, stack = set(), list(pred[v])
        while stack:
            u = stack.pop()
            if u not in seen:
                seen.add(u)
                stack.extend(pred[u])
        out.append(seen)
    return out


def hop_levels(row_ptr, col):
    """Longest number of edges on any path ending at v."""
    pred = pred_lists(row_ptr, col)
    V = len(pred)
    memo = [None] * V

    def lev(v):
        if memo[v] is None:
            memo[v] = 0 if not pred[v] else 1 + max(lev(p) for p in pred[v])
        return memo[v]

    import sys
    sys.setrecursionlimit(max(10000, 4 * V))
    return [lev(v) for v in range(V)]


def amdahl_time(load, k, m, M):
    """Eq.1 with t_min = 1 and an Amdahl parallel fraction f = k/64, computed with
    exact rationals: ceil(m/M) * load * ((1 - f) + f / m), rounded up, at least 1."""
    f = Fraction(k, 64)
    t = math.ceil(Fraction(m, M)) * load * ((1 - f) + f / m)
    return max(1, math.ceil(t))


def longest_weighted_path(n, edges, weight):
    """Max over paths of the sum of node weights, by DP over a topological order."""
    succ = [[] for _ in range(n)]
    indeg = [0] * n
    for a, b in edges:
        succ[a].append(b)
        indeg[b] += 1
    order = [v for v in range(n) if indeg[v] == 0]
    i = 0
    while i < len(order):
        for s in succ[order[i]]:
            indeg[s] -= 1
            if indeg[s] == 0:
                order.append(s)
        i += 1
    assert len(order) == n, "expanded graph has a cycle"
    best = [0] * n
    for v in order:
        best[v] += weight[v]
        for s in succ[v]:
            best[s] = max(best[s], best[v])
    return max(best) if n else 0


def random_small_dag(rng, V, p, wmax, kmin=0):
    from paper_2602_20826_gb300 import workloads as wl
    s, t = wl.er_edges(rng, V, p)
    rp, col = wl.csr_from_edges(V, s, t)
    w = rng.integers(1, wmax + 1, size=V).astype(np.int64)
    k = rng.integers(kmin, 65, size=V).astype(np.uint8)
    return rp, col, w, k
