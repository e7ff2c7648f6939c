"""CPU oracle for conditional DAGs (test infrastructure only).

The paper leaves conditional DAGs to future work; the reading used here: a conditional node
takes exactly one of its out-edges per job. A node runs when it has no predecessor, or when
one of its in-edges is active; an edge is active when its tail runs and either is not
conditional or chose that edge. Each choice of one out-edge per conditional node gives a
realisation, a plain DAG (the running nodes renumbered in increasing order, the active
edges); the same realisation reached by several choices counts once, at its first choice in
mixed-radix order with the lowest-id conditional node varying fastest.

Bounds (Theorem 1 through the bound oracle): `adaptive` is the largest bound over the
realisations, each scheduled on its own; `fixed` is the bound of the whole DAG with every
branch present. Written with plain Python loops and a recursive reachability walk; nothing
is shared with the library's expansion.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import OK, schedule


def realisations(row_ptr, col, cond):
    """The distinct realisations of one conditional DAG, in enumeration order: a list of
    (nodes, edges), nodes the running original ids (ascending), edges the active (u, v)."""
    V = len(row_ptr) - 1
    succ = [[int(c) for c in col[row_ptr[u]:row_ptr[u + 1]]] for u in range(V)]
    has_pred = [False] * V
    for u in range(V):
        for v in succ[u]:
            has_pred[v] = True
    conds = [u for u in range(V) if cond[u] and succ[u]]
    out, seen = [], set()
    # mixed radix, the first conditional node fastest: itertools.product varies the last
    # position fastest, so enumerate the reversed tuple
    for rev in itertools.product(*[range(len(succ[c])) for c in reversed(conds)]):
        pick = dict(zip(reversed(conds), rev))
        running = set()

        def visit(u):
            if u in running:
                return
            running.add(u)
            for i, v in enumerate(succ[u]):
                if u not in pick or pick[u] == i:
                    visit(v)

        for u in range(V):
            if not has_pred[u]:
                visit(u)
        edges = sorted((u, v) for u in running for i, v in enumerate(succ[u])
                       if u not in pick or pick[u] == i)
        key = (tuple(sorted(running)), tuple(edges))
        if key not in seen:
            seen.add(key)
            out.append((sorted(running), edges))
    return out


def realisation_csr(nodes, edges):
    """Row pointers and successor ids of a realisation, nodes renumbered by their order."""
    idx = {u: i for i, u in enumerate(nodes)}
    rp = np.zeros(len(nodes) + 1, np.int32)
    cols = []
    for i, u in enumerate(nodes):
        succ = sorted(idx[v] for a, v in edges if a == u)
        cols += succ
        rp[i + 1] = rp[i] + len(succ)
    return rp, np.asarray(cols, np.int32)


def cond_bounds(row_ptr, col, wcet, k64, cond, M: int, variant: int = 0):
    """(adaptive, fixed, worst realisation index, number of realisations) of one DAG."""
    wcet = np.asarray(wcet, np.int64)
    k64 = np.asarray(k64, np.uint8)
    rc, whole = schedule(row_ptr, col, wcet, k64, M, variant, extra_cap=0)
    fixed = whole["bound"] if rc == OK else -1
    best, arg = -1, -1
    reals = realisations(row_ptr, col, cond)
    for i, (nodes, edges) in enumerate(reals):
        rp, cl = realisation_csr(nodes, edges)
        rc, r = schedule(rp, cl, wcet[nodes], k64[nodes], M, variant, extra_cap=0)
        if rc != OK:
            return -1, fixed, -1, len(reals)
        if r["bound"] > best:
            best, arg = r["bound"], i
    return best, fixed, arg, len(reals)
