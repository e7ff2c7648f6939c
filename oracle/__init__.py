"""CPU oracle for the makespan bound (test infrastructure only).

The oracle is plain C (`oracle.c`), compiled with gcc into `liboracle.so` next to
this file and called through ctypes. Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this package; the library's product path
never does. It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, E_INVAL, E_CYCLE, E_RANGE, E_OOM, E_CAP = 0, -1, -2, -3, -4, -7
VAR_PAPER, VAR_NOPARA, VAR_NOSEG, VAR_LITERAL, VAR_NOREPAIR = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no CUDA involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_P32 = C.POINTER(C.c_int32)
_P64 = C.POINTER(C.c_int64)
_PU8 = C.POINTER(C.c_uint8)


class _Out(C.Structure):
    _fields_ = [("level", _P32), ("wanc", _P64), ("block_of", _P32), ("group_of", _P32),
                ("exec_group", _P32), ("m", _P32), ("theta", _P32), ("group_R", _P64),
                ("seg_parent", _P32), ("seg_load", _P64), ("seg_m", _P32), ("seg_group", _P32),
                ("row_id", _P32), ("row_load", _P64), ("row_k", _P32), ("row_m0", _P32),
                ("row_group", _P32), ("extra_src", _P32), ("extra_dst", _P32),
                ("extra_cap", C.c_int64), ("n_join", C.c_int32), ("n_groups", C.c_int32),
                ("n_seg", C.c_int32), ("n_rows", C.c_int32), ("n_extra", C.c_int64),
                ("bound", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.or_exec_time.restype = C.c_int64
        _lib.or_exec_time.argtypes = [C.c_int64] * 4
        _lib.or_validate.restype = C.c_int
        _lib.or_validate.argtypes = [C.c_int32, _P32, C.c_int64, _P32, _P64, _PU8, C.c_int32]
        _lib.or_schedule_dag.restype = C.c_int
        _lib.or_schedule_dag.argtypes = [C.c_int32, _P32, _P32, _P64, _PU8, C.c_int32, C.c_int32,
                                         C.POINTER(_Out)]
        _lib.or_bound_plan.restype = C.c_int64
        _lib.or_bound_plan.argtypes = [C.c_int32, _P64, _P32, _P32, _P32, C.c_int32, _PU8, C.c_int64]
        _lib.or_splitmix64.restype = C.c_uint64
        _lib.or_splitmix64.argtypes = [C.c_uint64]
        _lib.or_gen_level.restype = C.c_int32
        _lib.or_gen_level.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int64, C.c_int32]
        _lib.or_exhaustive_plan.restype = None
        _lib.or_exhaustive_plan.argtypes = [C.c_int32, _P64, _P32, _P32, _P32, _P32, C.c_int32, C.c_int32, _PU8,
                                            C.c_int64, _P64]
        _lib.or_baselines.restype = C.c_int
        _lib.or_baselines.argtypes = [C.c_int32, _P32, _P32, _P64, _PU8, C.c_int32, _P64]
        _lib.or_schedule_batch.restype = C.c_int64
        _lib.or_schedule_batch.argtypes = [C.c_int32, _P64, _P64, _P32, _P32, _P64, _PU8, C.c_int32,
                                           C.c_int32, _P64, _P32]
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t)


def exec_time(load: int, k: int, m: int, M: int) -> int:
    """Eq.1 (+ parallel fraction k/64), integer ticks."""
    return int(lib().or_exec_time(int(load), int(k), int(m), int(M)))


def schedule(row_ptr, col, wcet, k64, M: int, variant: int = VAR_PAPER, extra_cap: int = -1):
    """Alg.1 + Alg.2 + Theorem 1 on one DAG. Returns (status, dict of numpy arrays).
    extra_cap < 0 sizes the extra-edge buffer to hold every edge (two passes)."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    wcet = np.ascontiguousarray(wcet, np.int64)
    k64 = np.ascontiguousarray(k64, np.uint8)
    V = len(wcet)
    if len(col) == 0:
        col = np.zeros(1, np.int32)[:0]
    nv = max(V, 1)
    a = {
        "level": np.zeros(nv, np.int32), "wanc": np.zeros(nv, np.int64),
        "block_of": np.zeros(nv, np.int32), "group_of": np.zeros(nv, np.int32),
        "exec_group": np.zeros(nv, np.int32), "m": np.zeros(nv, np.int32),
        "theta": np.zeros(nv, np.int32), "group_R": np.zeros(nv, np.int64),
        "seg_parent": np.zeros(nv, np.int32), "seg_load": np.zeros(nv, np.int64),
        "seg_m": np.zeros(nv, np.int32), "seg_group": np.zeros(nv, np.int32),
        "row_id": np.zeros(2 * nv, np.int32), "row_load": np.zeros(2 * nv, np.int64),
        "row_k": np.zeros(2 * nv, np.int32), "row_m0": np.zeros(2 * nv, np.int32),
        "row_group": np.zeros(2 * nv, np.int32),
    }

    def run(cap):
        es = np.zeros(max(cap, 1), np.int32)
        ed = np.zeros(max(cap, 1), np.int32)
        o = _Out()
        for name, arr in a.items():
            setattr(o, name, _ptr(arr, _P64 if arr.dtype == np.int64 else _P32))
        o.extra_src = _ptr(es, _P32)
        o.extra_dst = _ptr(ed, _P32)
        o.extra_cap = cap
        rc = lib().or_schedule_dag(V, _ptr(row_ptr, _P32), _ptr(col, _P32), _ptr(wcet, _P64),
                                   _ptr(k64, _PU8), int(M), int(variant), C.byref(o))
        return rc, o, es, ed

    rc, o, es, ed = run(max(extra_cap, 0))
    if extra_cap < 0 and rc == OK and o.n_extra > 0:
        rc, o, es, ed = run(int(o.n_extra))
    res = {
        "V": V, "bound": int(o.bound), "n_join": int(o.n_join), "n_groups": int(o.n_groups),
        "n_seg": int(o.n_seg), "n_rows": int(o.n_rows), "n_extra": int(o.n_extra),
    }
    for name in ("level", "wanc", "block_of", "group_of", "exec_group", "m"):
        res[name] = a[name][:V].copy()
    res["theta"] = a["theta"][:o.n_join].copy()
    res["group_R"] = a["group_R"][:o.n_groups].copy()
    for name in ("seg_parent", "seg_load", "seg_m", "seg_group"):
        res[name] = a[name][:o.n_seg].copy()
    for name in ("row_id", "row_load", "row_k", "row_m0", "row_group"):
        res[name] = a[name][:o.n_rows].copy()
    ne = min(int(o.n_extra), len(es)) if (extra_cap != 0) else 0
    res["extra"] = np.stack([es[:ne], ed[:ne]], axis=1) if ne else np.zeros((0, 2), np.int32)
    return rc, res


def baselines(row_ptr, col, wcet, k64, M: int):
    """(status, greedy, greedy_unaware, graham_para): the Evaluation section's baseline
    bounds of one DAG (see or_baselines)."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int32)
    col = np.ascontiguousarray(col if len(col) else np.zeros(1, np.int32), np.int32)
    wcet = np.ascontiguousarray(wcet, np.int64)
    k64 = np.ascontiguousarray(k64, np.uint8)
    out = np.zeros(3, np.int64)
    rc = lib().or_baselines(len(wcet), _ptr(row_ptr, _P32), _ptr(col, _P32), _ptr(wcet, _P64), _ptr(k64, _PU8),
                            int(M), _ptr(out, _P64))
    return (int(rc), int(out[0]), int(out[1]), int(out[2])) if rc == OK else (int(rc), -1, -1, -1)


def crit_path(plan: dict, row_ptr, col, M: int) -> int:
    """Lower bound of every execution of a schedule: the longest chain of its parts along
    G's edges (a node's parts one after another; an edge waits for its tail's last part),
    each part weighted by its Eq.1 time, or the work bound ceil(sum m C / M) if larger."""
    V = int(plan["V"])
    own = row_owner(plan)
    T = [0] * V
    work = 0
    for r in range(int(plan["n_rows"])):
        c = exec_time(int(plan["row_load"][r]), int(plan["row_k"][r]), int(plan["row_m0"][r]), M)
        T[int(own[r])] += c
        work += int(plan["row_m0"][r]) * c
    indeg = [0] * V
    for e in range(int(row_ptr[V]) if V else 0):
        indeg[int(col[e])] += 1
    order = [v for v in range(V) if indeg[v] == 0]
    best = [0] * V
    i = 0
    while i < len(order):
        u = order[i]
        i += 1
        best[u] += T[u]
        for e in range(int(row_ptr[u]), int(row_ptr[u + 1])):
            s = int(col[e])
            best[s] = max(best[s], best[u])
            indeg[s] -= 1
            if indeg[s] == 0:
                order.append(s)
    path = max(best) if V else 0
    return max(path, -(-work // M))


def bound_plan(plan: dict, M: int, alloc=None, stride: int = 1) -> int:
    """Bound of one allocation (per plan row; 0 = keep the scheduled m) on a fixed
    schedule structure."""
    n = int(plan["n_rows"])
    load = np.ascontiguousarray(plan["row_load"], np.int64)
    k = np.ascontiguousarray(plan["row_k"], np.int32)
    m0 = np.ascontiguousarray(plan["row_m0"], np.int32)
    g = np.ascontiguousarray(plan["row_group"], np.int32)
    if n == 0:
        return 0
    ap = None
    if alloc is not None:
        alloc = np.ascontiguousarray(alloc, np.uint8)
        ap = _ptr(alloc, _PU8)
    return int(lib().or_bound_plan(n, _ptr(load, _P64), _ptr(k, _P32), _ptr(m0, _P32),
                                   _ptr(g, _P32), int(M), ap, int(stride)))


def schedule_batch(batch, variant: int = VAR_PAPER, dags=None):
    """Paper-schedule bound of every DAG (or of the listed DAGs): (bound, status)."""
    if dags is not None:
        batch = batch.subset(dags)
    n = batch.n_dags
    bound = np.zeros(n, np.int64)
    status = np.zeros(n, np.int32)
    col = batch.col if len(batch.col) else np.zeros(1, np.int32)
    lib().or_schedule_batch(n, _ptr(batch.node_off, _P64), _ptr(batch.edge_off, _P64),
                            _ptr(batch.row_ptr, _P32), _ptr(col, _P32), _ptr(batch.wcet, _P64),
                            _ptr(batch.k64, _PU8), int(batch.M), int(variant),
                            _ptr(bound, _P64), _ptr(status, _P32))
    return bound, status


def _at(a, off, t):
    """Pointer to element `off` of numpy array `a` (no copy)."""
    return C.cast(a.ctypes.data + int(off) * a.itemsize, t)


def schedule_range(batch, lo: int, hi: int, variant: int = VAR_PAPER):
    """Paper-schedule bound of DAGs lo..hi-1 of the batch, read in place (no copy, so that
    host threads can run disjoint ranges at once): (bound, status)."""
    n = hi - lo
    bound = np.zeros(max(n, 1), np.int64)
    status = np.zeros(max(n, 1), np.int32)
    col = batch.col if len(batch.col) else np.zeros(1, np.int32)
    # DAG lo + i reads row_ptr[node_off[lo + i] + lo + i]: shift the row_ptr base by lo
    lib().or_schedule_batch(n, _at(batch.node_off, lo, _P64), _at(batch.edge_off, lo, _P64),
                            _at(batch.row_ptr, lo, _P32), _ptr(col, _P32), _ptr(batch.wcet, _P64),
                            _ptr(batch.k64, _PU8), int(batch.M), int(variant), _ptr(bound, _P64),
                            _ptr(status, _P32))
    return bound[:n], status[:n]


def schedule_dag_of(batch, d: int, variant: int = VAR_PAPER, extra_cap: int = 0):
    rp, col, w, k = batch.dag(d)
    return schedule(rp, col, w, k, batch.M, variant, extra_cap)


def search_dag(batch, d: int, alloc, cand_stride: int, n_variants: int, n_alloc: int,
               variant_ids=None):
    """Bounds of every candidate of DAG d and the argmin (min bound, lowest id).
    alloc is the [2*node_off[d]+row][cand] uint8 buffer of the whole batch."""
    if variant_ids is None:
        variant_ids = list(range(n_variants))
    n0 = int(batch.node_off[d])
    plans = {}
    out = np.zeros(n_variants * n_alloc, np.int64)
    for vi in range(n_variants):
        var = int(variant_ids[vi])
        if var not in plans:
            rc, plans[var] = schedule_dag_of(batch, d, var)
            if rc != OK:
                raise RuntimeError(f"oracle schedule failed: {rc}")
        plan = plans[var]
        for a in range(n_alloc):
            c = vi * n_alloc + a
            col = alloc[2 * n0: 2 * n0 + max(plan["n_rows"], 1), c]
            out[c] = bound_plan(plan, batch.M, np.ascontiguousarray(col), 1)
    best = int(np.argmin(out)) if len(out) else -1
    return out, (int(out[best]) if best >= 0 else 0), best


def splitmix64(x: int) -> int:
    return int(lib().or_splitmix64(C.c_uint64(x & (2**64 - 1))))


def generated_allocation(seed: int, d: int, c: int, n_rows: int, levels, n_alloc: int):
    """Allocation of generated candidate c of DAG d over n_rows plan rows (uint8 array):
    zeros (keep the schedule) when c is the first allocation of its variant."""
    out = np.zeros(max(n_rows, 1), np.uint8)[:n_rows]
    if c % n_alloc == 0:
        return out
    L = lib()
    for r in range(n_rows):
        out[r] = levels[L.or_gen_level(C.c_uint64(seed), d, c, r, len(levels))]
    return out


SEARCH_RANDOM, SEARCH_EXHAUSTIVE, SEARCH_PERTURB = 0, 1, 2


def row_owner(plan: dict) -> np.ndarray:
    """Node each plan row belongs to: the row's node, or a segment's parent."""
    V = int(plan["V"])
    out = [int(r) if r < V else int(plan["seg_parent"][r - V]) for r in plan["row_id"][:plan["n_rows"]]]
    return np.asarray(out, np.int32)


def exhaustive_plan(plan: dict, M: int, levels, n_alloc: int) -> np.ndarray:
    """Bounds of allocations 0..n_alloc-1 of the exhaustive search on one plan (see
    or_exhaustive_plan): node u's digit (a / B^u) % B, B = len(levels) + 1, keeps (0) or
    picks levels[digit - 1] on every plan row of u."""
    n = int(plan["n_rows"])
    out = np.zeros(max(n_alloc, 1), np.int64)
    lev = np.ascontiguousarray(levels, np.uint8)
    own = np.ascontiguousarray(row_owner(plan) if n else np.zeros(1, np.int32), np.int32)
    load = np.ascontiguousarray(plan["row_load"] if n else np.zeros(1, np.int64), np.int64)
    k = np.ascontiguousarray(plan["row_k"] if n else np.zeros(1, np.int32), np.int32)
    m0 = np.ascontiguousarray(plan["row_m0"] if n else np.zeros(1, np.int32), np.int32)
    g = np.ascontiguousarray(plan["row_group"] if n else np.zeros(1, np.int32), np.int32)
    lib().or_exhaustive_plan(n, _ptr(load, _P64), _ptr(k, _P32), _ptr(m0, _P32), _ptr(g, _P32), _ptr(own, _P32),
                             int(M), len(lev), _ptr(lev, _PU8), int(n_alloc), _ptr(out, _P64))
    return out[:n_alloc]


def exhaustive_search_dag(batch, d: int, variant_ids, levels, n_alloc: int):
    """Bounds of every candidate c = v * n_alloc + a of the exhaustive search of DAG d and
    the argmin (smallest bound, lowest candidate id)."""
    out = np.zeros(len(variant_ids) * n_alloc, np.int64)
    for vi, var in enumerate(variant_ids):
        rc, plan = schedule_dag_of(batch, d, int(var))
        if rc != OK:
            raise RuntimeError(f"oracle schedule failed: {rc}")
        out[vi * n_alloc:(vi + 1) * n_alloc] = exhaustive_plan(plan, batch.M, levels, n_alloc)
    best = int(np.argmin(out))
    return out, int(out[best]), best


def perturbed_m(m0: int, code: int) -> int:
    """SMs of a row scheduled on m0 SMs under perturbation `code`: 0 keeps the schedule
    (returned as 0), 1 halves, 2 takes one away, 3 adds one, 4 doubles; a changed count is
    at least 1 and at most 255."""
    if code == 0:
        return 0
    m = {1: m0 // 2, 2: m0 - 1, 3: m0 + 1, 4: 2 * m0}[code]
    return min(255, max(1, m))


def search_dag_generated(batch, d: int, variant_ids, n_alloc: int, levels, seed: int, mode: int = SEARCH_RANDOM):
    """Bounds of every generated candidate of DAG d and the argmin (min bound, lowest id)
    for the random, exhaustive or perturbation search."""
    if mode == SEARCH_EXHAUSTIVE:
        return exhaustive_search_dag(batch, d, variant_ids, levels, n_alloc)
    if mode == SEARCH_PERTURB:
        plans = {}
        out = np.zeros(len(variant_ids) * n_alloc, np.int64)
        L = lib()
        for vi, var in enumerate(variant_ids):
            if var not in plans:
                rc, plans[var] = schedule_dag_of(batch, d, int(var))
                if rc != OK:
                    raise RuntimeError(f"oracle schedule failed: {rc}")
            plan = plans[var]
            n = int(plan["n_rows"])
            for a in range(n_alloc):
                c = vi * n_alloc + a
                alloc = np.zeros(max(n, 1), np.uint8)[:n]
                if a:
                    for r in range(n):
                        code = int(levels[L.or_gen_level(C.c_uint64(seed), d, c, r, len(levels))])
                        alloc[r] = perturbed_m(int(plan["row_m0"][r]), code)
                out[c] = bound_plan(plan, batch.M, alloc if n else None, 1)
        best = int(np.argmin(out))
        return out, int(out[best]), best
    return search_dag_random(batch, d, variant_ids, n_alloc, levels, seed)


def search_dag_random(batch, d: int, variant_ids, n_alloc: int, levels, seed: int):
    """Bounds of every generated candidate of DAG d and the argmin (min bound, lowest id)."""
    plans = {}
    nv = len(variant_ids)
    out = np.zeros(nv * n_alloc, np.int64)
    for vi, var in enumerate(variant_ids):
        if var not in plans:
            rc, plans[var] = schedule_dag_of(batch, d, int(var))
            if rc != OK:
                raise RuntimeError(f"oracle schedule failed: {rc}")
        plan = plans[var]
        for a in range(n_alloc):
            c = vi * n_alloc + a
            alloc = generated_allocation(seed, d, c, plan["n_rows"], levels, n_alloc)
            out[c] = bound_plan(plan, batch.M, alloc if len(alloc) else None, 1)
    best = int(np.argmin(out))
    return out, int(out[best]), best
