"""Seeded synthetic workloads (DAG batches and candidate allocations).

This module only draws random inputs. It holds none of the scheduling or bound
arithmetic, so both the CUDA path and the CPU oracle can take their inputs from it.

Batch format (the C-ABI's `dagrt_load_csr` layout):
  node_off[n+1] int64  - first node of DAG d is node_off[d]; V_d = node_off[d+1]-node_off[d]
  edge_off[n+1] int64  - first edge of DAG d is edge_off[d]
  row_ptr[sum(V_d+1)] int32 - DAG-local successor CSR; DAG d's V_d+1 entries start at
                              node_off[d] + d and are relative to edge_off[d]
  col[sum(E_d)] int32  - DAG-local successor ids, strictly increasing within a row
  wcet[sum(V_d)] int64 - computation load (WCET at one SM, integer ticks, >= 1)
  k64[sum(V_d)] uint8  - parallel fraction numerator k, fraction f = k/64

Generators follow the workload descriptions the paper's experiments use (layered
DAGs of the Evaluation section) and the five batch configurations this library is
measured on; where a description leaves a detail open, the choice is written next to
the code that makes it.
"""
from __future__ import annotations

import dataclasses
import numpy as np

BASE_SEED = 20260226


@dataclasses.dataclass
class Batch:
    node_off: np.ndarray
    edge_off: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    wcet: np.ndarray
    k64: np.ndarray
    M: int
    name: str = ""

    @property
    def n_dags(self) -> int:
        return len(self.node_off) - 1

    def n_nodes(self, d: int) -> int:
        return int(self.node_off[d + 1] - self.node_off[d])

    def dag(self, d: int):
        """Return (row_ptr, col, wcet, k64) views of DAG d, all DAG-local."""
        n0, n1 = int(self.node_off[d]), int(self.node_off[d + 1])
        e0, e1 = int(self.edge_off[d]), int(self.edge_off[d + 1])
        rp = self.row_ptr[n0 + d: n1 + d + 1]
        return rp, self.col[e0:e1], self.wcet[n0:n1], self.k64[n0:n1]

    def subset(self, ids) -> "Batch":
        return from_dags([self.dag(int(d)) for d in ids], self.M, self.name + "-subset")

    def total_nodes(self) -> int:
        return int(self.node_off[-1])

    def total_edges(self) -> int:
        return int(self.edge_off[-1])

    def input_bytes(self) -> int:
        """Bytes of the batch arrays a bound evaluation must read once."""
        return int(self.node_off.nbytes + self.edge_off.nbytes + self.row_ptr.nbytes
                   + self.col.nbytes + self.wcet.nbytes + self.k64.nbytes)


def from_dags(dags, M: int, name: str = "") -> Batch:
    """Pack a list of (row_ptr, col, wcet, k64) DAG-local arrays into a Batch."""
    n = len(dags)
    node_off = np.zeros(n + 1, np.int64)
    edge_off = np.zeros(n + 1, np.int64)
    for d, (rp, col, w, k) in enumerate(dags):
        node_off[d + 1] = node_off[d] + len(w)
        edge_off[d + 1] = edge_off[d] + len(col)
    row_ptr = np.concatenate([np.asarray(x[0], np.int32) for x in dags]) if n else np.zeros(0, np.int32)
    col = np.concatenate([np.asarray(x[1], np.int32) for x in dags]) if n else np.zeros(0, np.int32)
    wcet = np.concatenate([np.asarray(x[2], np.int64) for x in dags]) if n else np.zeros(0, np.int64)
    k64 = np.concatenate([np.asarray(x[3], np.uint8) for x in dags]) if n else np.zeros(0, np.uint8)
    return Batch(node_off, edge_off, row_ptr, col, wcet, k64, int(M), name)


def csr_from_edges(V: int, src, dst):
    """DAG-local successor CSR with strictly increasing successor ids per row."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(V + 1, np.int32)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return row_ptr, dst.astype(np.int32)


# ---------------------------------------------------------------- random pieces

def er_edges(rng: np.random.Generator, V: int, p: float):
    """Erdos-Renyi DAG over the topological order 0..V-1: each pair i<j is an edge
    independently with probability p. Pairs are visited in row-major order of the
    strict upper triangle and the gaps between chosen pairs are geometric(p)."""
    n_pairs = V * (V - 1) // 2
    if n_pairs == 0 or p <= 0.0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    want = int(n_pairs * p + 8 * np.sqrt(n_pairs * p + 1) + 16)
    chosen = []
    pos = -1
    while True:
        gaps = rng.geometric(p, size=want)
        idx = pos + np.cumsum(gaps)
        chosen.append(idx[idx < n_pairs])
        if idx[-1] >= n_pairs:
            break
        pos = int(idx[-1])
    t = np.concatenate(chosen)
    i = np.arange(V, dtype=np.int64)
    row_start = i * V - i * (i + 1) // 2  # linear index of pair (i, i+1)
    src = np.searchsorted(row_start, t, side="right") - 1
    dst = t - row_start[src] + src + 1
    return src, dst


def wcet_log_uniform(rng, V: int, decades: float = 4.0):
    """floor(10^(decades*U)), U ~ U[0,1): integer ticks in [1, 10^decades)."""
    return np.floor(10.0 ** (decades * rng.random(V))).astype(np.int64)


def wcet_uniform(rng, V: int, lo: int, hi: int):
    return rng.integers(lo, hi + 1, size=V, dtype=np.int64)


def wcet_lognormal(rng, V: int, mu: float = 4.0, sigma: float = 1.5):
    """max(1, floor(exp(N(mu, sigma^2)) + 0.5)), clamped below 2^32."""
    x = np.floor(np.exp(rng.normal(mu, sigma, size=V)) + 0.5)
    return np.clip(x, 1, 2**32 - 1).astype(np.int64)


def k64_uniform(rng, V: int, frac_lo: float):
    """Parallel fraction uniform on [frac_lo, 1] in steps of 1/64: k in [round(64 lo), 64]."""
    lo = int(round(64 * frac_lo))
    return rng.integers(lo, 65, size=V).astype(np.uint8)


def layered_edges(rng, V: int, depth: int, max_width: int = 64, skip_p: float = 0.02):
    """Compiler-style layered DAG: raw layer widths U[1, max_width] scaled to sum to V
    (the last layer absorbs the remainder, every layer keeps >= 1 node); each node after
    the first layer takes 1-3 distinct predecessors from the previous layer (fork-join);
    with probability skip_p a node also takes one skip edge from a uniformly chosen node
    at least two layers back."""
    depth = max(1, min(depth, V))
    raw = rng.integers(1, max_width + 1, size=depth).astype(np.float64)
    widths = np.maximum(1, np.floor(raw * V / raw.sum())).astype(np.int64)
    while widths.sum() > V:
        j = int(np.argmax(widths))
        widths[j] -= 1
    widths[-1] += V - widths.sum()
    start = np.concatenate([[0], np.cumsum(widths)])
    src, dst = [], []
    for l in range(1, depth):
        p0, p1 = start[l - 1], start[l]
        for v in range(start[l], start[l + 1]):
            npred = min(int(rng.integers(1, 4)), p1 - p0)
            preds = rng.choice(np.arange(p0, p1), size=npred, replace=False)
            src.extend(int(u) for u in preds)
            dst.extend([v] * npred)
            if l >= 2 and rng.random() < skip_p:
                u = int(rng.integers(0, start[l - 1]))
                if u not in preds:
                    src.append(u)
                    dst.append(v)
    return np.asarray(src, np.int64), np.asarray(dst, np.int64)


def paper_layered_edges(rng, depth: int, P: int):
    """Layered DAG in the style of the paper's synthetic setup: a single source, then
    `depth` layers whose widths are uniform in [2, P]; every node takes 1-3 predecessors
    from the previous layer, and a single sink closes the graph."""
    widths = [1] + [int(rng.integers(2, P + 1)) for _ in range(depth)] + [1]
    start = np.concatenate([[0], np.cumsum(widths)])
    V = int(start[-1])
    src, dst = [], []
    for l in range(1, len(widths)):
        p0, p1 = start[l - 1], start[l]
        for v in range(start[l], start[l + 1]):
            if l == len(widths) - 1:
                preds = np.arange(p0, p1)
            else:
                npred = min(int(rng.integers(1, 4)), p1 - p0)
                preds = rng.choice(np.arange(p0, p1), size=npred, replace=False)
            src.extend(int(u) for u in preds)
            dst.extend([v] * len(preds))
    # nodes of a layer with no successor link to the next layer's first node
    src_a = np.asarray(src, np.int64)
    has_succ = np.zeros(V, bool)
    has_succ[src_a] = True
    for l in range(1, len(widths) - 1):
        for v in range(start[l], start[l + 1]):
            if not has_succ[v]:
                src.append(v)
                dst.append(int(start[l + 1]))
    return V, np.asarray(src, np.int64), np.asarray(dst, np.int64)


def paper_layered_batch(n_dags: int, P: int, M: int, c_avg: int, seed: int, depth_lo: int = 5,
                        depth_hi: int = 8, name: str = "paper-layered") -> Batch:
    """The paper's synthetic set-up: per DAG a depth uniform in [depth_lo, depth_hi] and
    layers of width U[2, P] between a single source and a single sink (paper_layered_edges),
    node loads uniform on [1, 2 c_avg - 1] (mean c_avg), fully parallel kernels (k = 64)."""
    dags = []
    for d in range(n_dags):
        rng = _rng(seed, d)
        depth = int(rng.integers(depth_lo, depth_hi + 1))
        V, s, t = paper_layered_edges(rng, depth, P)
        rp, col = csr_from_edges(V, s, t)
        w = rng.integers(1, 2 * c_avg, size=V).astype(np.int64)
        dags.append((rp, col, w, np.full(V, 64, np.uint8)))
    return from_dags(dags, M, name)


def small_m_batch(n_dags: int, seed: int, M: int = 8, v_lo: int = 3, v_hi: int = 6, p: float = 0.35,
                  load_hi: int = 40, frac_lo: float = 0.5) -> Batch:
    """Small DAGs on a small GPU, where the Eq.5 allocation is often not the best one and an
    exhaustive allocation search is cheap: V ~ U[v_lo, v_hi], Erdos-Renyi edges with
    probability p over a topological order, loads U[1, load_hi] ticks, parallel fractions
    U[frac_lo, 1] in 1/64 steps."""
    dags = []
    for d in range(n_dags):
        rng = _rng(seed, d)
        V = int(rng.integers(v_lo, v_hi + 1))
        s, t = er_edges(rng, V, p)
        rp, col = csr_from_edges(V, s, t)
        dags.append((rp, col, wcet_uniform(rng, V, 1, load_hi), k64_uniform(rng, V, frac_lo)))
    return from_dags(dags, M, "small-m")


def implicit_deadlines(batch: Batch, utilisation: float) -> np.ndarray:
    """Implicit deadlines D = T of a periodic task per DAG at normalised utilisation U:
    T = ceil(sum of C^ / (M U)) ticks (the DAG's work over the GPU's capacity in one
    period)."""
    vol = np.add.reduceat(batch.wcet, batch.node_off[:-1]) if batch.total_nodes() else np.zeros(batch.n_dags)
    vol = np.where(np.diff(batch.node_off) > 0, vol, 0).astype(np.float64)
    return np.ceil(vol / (batch.M * float(utilisation))).astype(np.int64)


# ---------------------------------------------------------------- batch configs

def _rng(seed: int, d: int):
    return np.random.default_rng([int(seed), int(d)])


def er_sizes(n_dags: int, v_lo: int, v_hi: int, seed: int) -> np.ndarray:
    """Node count of every DAG of er_batch(n_dags, v_lo, v_hi, ..., seed): the first draw
    of each DAG's own stream, without generating the DAG."""
    return np.asarray([int(_rng(seed, d).integers(v_lo, v_hi + 1)) for d in range(n_dags)], np.int64)


def er_batch(n_dags: int, v_lo: int, v_hi: int, p: float, M: int, seed: int,
             wcet="loguniform", frac_lo: float = 0.3, name: str = "", ids=None) -> Batch:
    """Erdos-Renyi DAGs, each from its own stream (seed, d); with `ids` only those DAGs of
    the n_dags-DAG batch, in the order given (DAG ids[i] is identical to DAG ids[i] of the
    whole batch)."""
    dags = []
    for d in (range(n_dags) if ids is None else ids):
        rng = _rng(seed, d)
        V = int(rng.integers(v_lo, v_hi + 1))
        s, t = er_edges(rng, V, p)
        rp, col = csr_from_edges(V, s, t)
        if wcet == "loguniform":
            w = wcet_log_uniform(rng, V)
        elif wcet == "uniform100":
            w = wcet_uniform(rng, V, 1, 100)
        else:
            raise ValueError(wcet)
        k = k64_uniform(rng, V, frac_lo)
        dags.append((rp, col, w, k))
    return from_dags(dags, M, name)


def config(idx: int, n_dags: int | None = None, seed: int | None = None, ids=None) -> Batch:
    """The five measured workloads (1-based index). `n_dags` shrinks a batch (same
    per-DAG streams, so DAG d is identical at every batch size); `ids` (configs 2-4) keeps
    only those DAGs of the batch."""
    seed = BASE_SEED + idx if seed is None else seed
    if ids is not None and idx in (2, 3, 4):
        lo, hi, p = {2: (20, 200, 0.1), 3: (50, 500, 0.05), 4: (100, 1000, 0.05)}[idx]
        return er_batch(len(ids), lo, hi, p, 148, seed, name=f"cfg{idx}-shard", ids=[int(d) for d in ids])
    if idx == 1:   # single DAG, 20 nodes, p=0.2, WCET U[1,100], f U[0.5,1], M=8
        return er_batch(1 if n_dags is None else n_dags, 20, 20, 0.2, 8, seed,
                        wcet="uniform100", frac_lo=0.5, name="cfg1-er20")
    if idx == 2:   # 10,000 DAGs, 20-200 nodes, p=0.1, log-uniform WCET, f U[0.3,1], M=148
        return er_batch(10000 if n_dags is None else n_dags, 20, 200, 0.1, 148, seed,
                        name="cfg2-er20-200")
    if idx == 3:   # 1,000 DAGs, 50-500 nodes, p=0.05, M=148
        return er_batch(1000 if n_dags is None else n_dags, 50, 500, 0.05, 148, seed,
                        name="cfg3-er50-500")
    if idx == 4:   # 10,000 DAGs, 100-1,000 nodes, p=0.05, M=148
        return er_batch(10000 if n_dags is None else n_dags, 100, 1000, 0.05, 148, seed,
                        name="cfg4-er100-1000")
    if idx == 5:   # 200 layered DAGs, 2,000-20,000 nodes, depth 20-60, width 1-64
        n = 200 if n_dags is None else n_dags
        dags = []
        for d in range(n):
            rng = _rng(seed, d)
            V = int(rng.integers(2000, 20001))
            D = int(rng.integers(20, 61))
            s, t = layered_edges(rng, V, D)
            rp, col = csr_from_edges(V, s, t)
            w = wcet_lognormal(rng, V)
            k = k64_uniform(rng, V, 0.3)
            dags.append((rp, col, w, k))
        return from_dags(dags, 148, "cfg5-layered")
    raise ValueError(idx)


def small_config(idx: int, n_dags: int, v_lo: int, v_hi: int, seed: int | None = None) -> Batch:
    """A config's distributions at reduced DAG sizes, for oracle-speed parity runs."""
    seed = (BASE_SEED + 100 + idx) if seed is None else seed
    p = {1: 0.2, 2: 0.1, 3: 0.05, 4: 0.05}[idx]
    M = 8 if idx == 1 else 148
    wc = "uniform100" if idx == 1 else "loguniform"
    fl = 0.5 if idx == 1 else 0.3
    return er_batch(n_dags, v_lo, v_hi, p, M, seed, wcet=wc, frac_lo=fl, name=f"cfg{idx}-small")


# ---------------------------------------------------------------- candidates

def row_capacity(batch: Batch) -> np.ndarray:
    """Rows reserved per DAG in a candidate buffer: 2*V_d (every node plus at most one
    segment per group, and a DAG has at most V_d groups)."""
    return 2 * np.diff(batch.node_off)


def candidate_allocations(batch: Batch, n_variants: int, n_alloc: int, levels, seed: int,
                          cand_stride: int | None = None, keep_scheduled: bool = True):
    """Random per-node SM allocations, uint8, laid out [2*node_off[d] + row][cand].

    Candidate c = v*n_alloc + a belongs to structure variant v. Column a == 0 of each
    variant is all zeros when keep_scheduled is set: a zero byte means "keep the
    schedule's own allocation for this row". Other bytes are drawn uniformly from
    `levels`. Columns past n_cand (stride padding) are zero and never read."""
    n_cand = n_variants * n_alloc
    if cand_stride is None:
        cand_stride = (n_cand + 15) // 16 * 16
    levels = np.asarray(levels, np.uint8)
    rows = int(2 * batch.total_nodes())
    out = np.zeros((rows, cand_stride), np.uint8)
    rng = np.random.default_rng([int(seed), 7])
    if rows:
        idx = rng.integers(0, len(levels), size=(rows, n_cand))
        out[:, :n_cand] = levels[idx]
        if keep_scheduled:
            out[:, 0:n_cand:n_alloc] = 0
    return out, cand_stride
