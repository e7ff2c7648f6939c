"""CPU oracle of the learned proposer (test infrastructure only).

The paper has no learned component: it bounds the makespan of ONE allocation (Eq.1,
Lemma 1, Theorem 1) and picks the allocation with the Eq.5 heuristic of Alg.2. The
library adds a proposer whose output is always checked exactly against that bound, so
only its definition matters here. This module writes the definition out in float64
numpy, slowly and plainly, for the tests: node features, mean aggregation over
predecessors and successors, three ReLU layers of width 128, a linear head, softmax
cross-entropy, the analytic gradient (hand-derived backward pass), one Adam step, and the
k most likely joint level assignments of independent per-node distributions.

With `bf16=True` the forward pass rounds to bfloat16 (round to nearest even) exactly where
the library stores bf16 values: node features, layer inputs after aggregation, weights of
the three layers, and layer outputs. The backward pass treats that rounding as the
identity. With `bf16=False` everything is float64, which the finite-difference tests use.

Nothing here is shared with the CUDA path; only tests, the smoke check and the
benchmark's CPU leg may import it.
"""
from __future__ import annotations

import heapq

import numpy as np

FEAT, HIDDEN, MAX_LEVELS = 16, 128, 16

# parameter layout (float offsets): W1 [48 x 128], b1, W2 [384 x 128], b2, W3, b3,
# Wh [128 x 16], bh [16]
_SIZES = [("W1", (3 * FEAT, HIDDEN)), ("b1", (HIDDEN,)), ("W2", (3 * HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (3 * HIDDEN, HIDDEN)), ("b3", (HIDDEN,)), ("Wh", (HIDDEN, MAX_LEVELS)), ("bh", (MAX_LEVELS,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in _SIZES)


def unpack(p):
    """Flat parameter vector -> dict of arrays (views)."""
    out, o = {}, 0
    for name, shape in _SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in _SIZES])


def bf16(x):
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ------------------------------------------------------------------ graph and features
def graph(batch):
    """Global predecessor / successor lists of every node (node ids offset by node_off)."""
    N = int(batch.node_off[-1])
    preds = [[] for _ in range(N)]
    succs = [[] for _ in range(N)]
    for d in range(batch.n_dags):
        rp, col, _, _ = batch.dag(d)
        n0 = int(batch.node_off[d])
        for u in range(len(rp) - 1):
            for e in range(rp[u], rp[u + 1]):
                v = int(col[e])
                succs[n0 + u].append(n0 + v)
                preds[n0 + v].append(n0 + u)
    return preds, succs


def features(batch, level, wanc, m, preds, succs):
    """x_i: log2 C^_i / 32, k_i / 64, log2(1 + indeg) / 8, log2(1 + outdeg) / 8,
    level_i / depth of its DAG (0 if the DAG has one level), W^anc_i / sum of C^ over its
    DAG, log2 max(m_i, 1) / 12, 1, then zeros to 16 columns. level, wanc and m are the
    paper schedule's per-node outputs (topological level, Eq.2 ancestor weight, Eq.5 SMs)."""
    N = int(batch.node_off[-1])
    x = np.zeros((N, FEAT))
    for d in range(batch.n_dags):
        a, b = int(batch.node_off[d]), int(batch.node_off[d + 1])
        tot = float(np.sum(batch.wcet[a:b], dtype=np.float64))
        depth = int(np.max(level[a:b])) if b > a else 0
        for i in range(a, b):
            x[i, 0] = np.log2(float(batch.wcet[i])) / 32.0
            x[i, 1] = float(batch.k64[i]) / 64.0
            x[i, 2] = np.log2(1.0 + len(preds[i])) / 8.0
            x[i, 3] = np.log2(1.0 + len(succs[i])) / 8.0
            x[i, 4] = level[i] / depth if depth > 0 else 0.0
            x[i, 5] = float(wanc[i]) / tot if tot > 0 else 0.0
            x[i, 6] = np.log2(max(int(m[i]), 1)) / 12.0
            x[i, 7] = 1.0
    return x


def aggregate(h, preds, succs):
    """[h | mean over predecessors | mean over successors] (zeros where none)."""
    N, K = h.shape
    mp = np.zeros((N, K))
    ms = np.zeros((N, K))
    for v in range(N):
        if preds[v]:
            mp[v] = h[preds[v]].mean(axis=0)
        if succs[v]:
            ms[v] = h[succs[v]].mean(axis=0)
    return np.concatenate([h, mp, ms], axis=1)


def aggregate_T(dA, preds, succs, K):
    """Transpose of aggregate: gradient w.r.t. h from the gradient w.r.t. [h | mp | ms]."""
    N = dA.shape[0]
    dh = dA[:, :K].copy()
    for v in range(N):
        if preds[v]:
            g = dA[v, K:2 * K] / len(preds[v])
            for u in preds[v]:
                dh[u] += g
        if succs[v]:
            g = dA[v, 2 * K:] / len(succs[v])
            for w in succs[v]:
                dh[w] += g
    return dh


# ------------------------------------------------------------------ network
def forward(p, x, preds, succs, n_levels, bf=True):
    """Returns logits [N x n_levels] and the cache the backward pass needs."""
    P = unpack(p)
    rnd = bf16 if bf else (lambda a: np.asarray(a, np.float64))
    h = rnd(x)
    cache = []
    for l in range(3):
        W, b = P[f"W{l + 1}"], P[f"b{l + 1}"]
        A = rnd(aggregate(h, preds, succs))
        z = A @ rnd(W) + b
        out = rnd(np.maximum(z, 0.0))
        cache.append((h, A, z, out))
        h = out
    logits = h @ P["Wh"][:, :n_levels] + P["bh"][:n_levels]
    return logits, cache


def loss_and_grad(p, x, preds, succs, labels, n_levels, bf=True):
    """Mean softmax cross-entropy over nodes with 0 <= label < n_levels, and its gradient
    w.r.t. the flat parameter vector (bf16 rounding passed straight through)."""
    P = unpack(p)
    logits, cache = forward(p, x, preds, succs, n_levels, bf)
    lab = np.asarray(labels)
    mask = (lab >= 0) & (lab < n_levels)
    n = int(mask.sum())
    G = {name: np.zeros(shape) for name, shape in _SIZES}
    if n == 0:
        return 0.0, pack(G)
    z = logits - logits.max(axis=1, keepdims=True)
    lse = np.log(np.exp(z).sum(axis=1))
    idx = np.where(mask)[0]
    loss = float(np.sum(lse[idx] - z[idx, lab[idx]]) / n)
    dz = np.exp(z - lse[:, None])
    dz[np.arange(len(lab)), np.where(mask, lab, 0)] -= 1.0
    dz[~mask] = 0.0
    dz /= n
    h3 = cache[2][3]
    G["Wh"][:, :n_levels] = h3.T @ dz
    G["bh"][:n_levels] = dz.sum(axis=0)
    dh = dz @ P["Wh"][:, :n_levels].T
    for l in (2, 1, 0):
        h_in, A, zl, _ = cache[l]
        W = P[f"W{l + 1}"]
        dZ = dh * (zl > 0)
        G[f"W{l + 1}"] = A.T @ dZ
        G[f"b{l + 1}"] = dZ.sum(axis=0)
        if l > 0:
            Wr = bf16(W) if bf else W
            dh = aggregate_T(dZ @ Wr.T, preds, succs, h_in.shape[1])
    return loss, pack(G)


def grad_magnitude(p, x, preds, succs, labels, n_levels, bf=True, gate_slack=0.0):
    """Element-wise scales of the difference between this gradient and one computed with
    other rounding (bf16 operands, fp32 sums), as a pair (mag, flip):

    mag -- the backward pass of loss_and_grad run on absolute values (|dz|, |h|, |A|, |W|
    in place of the signed terms): every gradient element's sum of |products|, the quantity
    a relative rounding error of each product is proportional to, carried through the
    layers as the backward pass carries the gradient. By the triangle inequality it bounds
    |gradient| element-wise.

    flip -- a bound on what ReLU gates that rounding may set the other way can change: a
    gate is uncertain where |z| is within gate_slack of the sum |A| |W| + |b| that z adds
    up. An uncertain gate adds or drops its whole term |dh| at its layer, and that change
    flows down through the later (lower) layers on absolute values with every open or
    uncertain gate passing it.

    gate_slack = 0 gives exactly the gates of loss_and_grad (flip = 0)."""
    P = unpack(p)
    logits, cache = forward(p, x, preds, succs, n_levels, bf)
    lab = np.asarray(labels)
    mask = (lab >= 0) & (lab < n_levels)
    n = int(mask.sum())
    G = {name: np.zeros(shape) for name, shape in _SIZES}
    F = {name: np.zeros(shape) for name, shape in _SIZES}
    if n == 0:
        return pack(G), pack(F)
    z = logits - logits.max(axis=1, keepdims=True)
    lse = np.log(np.exp(z).sum(axis=1))
    dz = np.exp(z - lse[:, None])
    dz[np.arange(len(lab)), np.where(mask, lab, 0)] -= 1.0
    dz[~mask] = 0.0
    dz = np.abs(dz) / n
    h3 = cache[2][3]
    G["Wh"][:, :n_levels] = np.abs(h3).T @ dz
    G["bh"][:n_levels] = dz.sum(axis=0)
    dh = dz @ np.abs(P["Wh"][:, :n_levels]).T
    eh = np.zeros_like(dh)  # bound on the change of dh that flipped gates above can cause
    for l in (2, 1, 0):
        h_in, A, zl, _ = cache[l]
        W = P[f"W{l + 1}"]
        Wr = bf16(W) if bf else W
        zmag = np.abs(A) @ np.abs(Wr) + np.abs(P[f"b{l + 1}"])
        unsure = np.abs(zl) <= gate_slack * zmag
        gate = (zl > 0) | unsure
        dZ = dh * gate
        eZ = eh * gate + dh * unsure
        G[f"W{l + 1}"] = np.abs(A).T @ dZ
        G[f"b{l + 1}"] = dZ.sum(axis=0)
        F[f"W{l + 1}"] = np.abs(A).T @ eZ
        F[f"b{l + 1}"] = eZ.sum(axis=0)
        if l > 0:
            dh = aggregate_T(dZ @ np.abs(Wr).T, preds, succs, h_in.shape[1])
            eh = aggregate_T(eZ @ np.abs(Wr).T, preds, succs, h_in.shape[1])
    return pack(G), pack(F)


def adam(p, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected moments); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------ k best assignments
def k_best(logits, k):
    """The k most likely joint assignments of independent per-node categoricals given by
    logit rows: returns a list of (cost, assignment) with cost = sum_i (max_l z_il - z_i,a_i),
    smallest first. Exact: after each node, only the k cheapest partial assignments can
    extend to one of the k cheapest full assignments (costs are sums over nodes), so they
    are all that is kept."""
    z = np.asarray(logits, np.float64)
    beam = [(0.0, ())]
    for i in range(z.shape[0]):
        best = z[i].max()
        ext = [(c + (best - z[i, l]), a + (l,)) for c, a in beam for l in range(z.shape[1])]
        beam = heapq.nsmallest(k, ext, key=lambda t: t[0])
    return beam


def cost_of(logits, assignment):
    z = np.asarray(logits, np.float64)
    return float(sum(z[i].max() - z[i, a] for i, a in enumerate(assignment)))
