"""Pins of the proposer's CPU oracle (oracle/gnn.py) against facts that do not come from
the oracle itself: a library's bfloat16 rounding, hand-computed aggregates and features,
the adjoint identity of the aggregation, central finite differences of the loss, closed
forms of cross-entropy and of Adam's first step, and brute-force enumeration of joint
assignments."""
import itertools

import numpy as np
import pytest
import torch

from oracle import gnn as G
from paper_2602_20826_gb300 import workloads as W


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-8, 8, 5000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 65504.0]])
    ref = torch.from_numpy(x).to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(G.bf16(x), ref)


def test_aggregate_hand_example():
    # edges 0->1, 0->2, 1->2
    preds = [[], [0], [0, 1]]
    succs = [[1, 2], [2], []]
    h = np.array([[1.0], [2.0], [4.0]])
    A = G.aggregate(h, preds, succs)
    assert A.tolist() == [[1.0, 0.0, 3.0], [2.0, 1.0, 4.0], [4.0, 1.5, 0.0]]


def test_aggregate_transpose_is_adjoint():
    rng = np.random.default_rng(2)
    b = W.small_config(2, 3, 4, 12, seed=5)
    preds, succs = G.graph(b)
    N, K = b.total_nodes(), 7
    h = rng.normal(size=(N, K))
    Y = rng.normal(size=(N, 3 * K))
    lhs = float(np.sum(G.aggregate(h, preds, succs) * Y))
    rhs = float(np.sum(h * G.aggregate_T(Y, preds, succs, K)))
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


def test_graph_lists_follow_csr():
    b = W.small_config(2, 2, 4, 12, seed=3)
    preds, succs = G.graph(b)
    n_edges = sum(len(s) for s in succs)
    assert n_edges == b.total_edges() == sum(len(p) for p in preds)
    for u, ss in enumerate(succs):
        for v in ss:
            assert u in preds[v]


def test_features_hand_example():
    # one DAG 0 -> 1 with C^ = (4, 1), k = (32, 64); schedule outputs given explicitly
    b = W.from_dags([(np.array([0, 1, 1], np.int32), np.array([1], np.int32),
                      np.array([4, 1], np.int64), np.array([32, 64], np.uint8))], 8, "hand")
    preds, succs = G.graph(b)
    x = G.features(b, level=np.array([0, 1]), wanc=np.array([0, 4]), m=np.array([2, 1]), preds=preds, succs=succs)
    e0 = [2 / 32, 0.5, 0.0, 1 / 8, 0.0, 0.0, 1 / 12, 1.0] + [0.0] * 8
    e1 = [0.0, 1.0, 1 / 8, 0.0, 1.0, 0.8, 0.0, 1.0] + [0.0] * 8
    assert np.allclose(x, [e0, e1], rtol=0, atol=1e-15)


def _tiny(seed=0, n_dags=2, scale=1.0):
    b = W.small_config(2, n_dags, 4, 12, seed=seed)
    preds, succs = G.graph(b)
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, size=(b.total_nodes(), G.FEAT))
    p = rng.normal(size=G.N_PARAMS) * 0.2 * scale
    return b, preds, succs, x, p, rng


def test_forward_matches_per_node_loops():
    b, preds, succs, x, p, _ = _tiny(1)
    L = 5
    logits, _ = G.forward(p, x, preds, succs, L, bf=False)
    P = G.unpack(p)
    h = x
    for l in range(3):
        Wl, bl = P[f"W{l + 1}"], P[f"b{l + 1}"]
        K = h.shape[1]
        out = np.zeros((len(h), G.HIDDEN))
        for v in range(len(h)):
            z = bl.copy()
            z += h[v] @ Wl[:K]
            for u in preds[v]:
                z += (h[u] @ Wl[K:2 * K]) / len(preds[v])
            for w in succs[v]:
                z += (h[w] @ Wl[2 * K:]) / len(succs[v])
            out[v] = np.maximum(z, 0)
        h = out
    ref = h @ P["Wh"][:, :L] + P["bh"][:L]
    assert np.allclose(logits, ref, rtol=1e-12, atol=1e-12)


def test_gradient_central_differences():
    b, preds, succs, x, p, rng = _tiny(3, n_dags=2)
    L = 6
    labels = rng.integers(-1, L, size=b.total_nodes())
    loss, g = G.loss_and_grad(p, x, preds, succs, labels, L, bf=False)
    offs = {}
    o = 0
    for name, shape in G._SIZES:
        offs[name] = (o, o + int(np.prod(shape)))
        o += int(np.prod(shape))
    idx = []
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a, e = offs[name]
        idx += list(rng.integers(a, e, size=6))
    a, e = offs["Wh"]  # only the first L columns of Wh are live
    idx += [a + int(r) * G.MAX_LEVELS + int(c) for r, c in zip(rng.integers(0, G.HIDDEN, 6), rng.integers(0, L, 6))]
    a, _ = offs["bh"]
    idx += [a + i for i in range(L)]
    eps = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (G.loss_and_grad(pp, x, preds, succs, labels, L, bf=False)[0] -
              G.loss_and_grad(pm, x, preds, succs, labels, L, bf=False)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])
    # dead head columns get no gradient
    a, e = offs["Wh"]
    assert np.all(g[a:e].reshape(G.HIDDEN, G.MAX_LEVELS)[:, L:] == 0)


def test_grad_magnitude_bounds_gradient_and_is_exact_without_cancellation():
    """grad_magnitude (the error scale of the GPU gradient test) is the backward pass on
    absolute values: it bounds |gradient| element-wise, and equals it where no term can
    cancel -- all parameters and inputs non-negative and one labelled node whose softmax
    gradient is zero except on its label (a one-level head)."""
    b, preds, succs, x, p, rng = _tiny(5, n_dags=2)
    L = 6
    labels = rng.integers(-1, L, size=b.total_nodes())
    _, g = G.loss_and_grad(p, x, preds, succs, labels, L, bf=False)
    mag, flip = G.grad_magnitude(p, x, preds, succs, labels, L, bf=False)
    assert not flip.any()
    assert (np.abs(g) <= mag * (1 + 1e-12) + 1e-300).all()
    assert mag.max() > 0
    # no cancellation: non-negative inputs and weights, two levels whose head column 0 is
    # zero, so dh = p_1 * Wh[:, 1] >= 0 and every product below the head is >= 0
    pa = np.abs(p) * 0.05
    P = G.unpack(pa)
    P["Wh"][:, 0] = 0.0
    P["bh"][:] = 0.0
    xa = np.abs(x)
    lab = np.full(b.total_nodes(), -1)
    lab[:3] = 0
    _, g1 = G.loss_and_grad(pa, xa, preds, succs, lab, 2, bf=False)
    m1, _ = G.grad_magnitude(pa, xa, preds, succs, lab, 2, bf=False)
    blocks = {}
    o = 0
    for name, shape in G._SIZES:
        n = int(np.prod(shape))
        blocks[name] = (o, o + n)
        o += n
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a, e = blocks[name]
        assert m1[a:e].max() > 0, name
        assert np.allclose(np.abs(g1[a:e]), m1[a:e], rtol=1e-10, atol=1e-300), name


def _grad_with_gates(p, x, preds, succs, labels, L, flip_layers):
    """The float64 gradient with the uncertain ReLU gates (|z| below 5% of its sum of
    |terms|) of the given layers set the other way, written out here: the backward pass of
    the network with those gate values, activations left as they are."""
    P = G.unpack(p)
    logits, cache = G.forward(p, x, preds, succs, L, bf=False)
    lab = np.asarray(labels)
    mask = (lab >= 0) & (lab < L)
    n = int(mask.sum())
    z = logits - logits.max(axis=1, keepdims=True)
    sm = np.exp(z) / np.exp(z).sum(axis=1, keepdims=True)
    dz = sm.copy()
    dz[np.arange(len(lab)), np.where(mask, lab, 0)] -= 1.0
    dz[~mask] = 0.0
    dz /= n
    out = {name: np.zeros(shape) for name, shape in G._SIZES}
    out["Wh"][:, :L] = cache[2][3].T @ dz
    out["bh"][:L] = dz.sum(axis=0)
    dh = dz @ P["Wh"][:, :L].T
    for l in (2, 1, 0):
        h_in, A, zl, _ = cache[l]
        W = P[f"W{l + 1}"]
        gate = zl > 0
        if l in flip_layers:
            unsure = np.abs(zl) <= 0.05 * (np.abs(A) @ np.abs(W) + np.abs(P[f"b{l + 1}"]))
            gate = gate ^ unsure
        dZ = dh * gate
        out[f"W{l + 1}"] = A.T @ dZ
        out[f"b{l + 1}"] = dZ.sum(axis=0)
        if l > 0:
            dh = G.aggregate_T(dZ @ W.T, preds, succs, h_in.shape[1])
    return G.pack(out)


def test_grad_magnitude_flip_bound_covers_a_flipped_gate():
    """The flip part of grad_magnitude bounds the change of the gradient when ReLU gates
    near z = 0 go the other way: with a 5% slack, the gradient with every uncertain gate of
    layers 2 and 3 flipped differs from the oracle's by at most `flip` in every element,
    and flipping no gate reproduces loss_and_grad."""
    b, preds, succs, x, p, rng = _tiny(6, n_dags=2)
    L = 5
    labels = rng.integers(-1, L, size=b.total_nodes())
    _, g0 = G.loss_and_grad(p, x, preds, succs, labels, L, bf=False)
    assert np.allclose(_grad_with_gates(p, x, preds, succs, labels, L, ()), g0, rtol=1e-9,
                       atol=1e-12 * np.abs(g0).max())
    _, flip = G.grad_magnitude(p, x, preds, succs, labels, L, bf=False, gate_slack=0.05)
    g1 = _grad_with_gates(p, x, preds, succs, labels, L, (1, 2))
    assert np.abs(g1 - g0).max() > 0  # some gates did flip
    assert (np.abs(g1 - g0) <= flip * (1 + 1e-9) + 1e-12 * np.abs(g0).max()).all()


def test_cross_entropy_closed_form_at_zero_head():
    b, preds, succs, x, p, rng = _tiny(4)
    P = G.unpack(p)
    P["Wh"][:] = 0
    P["bh"][:] = 0
    L = 4
    labels = rng.integers(0, L, size=b.total_nodes())
    loss, g = G.loss_and_grad(p, x, preds, succs, labels, L, bf=True)
    assert abs(loss - np.log(L)) < 1e-12
    gb = G.unpack(g)["bh"][:L]
    freq = np.bincount(labels, minlength=L) / len(labels)
    assert np.allclose(gb, 1.0 / L - freq, atol=1e-12)


def test_unlabelled_nodes_give_zero():
    b, preds, succs, x, p, _ = _tiny(5)
    loss, g = G.loss_and_grad(p, x, preds, succs, np.full(b.total_nodes(), -1), 4)
    assert loss == 0.0 and not np.any(g)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(6)
    g = rng.normal(size=100)
    p = rng.normal(size=100)
    p1, m1, v1 = G.adam(p, np.zeros(100), np.zeros(100), g, 1, 1e-3)
    assert np.allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


@pytest.mark.parametrize("V,L,k", [(5, 3, 16), (4, 4, 7), (3, 2, 16), (6, 2, 1)])
def test_k_best_brute_force(V, L, k):
    rng = np.random.default_rng(V * 100 + L)
    z = rng.normal(size=(V, L)).astype(np.float32)
    allc = sorted(G.cost_of(z, a) for a in itertools.product(range(L), repeat=V))
    got = G.k_best(z, k)
    n = min(k, L ** V)
    assert len(got) == n
    assert np.allclose([c for c, _ in got], allc[:n], atol=1e-12)
    for c, a in got:
        assert abs(G.cost_of(z, a) - c) < 1e-12
    assert len({a for _, a in got}) == n
