"""Training and evaluation driver of the learned allocation proposer.

The network, its loss, gradients and optimiser all run in libdagrt's kernels (dagrt_model_*,
dagrt_train_step); this module only prepares labels and loops over batches.

Labels. The plain search (dagrt_search: structure variants x seeded sparse perturbations of
the schedule's own allocation, every candidate judged by the exact bound of Theorem 1) picks a winner
per DAG; a kernel's label is the level of the proposer's level list nearest (in log2) to
the SMs the winner gives the kernel's own plan row (0 in the winner's column means the
schedule's own m, Eq.5). DAGs whose schedule failed are unlabelled (-1).

Checkpoints (npz) hold the whole training state -- fp32 parameters, Adam's moments, the
step count -- and the level list; a run resumed from one continues exactly as the
uninterrupted run would.
"""
from __future__ import annotations

import time

import numpy as np

from . import dagrt

# SM levels the proposer chooses among (M = 148 on the measured configs)
LEARN_LEVELS = (1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 148)
# the plain search (4 structure variants x 64 allocations): allocation 0 keeps each
# schedule's own SMs, the others are sparse perturbations of them (a row keeps its m with
# probability 12/16, else it is halved, lowered by one, raised by one or doubled), the
# neighbourhood in which a search can beat the paper's Eq.5 allocation at all
SEARCH_LEVELS = (0,) * 12 + (1, 2, 3, 4)
SEARCH_MODE = dagrt.SEARCH_PERTURB
SEARCH_VARIANTS = (0, 1, 2, 3)
SEARCH_ALLOC = 64


def nearest_level(m, levels) -> np.ndarray:
    """Index of the level nearest to each m in log2 (ties: the smaller level)."""
    lv = np.log2(np.asarray(levels, np.float64))
    x = np.log2(np.maximum(np.asarray(m, np.float64), 1.0))
    d = np.abs(x[:, None] - lv[None, :])
    return np.argmin(d, axis=1).astype(np.int8)


def own_rows(lb: "dagrt.LoadedBatch", sched: dict, node_off: np.ndarray):
    """For every node, the global index of its own plan row (row_id == node)."""
    nd = lb.n_dags
    V = np.diff(node_off)
    n_rows = sched["n_rows"][:nd]
    dag = np.repeat(np.arange(nd), 2 * V)
    local = np.arange(2 * int(node_off[-1])) - 2 * node_off[dag]
    rid = sched["row_id"][:2 * int(node_off[-1])]
    ok = (local < n_rows[dag]) & (rid >= 0) & (rid < V[dag])
    rows = np.nonzero(ok)[0]
    owner = node_off[dag[rows]] + rid[rows]
    out = np.full(int(node_off[-1]), -1, np.int64)
    out[owner] = rows
    return out


def search_labels(ctx: "dagrt.Context", batch, levels=LEARN_LEVELS, seed: int = 1):
    """Per-node labels from the plain search's winner (see the module docstring).
    Returns (labels int8 [N], search result dict)."""
    lb = ctx.load(batch)
    scheds = {}
    for v in SEARCH_VARIANTS:
        scheds[v] = lb.schedule(v, fields=("status", "n_rows", "row_id", "row_m0"), check=False)
    res = lb.search(list(SEARCH_VARIANTS), SEARCH_ALLOC, list(SEARCH_LEVELS), seed, want_m=True, mode=SEARCH_MODE)
    node_off = np.asarray(batch.node_off, np.int64)
    N = int(node_off[-1])
    V = np.diff(node_off)
    win_var = np.asarray(SEARCH_VARIANTS)[res["best_cand"] // SEARCH_ALLOC]
    labels = np.full(N, -1, np.int8)
    node_dag = np.repeat(np.arange(lb.n_dags), V)
    for v in SEARCH_VARIANTS:
        sel = (win_var == v) & (scheds[v]["status"][:lb.n_dags] == 0) & (res["best_cand"] >= 0)
        if not sel.any():
            continue
        rows = own_rows(lb, scheds[v], node_off)
        nodes = np.nonzero(sel[node_dag] & (rows >= 0))[0]
        r = rows[nodes]
        m = res["best_m"][r].astype(np.int64)
        m = np.where(m == 0, scheds[v]["row_m0"][r], m)
        labels[nodes] = nearest_level(m, levels)
    lb.free()
    return labels, res


def exhaustive_labels(ctx: "dagrt.Context", batch, levels, v_max: int):
    """Per-node labels from the exhaustive search of the paper structure (dagrt_search,
    DAGRT_SEARCH_EXHAUSTIVE: every node's SMs from {the schedule's own} + levels, all
    combinations): the index in `levels` of the SMs the optimum gives the node's own plan
    row (the schedule's own m when the optimum keeps it; nearest level in log2 if that m is
    not a level). Needs (len(levels) + 1)^v_max <= 2^20 and DAGs of at most v_max nodes.
    Returns (labels int8 [N], loaded batch, paper bound per DAG, optimum per DAG)."""
    lb = ctx.load(batch)
    s = lb.schedule(dagrt.VAR_PAPER, fields=("status", "bound", "n_rows", "row_id", "row_m0"))
    n_alloc = (len(levels) + 1) ** v_max
    res = lb.search([dagrt.VAR_PAPER], n_alloc, list(levels), mode=dagrt.SEARCH_EXHAUSTIVE, want_m=True)
    node_off = np.asarray(batch.node_off, np.int64)
    V = np.diff(node_off)
    rows = own_rows(lb, s, node_off)
    labels = np.full(int(node_off[-1]), -1, np.int8)
    ok = np.repeat(s["status"][:lb.n_dags] == 0, V) & (rows >= 0)
    r = rows[ok]
    m = res["best_m"][r].astype(np.int64)
    m = np.where(m == 0, s["row_m0"][r], m)
    labels[ok] = nearest_level(m, levels)
    return labels, lb, s["bound"][:lb.n_dags], res["best_bound"]


def train(ctx, model: "dagrt.Model", data, epochs: int, lr: float, log=None):
    """data: list of (LoadedBatch, labels). One train step per batch per epoch; returns the
    loss of every step."""
    losses = []
    t0 = time.time()
    for ep in range(epochs):
        for lb, labels in data:
            losses.append(model.train_step(lb, labels, lr))
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {np.mean(losses[-len(data):]):.4f} ({time.time() - t0:.1f} s)")
    return losses


def save(model: "dagrt.Model", path: str, **meta):
    state, step = model.state()
    np.savez(path, state=state, step=step, levels=model.levels, **meta)


def load(ctx, path: str) -> "dagrt.Model":
    z = np.load(path)
    m = dagrt.Model(ctx, z["levels"], seed=0)
    m.set_state(z["state"], int(z["step"]))
    return m


def timed_compare(ctx, model: "dagrt.Model", dev_batch: dict, M: int, k: int = 16, seed: int = 3,
                  reps: int = 3):
    """Wall time on the GPU (CUDA events on the context's stream) of
      plain:   the 4 structure variants' schedules + dagrt_search (4 x 64 perturbation candidates), and
      learned: dagrt_propose (paper schedule, features, network, top-k decode, exact check
               of the paper's allocation and the k proposals),
    each on a freshly loaded copy of the same device-resident batch (the load itself is not
    timed), after one warm-up.
    Returns per-DAG best bounds of both and the median times in ms."""
    import torch
    st = torch.cuda.current_stream()
    nd = int(dev_batch["node_off"].shape[0]) - 1
    outs = {}

    def plain(lb):
        for v in SEARCH_VARIANTS:
            lb.schedule(v, out={"status": torch.empty(nd, dtype=torch.int32, device="cuda")})
        o = {"best_bound": torch.empty(nd, dtype=torch.int64, device="cuda"),
             "best_cand": torch.empty(nd, dtype=torch.int32, device="cuda")}
        lb.search(list(SEARCH_VARIANTS), SEARCH_ALLOC, list(SEARCH_LEVELS), seed, out=o, mode=SEARCH_MODE)
        return o

    def learned(lb):
        o = {"best_bound": torch.empty(nd, dtype=torch.int64, device="cuda"),
             "best_cand": torch.empty(nd, dtype=torch.int32, device="cuda")}
        model.propose(lb, k, out=o)
        return o

    times = {"plain": [], "learned": []}
    for name, fn in (("plain", plain), ("learned", learned)):
        for r in range(reps + 1):
            lb = ctx.load(dev_batch, M)  # loading is common to both and not timed
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            o = fn(lb)
            e1.record(st)
            torch.cuda.synchronize()
            if r > 0:
                times[name].append(e0.elapsed_time(e1))
            outs[name] = {kk: t.cpu().numpy() for kk, t in o.items()}
            lb.free()
    return outs, {k2: float(np.median(v)) for k2, v in times.items()}
