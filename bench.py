#!/usr/bin/env python
"""Benchmark: exact makespan-bound evaluations per second on GB300.

Workload (one step): the 10,000-DAG batch -- Erdos-Renyi DAGs of 20-200 nodes, edge
probability 0.1, log-uniform WCETs in [1, 10^4) ticks, parallel fractions U[0.3, 1] in
1/64 steps, M = 148 SMs -- loaded through dagrt_load_csr from device-resident arrays and
scheduled with dagrt_schedule (validation, Kahn levels, ancestor closure and W^anc,
Theta and blocks, Alg.1 groups, Alg.2 scheduling, Theorem-1 bound), one exact bound per
DAG. `value` = DAG bounds per second over all ranks; `e2e` repeats the step through the
same C ABI from pinned host buffers, host<->device copies included.

Rank layout (torchrun): one batch of N x 10,000 DAGs is split over the N ranks, balanced by
node count (weak scaling: about 10,000 DAGs per GPU); each rank generates, loads and
schedules only its own DAGs, with no collective on the data path. The timed region is
bracketed by a barrier and a device synchronize, the slowest rank's time is reported, and
the per-DAG bounds are gathered on rank 0 afterwards.

--impl reference times the CPU oracle (the only reference this method has: the paper ships
no code) on a bounded sample of the same workload, on the host cores of rank 0.
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact makespan-bound evals/s"
UNIT = "evals/s"
WORKLOAD = ("10,000 Erdos-Renyi DAGs, 20-200 nodes, edge prob 0.1, log-uniform WCET [1,1e4) "
            "ticks, parallel fraction U[0.3,1] in 1/64 steps, M=148; paper schedule + exact "
            "Theorem-1 bound per DAG")


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="dagrt", choices=["dagrt", "reference"])
    p.add_argument("--workload", default="cfg2", choices=["cfg2", "cfg3-bound", "cfg4-learned", "cfg5"],
                   help="cfg2: the headline step; cfg3-bound: candidate bounds of config 3; "
                        "cfg4-learned: learned proposal + exact check vs plain search; "
                        "cfg5: large layered DAGs, paper schedule + bound and top-16 + check")
    p.add_argument("--train-dags", type=int, default=50000, help="cfg4-learned: training DAGs")
    p.add_argument("--epochs", type=int, default=8, help="cfg4-learned: training epochs")
    p.add_argument("--eval-dags", type=int, default=10000,
                   help="cfg4-learned: evaluation DAGs (smaller cases for profiling)")
    p.add_argument("--cpu-seconds", type=float, default=10.0,
                   help="bounded CPU work of the oracle baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-cfg3", action="store_true", help="skip the config-3 candidate-bound keys")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank floats over all ranks (the slowest rank's time);
    `dist` is None on a single rank."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic(kernel: str, source: str, key: str = "bytes_per_launch"):
    """DRAM bytes (or another counter, `key`) per launch from the committed ncu capture, or
    None when the kernel's source changed since the capture (profiles/traffic.json records
    its sha256)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, "paper_2602_20826_gb300", "csrc", source), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        return rec[key] if rec["source_sha256"] == sha else None
    except Exception:
        return None


def issue_roofline(warp_inst, seconds: float, clk: dict):
    """Instruction-issue roofline of a call: its warp instructions (ncu count of the same
    code, from profiles/traffic.json) per second against the GPU's issue peak, SMs x 4
    schedulers x one warp instruction per cycle x the median SM clock sampled during the
    timed region. None without a valid count or clock."""
    import torch
    mhz = (clk or {}).get("sm_mhz")
    if not warp_inst or not mhz:
        return None
    peak = torch.cuda.get_device_properties(0).multi_processor_count * 4 * mhz * 1e6
    return {"achieved": warp_inst / seconds, "peak": peak, "unit": "warp instructions/s",
            "frac": warp_inst / seconds / peak, "warp_instructions_per_call": warp_inst}


def measure_cfg3_bound(args, ctx):
    """Candidate bounds of config 3: 1,000 DAGs x (4 variants x 64 allocations from
    {1,...,32}, allocation 0 = the schedule's own), materialised in HBM, argmin per DAG.
    One dagrt_bound call per step, CUDA events on the launching stream, L2 flushed between
    steps; e2e repeats the call with host buffers. Returns the measurement record."""
    import torch
    from paper_2602_20826_gb300 import workloads as wl
    b = wl.config(3)
    stream = torch.cuda.current_stream()
    lb = ctx.load(b)
    rows = 0
    for v in range(4):
        rows += int(lb.schedule(v, fields=("n_rows",))["n_rows"].sum())
    alloc, stride = wl.candidate_allocations(b, 4, 64, [1, 2, 4, 8, 16, 32], seed=wl.BASE_SEED + 13)
    da = torch.from_numpy(alloc).cuda()
    nd, nc = b.n_dags, 256
    ob = torch.zeros(nd * nc, dtype=torch.int64, device="cuda")
    bb = torch.zeros(nd, dtype=torch.int64, device="cuda")
    bc = torch.zeros(nd, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    steps = max(args.steps, 3)
    # the timed steps take well under a millisecond: the clock sampler (100 ms period)
    # runs from a half-second warm-up through the timed region
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    w, t_hot = 0, time.perf_counter()
    while w < max(args.warmup, 3) or time.perf_counter() - t_hot < 0.5:
        lb.bound([0, 1, 2, 3], 64, da, stride, ob, bb, bc)
        if w % 64 == 63:
            torch.cuda.synchronize()
        w += 1
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    l0 = ctx.launches()
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        lb.bound([0, 1, 2, 3], 64, da, stride, ob, bb, bc)
        e1.record(stream)
    torch.cuda.synchronize()
    launches = (ctx.launches() - l0) // steps
    clk = clocks.stop()
    t = sum(a.elapsed_time(c) for a, c in evs) / 1e3 / steps
    gpu_best = bb.cpu().numpy()
    # end to end: the candidate bytes from pinned host memory, every bound and the argmin
    # back to host memory, through the same C call with host pointers
    ha = torch.from_numpy(alloc).pin_memory().numpy()
    for _ in range(2):
        lb.bound([0, 1, 2, 3], 64, ha, stride)
    t_e2e = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hob, hbb, hbc = lb.bound([0, 1, 2, 3], 64, ha, stride)
        t_e2e.append(time.perf_counter() - t0)
    ok = np.array_equal(hbb, gpu_best) and np.array_equal(hbc, bc.cpu().numpy())
    te = float(np.median(t_e2e))
    lb.free()
    # algorithmic bytes: each variant's candidate bytes of its plan rows once (64 B a row),
    # the DAG data once, one int64 bound per candidate and the argmin per DAG
    peak, kind = _peaks()
    alg = rows * 64 + b.input_bytes() + nd * nc * 8 + nd * 12
    return {"b": b, "alloc": alloc, "stride": stride, "gpu_best": gpu_best, "ok": ok,
            "rec": {"value": nd * nc / t, "unit": UNIT, "us_per_call": 1e6 * t, "steps": steps,
                    "gpu_launches": launches, "clocks": clk,
                    "e2e": {"value": nd * nc / te, "unit": UNIT, "h2d_bytes_per_step": int(alloc.nbytes),
                            "d2h_bytes_per_step": nd * nc * 8 + nd * 12},
                    "roofline": {"bound": "hbm", "achieved": alg / t / 1e9, "peak": peak, "unit": "GB/s",
                                 "frac": alg / t / 1e9 / peak, "traffic": traffic("k_bound_items", "bound.cu"),
                                 "kernel": "dagrt_bound: k_bound_items + k_bound_finish (timed together; "
                                           "traffic is k_bound_items alone)",
                                 "alg_bytes_per_launch": alg,
                                 "alg_bytes": "64 B of candidate bytes per plan row of each variant "
                                              f"({rows} rows) + DAG data once + 8 B per candidate + 12 B per DAG",
                                 "peak_source": f"{kind} hbm_gbs",
                                 "issue": issue_roofline(traffic("k_bound_items", "bound.cu",
                                                                 "warp_instructions_per_call"), t, clk)}}}


def measure_learned_small(ctx):
    """Learned proposal + exact check against the exhaustive allocation search, where the
    paper's Eq.5 allocation leaves room: 2,000 held-out DAGs of 3-6 nodes on an 8-SM GPU
    (exhaustive search of the paper structure: every node's SMs in 1..8, 9^6 = 531,441
    allocations per DAG). The network trains (untimed) on the exhaustive optimum's per-node
    SMs of 12,000 other DAGs. Timed on the GPU (CUDA events), each on a freshly loaded copy:
    plain = the paper schedule + the exhaustive search; learned = dagrt_propose (schedule,
    features, network, top-16, exact check of the paper's allocation and 16 proposals)."""
    import torch
    from paper_2602_20826_gb300 import train as T, workloads as wl
    from paper_2602_20826_gb300.dagrt import SEARCH_EXHAUSTIVE, VAR_PAPER, Model
    levels, vmax = list(range(1, 9)), 6
    t0 = time.perf_counter()
    data = []
    for c in range(4):
        lab, lb, _, _ = T.exhaustive_labels(ctx, wl.small_m_batch(3000, 700 + c), levels, vmax)
        data.append((lb, lab))
    t_lab = time.perf_counter() - t0
    ho = wl.small_m_batch(2000, 799)
    lab_ho, lho, paper, opt = T.exhaustive_labels(ctx, ho, levels, vmax)
    lho.free()
    res = {}
    stream = torch.cuda.current_stream()
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    keys = ("node_off", "edge_off", "row_ptr", "col", "wcet", "k64")
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(ho, k))).cuda() for k in keys}
    nd = ho.n_dags
    for name, epochs in (("untrained", 0), ("trained", 30)):
        model = Model(ctx, levels, seed=3)
        t1 = time.perf_counter()
        T.train(ctx, model, data, epochs=epochs, lr=3e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t1
        ts = []
        for r in range(4):
            lb = ctx.load(dev, ho.M)
            o = {"best_bound": torch.empty(nd, dtype=torch.int64, device="cuda"),
                 "best_cand": torch.empty(nd, dtype=torch.int32, device="cuda")}
            torch.cuda.synchronize()
            e0, e1 = E(), E()
            e0.record(stream)
            model.propose(lb, 16, out=o)
            e1.record(stream)
            torch.cuda.synchronize()
            if r:
                ts.append(e0.elapsed_time(e1))
            lb.free()
        got = o["best_bound"].cpu().numpy()
        res[name] = {"dags_better_than_paper": float(np.mean(got < paper)),
                     "dags_equal_to_plain": float(np.mean(got == opt)),
                     "mean_gap_to_plain": float(np.mean(got / opt - 1)), "ms": float(np.median(ts)),
                     "train_epochs": epochs, "train_seconds": t_train, "never_worse_than_paper": bool(np.all(got <= paper))}
        model.free()
    ts = []
    for r in range(3):
        lb = ctx.load(dev, ho.M)
        torch.cuda.synchronize()
        e0, e1 = E(), E()
        e0.record(stream)
        lb.schedule(VAR_PAPER, out={"status": torch.empty(nd, dtype=torch.int32, device="cuda")})
        lb.search([VAR_PAPER], 9 ** vmax, levels, mode=SEARCH_EXHAUSTIVE,
                  out={"best_bound": torch.empty(nd, dtype=torch.int64, device="cuda")})
        e1.record(stream)
        torch.cuda.synchronize()
        if r:
            ts.append(e0.elapsed_time(e1))
        lb.free()
    for lb, _ in data:
        lb.free()
    plain_ms = float(np.median(ts))
    return {"workload": "2,000 held-out DAGs of 3-6 nodes (ER p=0.35, loads U[1,40], f U[0.5,1]), M=8; plain "
                        "= exhaustive search of the paper structure (9^6 allocations per DAG); learned = top-16 "
                        "+ exact check, trained on the exhaustive optimum of 12,000 other DAGs",
            "dags_plain_better_than_paper": float(np.mean(opt < paper)), "plain_ms": plain_ms,
            "learned": res["trained"], "untrained": res["untrained"],
            "speedup_vs_plain": plain_ms / res["trained"]["ms"], "label_seconds": t_lab}


def run_cfg3_bound(args):
    import torch
    from paper_2602_20826_gb300.dagrt import Context
    torch.cuda.set_device(0)
    ctx = Context(0, torch.cuda.current_stream().cuda_stream)
    m = measure_cfg3_bound(args, ctx)
    r = m["rec"]
    nd = m["b"].n_dags
    line = {"metric": "exact candidate-bound evals/s", "value": r["value"], "unit": UNIT, "n_gpus": 1,
            "steps": r["steps"], "warmup": args.warmup, "ms_per_step": r["us_per_call"] / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": "config 3: 1,000 ER DAGs 50-500 nodes p=0.05, M=148, 4 variants x 64 "
                                   "allocations from {1..32} materialised in HBM, argmin per DAG",
                       "n_dags": nd, "l2": "flushed between steps (256 MB write)"},
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"], "e2e": r["e2e"],
            "roofline": r["roofline"], "status_ok": m["ok"]}
    print(json.dumps(line), flush=True)


def run_cfg4_learned(args):
    """Learned proposal + exact check against the plain search, config 4.

    Training (untimed): the plain search labels 50,000 DAGs of config 2's distribution;
    the network trains on them with the library's own forward/backward kernels. Timed: on
    10,000 fresh DAGs of 100-1,000 nodes (p = 0.05, M = 148), the plain search (4
    structure-variant schedules + 4 x 64 generated allocations: each schedule's own and 63
    sparse perturbations of it, exact bounds, argmin) against dagrt_propose (paper schedule, features, network, top-16 decode, exact
    check of the paper's allocation and the 16 proposals), each from a freshly loaded
    device-resident batch. `value` is the learned path's time; the line also carries the
    plain search's time and the gap between their best bounds."""
    import torch
    import oracle
    from paper_2602_20826_gb300 import train as T, workloads as wl
    from paper_2602_20826_gb300.dagrt import Context, Model
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = Context(0, stream.cuda_stream)
    t0 = time.perf_counter()
    data, n_nodes, chunk = [], 0, 10000
    for c0 in range(0, args.train_dags, chunk):
        b = wl.er_batch(min(chunk, args.train_dags - c0), 20, 200, 0.1, 148, wl.BASE_SEED + 400 + c0,
                        name="cfg2-train")
        labels, _ = T.search_labels(ctx, b, seed=wl.BASE_SEED + 41 + c0)
        data.append((ctx.load(b), labels))
        n_nodes += b.total_nodes()
    t_lab = time.perf_counter() - t0
    model = Model(ctx, T.LEARN_LEVELS, seed=wl.BASE_SEED)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = T.train(ctx, model, data, args.epochs, 2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    for lb, _ in data:
        lb.free()
    del data
    be = wl.config(4, n_dags=args.eval_dags)
    keys = ("node_off", "edge_off", "row_ptr", "col", "wcet", "k64")
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(be, k))).cuda() for k in keys}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    l0 = ctx.launches()
    reps = max(1, min(args.steps, 5))
    outs, times = T.timed_compare(ctx, model, dev, be.M, k=16, seed=wl.BASE_SEED + 43, reps=reps)
    launches = (ctx.launches() - l0) // (2 * (reps + 1))
    clk = clocks.stop()
    pb, lbest = outs["plain"]["best_bound"].astype(np.int64), outs["learned"]["best_bound"].astype(np.int64)
    # forward-pass throughput on the eval batch (features cached by the calls above)
    lb = ctx.load(dev, be.M)
    zbuf = torch.empty(be.total_nodes() * len(T.LEARN_LEVELS), dtype=torch.float32, device="cuda")
    model.logits(lb, out=zbuf)
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    fw = []
    for _ in range(reps + 1):
        e0, e1 = E(), E()
        e0.record(stream)
        model.logits(lb, out=zbuf)
        e1.record(stream)
        torch.cuda.synchronize()
        fw.append(e0.elapsed_time(e1))
    t_fw = float(np.median(fw[1:])) / 1e3
    paper = lb.schedule(0, fields=("bound",))["bound"]
    lb.free()
    N = be.total_nodes()
    flops = 2.0 * N * (48 * 128 + 2 * 384 * 128 + 128 * len(T.LEARN_LEVELS))
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        tf_peak = float(json.load(f)["bf16_tflops"])
    # end to end: host arrays in, host bests out, through the same C ABI
    e2e = []
    for _ in range(reps + 1):
        torch.cuda.synchronize()
        ta = time.perf_counter()
        lbh = ctx.load(be)
        r = model.propose(lbh, 16)
        lbh.free()
        e2e.append(time.perf_counter() - ta)
    t_e2e = float(np.median(e2e[1:]))
    # the oracle's plain search on a sample of the eval DAGs (single thread)
    ts = time.perf_counter()
    ns = 0
    while time.perf_counter() - ts < args.cpu_seconds:
        oracle.search_dag_generated(be, ns, list(T.SEARCH_VARIANTS), T.SEARCH_ALLOC, list(T.SEARCH_LEVELS),
                                    wl.BASE_SEED + 43, T.SEARCH_MODE)
        ns += 1
    cpu_ms = (time.perf_counter() - ts) / ns * be.n_dags * 1e3
    gap = float(lbest.sum() / pb.sum() - 1.0)
    line = {"metric": "learned-vs-plain search time at equal bound", "value": times["learned"], "unit": "ms",
            "n_gpus": 1, "steps": reps, "warmup": 1, "ms_per_step": times["learned"], "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16/fp32 network, int64 bounds", "data": "synthetic",
            "plain_ms": times["plain"], "speedup_vs_plain": times["plain"] / times["learned"],
            "bound_gap_vs_plain": gap, "dags_learned_worse_than_plain": int(np.sum(lbest > pb)),
            "dags_learned_better_than_plain": int(np.sum(lbest < pb)),
            "dags_plain_better_than_paper": int(np.sum(pb < paper)),
            "dags_learned_better_than_paper": int(np.sum(lbest < paper)),
            "training": {"dags": args.train_dags, "nodes": n_nodes, "epochs": args.epochs,
                         "label_seconds": t_lab, "train_seconds": t_train,
                         "first_loss": losses[0], "final_loss": float(np.mean(losses[-len(losses) // args.epochs:])),
                         "labels": "plain-search winner (4 variants x 64 perturbation candidates), nearest "
                                   "proposer level"},
            "config": {"workload": f"config 4: {be.n_dags:,} ER DAGs 100-1,000 nodes p=0.05, M=148; learned top-16 + "
                                   "exact check vs plain search (4 variants x 64 allocations: the schedule's own "
                                   "and sparse perturbations of it)",
                       "n_dags": be.n_dags, "nodes": N, "edges": be.total_edges(),
                       "levels": list(T.LEARN_LEVELS), "l2": "inputs 0.6 GB > L2"},
            "e2e": {"value": 1e3 * t_e2e, "unit": "ms", "h2d_bytes_per_step": be.input_bytes(),
                    "d2h_bytes_per_step": 12 * be.n_dags},
            "gpu_launches": launches,
            "roofline": {"bound": "tensor", "achieved": flops / t_fw / 1e12, "peak": tf_peak, "unit": "TFLOP/s",
                         "frac": flops / t_fw / 1e12 / tf_peak, "traffic": None,
                         "kernel": "network forward (3 k_gnn_fwd layers + head), dagrt_model_logits",
                         "flops_per_launch": flops, "kernel_ms": 1e3 * t_fw,
                         "peak_source": "measured bf16_tflops (burst)"},
            "clocks": clk,
            "cpu_baseline": {"value": cpu_ms, "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": f"plain search (4 schedules + 256 bounds per DAG) on the first {ns} "
                                       f"eval DAGs, single thread, scaled to {be.n_dags} DAGs"}}
    print(json.dumps(line), flush=True)


def run_cfg5(args):
    """Config 5: 200 layered DAGs of 2,000-20,000 nodes. One step = the paper schedule and
    its bound for every DAG (dagrt_load_csr from device-resident arrays + dagrt_schedule);
    the line also times dagrt_propose (top-16 + exact check, an untrained network: the
    time, not the proposals, is measured) on a freshly loaded copy."""
    import torch
    import oracle
    from paper_2602_20826_gb300 import workloads as wl
    from paper_2602_20826_gb300.dagrt import Context, Model
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = Context(0, stream.cuda_stream)
    b = wl.config(5)
    keys = ("node_off", "edge_off", "row_ptr", "col", "wcet", "k64")
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(b, k))).cuda() for k in keys}
    nd = b.n_dags
    out = {"bound": torch.zeros(nd, dtype=torch.int64, device="cuda"),
           "status": torch.zeros(nd, dtype=torch.int32, device="cuda")}
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    steps = max(1, min(args.steps, 5))

    def step():
        lb = ctx.load(dev, M=b.M)
        lb.schedule(0, out=out)
        lb.free()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # > L2 (129 MB)
    warm = max(3, args.warmup)
    for _ in range(warm):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    l0 = ctx.launches()
    evs = [(E(), E()) for _ in range(steps)]
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    launches = (ctx.launches() - l0) // steps
    t = sum(a.elapsed_time(c) for a, c in evs) / 1e3 / steps
    model = Model(ctx, [1, 2, 4, 8, 16, 32, 64, 148], seed=wl.BASE_SEED)
    po = {"best_bound": torch.zeros(nd, dtype=torch.int64, device="cuda"),
          "best_cand": torch.zeros(nd, dtype=torch.int32, device="cuda")}
    pt = []
    for r in range(3):
        lb = ctx.load(dev, M=b.M)
        torch.cuda.synchronize()
        e0, e1 = E(), E()
        e0.record(stream)
        model.propose(lb, 16, out=po)
        e1.record(stream)
        torch.cuda.synchronize()
        if r:
            pt.append(e0.elapsed_time(e1))
        lb.free()
    clk = clocks.stop()
    ok = bool((out["status"] == 0).all().item()) and bool((po["best_bound"] <= out["bound"]).all().item())
    gpu_bounds = out["bound"].cpu().numpy()
    # the oracle on the first DAGs (about args.cpu_seconds of work), parity included
    ts = time.perf_counter()
    ns = 0
    while time.perf_counter() - ts < args.cpu_seconds and ns < nd:
        bo, st = oracle.schedule_batch(b, dags=[ns])
        ok = ok and int(bo[0]) == int(gpu_bounds[ns])
        ns += 1
    cpu_v = ns / (time.perf_counter() - ts)
    peak, kind = _peaks()
    alg = b.input_bytes() + 12 * nd
    line = {"metric": METRIC, "value": nd / t, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warm,
            "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": "config 5: 200 layered DAGs, 2,000-20,000 nodes, depth 20-60, widths 1-64 "
                                   "scaled to V, skip edges p=0.02, lognormal WCET, M=148",
                       "n_dags": nd, "nodes": b.total_nodes(), "edges": b.total_edges(),
                       "l2": "flushed between steps (256 MB write)"},
            "propose_top16_ms": float(np.median(pt)), "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": alg / t / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / t / 1e9 / peak, "traffic": None,
                         "kernel": "dagrt_schedule (CTA teams, global workspaces)", "alg_bytes_per_launch": alg,
                         "peak_source": f"{kind} hbm_gbs"},
            "clocks": clk, "status_ok": ok,
            "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {ns} DAGs of the batch, single thread, parity checked"}}
    print(json.dumps(line), flush=True)


def oracle_rate(batch, seconds: float, threads: int, gpu_bounds=None, chunk: int = 64):
    """DAG schedules + bounds per second of the oracle as it stands, over whole passes of the
    batch's DAGs in order for about `seconds`, with `threads` host threads taking chunks of
    DAGs in turn (the oracle's C call releases the GIL and reads the batch in place). Checks
    the GPU bounds of every DAG it ran in its first pass."""
    import threading
    import oracle
    n = batch.n_dags
    lock = threading.Lock()
    st = {"next": 0, "done": 0, "mism": 0, "checked": 0}
    t0 = time.perf_counter()

    def worker():
        while True:
            with lock:
                if st["next"] >= chunk * threads and time.perf_counter() - t0 >= seconds:
                    return
                lo = st["next"] % n
                hi = min(lo + chunk, n)
                first = st["next"] < n
                st["next"] += hi - lo
            bo, _ = oracle.schedule_range(batch, lo, hi)
            with lock:
                st["done"] += hi - lo
                if gpu_bounds is not None and first:
                    st["mism"] += int(np.sum(bo != gpu_bounds[lo:hi]))
                    st["checked"] += hi - lo

    ts = [threading.Thread(target=worker) for _ in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    dt = time.perf_counter() - t0
    return {"value": st["done"] / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{st['done']} DAG schedules+bounds of the same batch (passes over its DAGs in "
                      f"order), plain-C oracle, {threads} host thread(s), {dt:.1f} s",
            "parity_checked_dags": st["checked"], "parity_mismatches": st["mism"]}


def cpu_baseline(batch, seconds: float, gpu_bounds=None):
    """The oracle on every host core (one thread per core, os.cpu_count()), with the
    single-thread rate beside it; each leg takes about half of `seconds`."""
    one = oracle_rate(batch, seconds / 2, 1, gpu_bounds)
    allc = oracle_rate(batch, seconds / 2, os.cpu_count() or 1, gpu_bounds)
    allc["single_thread"] = {k: one[k] for k in ("value", "cores", "sample")}
    allc["parity_checked_dags"] = max(one["parity_checked_dags"], allc["parity_checked_dags"])
    allc["parity_mismatches"] = one["parity_mismatches"] + allc["parity_mismatches"]
    return allc


def oracle_pass(batch, lo: int, hi: int, threads: int, chunk: int = 64):
    """The oracle on DAGs lo..hi-1 of the batch, `threads` host threads taking chunks of
    DAGs in turn; returns the bounds."""
    import threading
    import oracle
    out = np.zeros(hi - lo, np.int64)
    lock = threading.Lock()
    nxt = [lo]

    def worker():
        while True:
            with lock:
                a = nxt[0]
                nxt[0] = min(hi, a + chunk)
            if a >= hi:
                return
            b = min(hi, a + chunk)
            out[a - lo:b - lo] = oracle.schedule_range(batch, a, b)[0]

    ts = [threading.Thread(target=worker) for _ in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return out


def run_reference(args, rank, world):
    """The oracle (the paper ships no code) on the host cores of rank 0, one thread per
    core, each step a bounded sample of the same batch."""
    from paper_2602_20826_gb300 import workloads as wl
    if rank != 0:
        return
    batch = wl.config(2)
    import oracle
    oracle.lib()
    cores = os.cpu_count() or 1
    per_step = min(batch.n_dags, 250 * cores)  # DAGs per step: ~0.3 s of oracle work per core
    for _ in range(args.warmup):
        oracle_pass(batch, 0, min(per_step, 64 * cores), cores)
    t0 = time.perf_counter()
    for s in range(args.steps):
        lo = (s * per_step) % batch.n_dags
        oracle_pass(batch, lo, min(batch.n_dags, lo + per_step), cores)
    dt = time.perf_counter() - t0
    done = sum(min(batch.n_dags, (s * per_step) % batch.n_dags + per_step) - (s * per_step) % batch.n_dags
               for s in range(args.steps))
    val = done / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_dags": batch.n_dags, "M": batch.M,
                       "reference_step": f"{per_step} DAGs of the batch per step on {cores} host threads"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} DAGs per step x {args.steps} steps, one thread per host core"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "cfg3-bound":
        run_cfg3_bound(args)
        return
    if args.workload == "cfg4-learned":
        run_cfg4_learned(args)
        return
    if args.workload == "cfg5":
        run_cfg5(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    import numpy as np
    import torch
    from paper_2602_20826_gb300 import workloads as wl
    from paper_2602_20826_gb300.dagrt import Context

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    # one batch of world x 10,000 DAGs, sharded over the ranks by node count (LPT); every
    # rank generates and schedules only its own DAGs (weak scaling: ~10,000 per GPU)
    n_global = 10000 * world
    parts = None
    if world > 1:
        from paper_2602_20826_gb300 import shard
        parts = shard.partition(wl.er_sizes(n_global, 20, 200, wl.BASE_SEED + 2), world)
        batch = wl.config(2, ids=parts[rank])
    else:
        batch = wl.config(2)
    stream = torch.cuda.current_stream()
    ctx = Context(local, stream.cuda_stream)
    keys = ("node_off", "edge_off", "row_ptr", "col", "wcet", "k64")
    dev = {k: torch.from_numpy(getattr(batch, k)).cuda() for k in keys}
    nd = batch.n_dags
    out = {"bound": torch.zeros(nd, dtype=torch.int64, device="cuda"),
           "status": torch.zeros(nd, dtype=torch.int32, device="cuda")}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # > L2 (129 MB)

    def step(evs=None):
        lb = ctx.load(dev, M=batch.M)
        if evs is not None:
            evs[0].record(stream)
        lb.schedule(0, out=out)
        if evs is not None:
            evs[1].record(stream)
        lb.free()

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    step_ev = [(E(), E()) for _ in range(args.steps)]
    kern_ev = [(E(), E()) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    l0 = ctx.launches()
    for s in range(args.steps):
        flush.zero_()
        step_ev[s][0].record(stream)
        step(kern_ev[s])
        step_ev[s][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = ctx.launches() - l0
    clk = clocks.stop()
    t_step = sum(a.elapsed_time(b) for a, b in step_ev) / 1e3  # seconds, K steps
    t_kern = sum(a.elapsed_time(b) for a, b in kern_ev) / 1e3
    t_step, t_kern = max_over_ranks([t_step, t_kern], dist, "cuda")
    ok = bool((out["status"] == 0).all().item())
    gpu_bounds = out["bound"].cpu().numpy()
    if dist is not None:  # after the timed region: the per-DAG bounds of all shards on rank 0
        from paper_2602_20826_gb300 import shard
        allb = shard.gather_over_ranks(dist, parts, gpu_bounds, n_global)
        if rank == 0:
            ok = ok and bool((allb >= 0).all())

    # the same schedule call captured once into a CUDA graph and replayed on a resident
    # batch (the size-class partition of dagrt_load_csr is not repeated per step)
    lbg = ctx.load(dev, M=batch.M)
    lbg.schedule(0, out=out)
    torch.cuda.synchronize()
    ctx.graph_begin()
    lbg.schedule(0, out=out)
    graph = ctx.graph_end()
    for _ in range(args.warmup):
        flush.zero_()
        graph.launch()
    g_ev = [(E(), E()) for _ in range(args.steps)]
    for s_ in range(args.steps):
        flush.zero_()
        g_ev[s_][0].record(stream)
        graph.launch()
        g_ev[s_][1].record(stream)
    torch.cuda.synchronize()
    t_graph = max_over_ranks([sum(a.elapsed_time(b) for a, b in g_ev) / 1e3], dist, "cuda")[0]
    ok = ok and bool((out["status"] == 0).all().item()) and np.array_equal(out["bound"].cpu().numpy(), gpu_bounds)
    graph.free()
    lbg.free()

    # end to end through the C ABI from pinned host buffers (copies in the timed region)
    host = {k: torch.from_numpy(getattr(batch, k)).pin_memory() for k in keys}
    h2d = sum(int(t.numel() * t.element_size()) for t in host.values()) + 4 * nd  # + size-class lists
    d2h = 8 * nd + 4 * nd + 4 * nd  # bound, status and the call's own status read-back

    def e2e_step():
        lb = ctx.load(host, M=batch.M)
        r = lb.schedule(0, fields=("bound", "status"))
        lb.free()
        return r

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    e2e_sum = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ta = time.perf_counter()
        r = e2e_step()
        e2e_sum += time.perf_counter() - ta
    barrier()
    e2e_sum = max_over_ranks([e2e_sum], dist, "cuda")[0]
    ok = ok and bool((r["status"] == 0).all()) and np.array_equal(r["bound"], gpu_bounds)

    peak, peak_kind = _peaks()
    alg_bytes = batch.input_bytes() + 12 * nd  # inputs read once + bound and status written
    achieved = alg_bytes / (t_kern / args.steps) / 1e9
    n_all = n_global if world > 1 else nd
    line = {
        "metric": METRIC,
        "value": n_all * args.steps / t_step,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_step / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_dags": n_all, "M": batch.M, "nodes": batch.total_nodes(),
                   "edges": batch.total_edges(),
                   "parallelism": (f"{world} shards of one {n_all}-DAG batch balanced by node count (LPT), "
                                   "no collective on the data path; bounds gathered on rank 0 after timing")
                   if world > 1 else "1 GPU",
                   "l2": "flushed between steps (256 MB write); inputs 45 MB < L2"},
        "e2e": {"value": n_all * args.steps / e2e_sum, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "graph_replay": {"value": n_all * args.steps / t_graph, "unit": UNIT,
                         "ms_per_step": 1e3 * t_graph / args.steps,
                         "what": "dagrt_schedule captured in a CUDA graph, replayed on a resident batch"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic("k_sched_warp", "sched.cu"),
                     "kernel": "k_sched_warp (all size classes of one dagrt_schedule call)",
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "alg_bytes_per_launch": alg_bytes, "kernel_ms": 1e3 * t_kern / args.steps},
        "clocks": clk,
        "status_ok": ok,
    }
    line["roofline"]["issue"] = issue_roofline(traffic("k_sched_warp", "sched.cu", "warp_instructions_per_call"),
                                               t_kern / args.steps, clk)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(batch, args.cpu_seconds, gpu_bounds)
    if rank == 0 and world == 1 and not args.no_cfg3:
        # the candidate-bound kernel on config 3, the HBM-roofline part of the path
        m = measure_cfg3_bound(args, ctx)
        import oracle
        b3 = m["b"]
        for d in range(0, b3.n_dags, b3.n_dags // 8):
            _, rb, _ = oracle.search_dag(b3, d, m["alloc"], m["stride"], 4, 64)
            m["ok"] = m["ok"] and int(m["gpu_best"][d]) == rb
        line["learned_vs_plain_small_m"] = measure_learned_small(ctx)
        line["cfg3_bound"] = dict(m["rec"], status_ok=m["ok"],
                                  workload="config 3: 1,000 ER DAGs 50-500 nodes p=0.05, M=148; 4 variants x 64 "
                                           "allocations from {1..32} materialised in HBM (256k exact bounds), "
                                           "argmin per DAG; parity: 8 sampled DAGs against the oracle")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
