"""The paper's large-scale experiment and a schedulability sweep, run through libdagrt.

Normalised makespan (bound / Greedy + unaware) of the proposed bound (Theorem 1 on the
Alg.1 + Alg.2 schedule), Greedy and Graham_para on the paper's synthetic layered DAGs
(depth 5-8, layer widths U[2, P] between a single source and sink, loads of mean 20, fully
parallel kernels), 1,000 DAGs per setting, against M (P = 16), against P (M = 32) and
against the depth (P = 32, M = 32) -- the three sweeps of the Evaluation section -- and
the share of implicit-deadline tasks whose bound meets D = T at normalised utilisation U,
for the paper's schedule, its literal reading and Eq.5 without the repair.

Every number comes from the library's kernels (dagrt_schedule with the baseline outputs,
dagrt_schedulable); their parity with the CPU oracle is a test of the test suite.

    python -m paper_2602_20826_gb300.sweeps [--dags 1000] [--json out.jsonl]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import workloads as wl
from .dagrt import VAR_LITERAL, VAR_NOREPAIR, VAR_PAPER, Context

C_AVG = 20


def _normalised(ctx, b):
    lb = ctx.load(b)
    t0 = time.perf_counter()
    r = lb.schedule(VAR_PAPER, fields=("bound", "status", "greedy", "greedy_unaware", "graham_para"))
    dt = time.perf_counter() - t0
    assert (r["status"] == 0).all()
    ref = r["greedy_unaware"].astype(np.float64)
    out = {"proposed": float(np.mean(r["bound"] / ref)), "greedy": float(np.mean(r["greedy"] / ref)),
           "graham_para": float(np.mean(r["graham_para"] / ref)), "dags": b.n_dags, "call_s": dt}
    out["gap_vs_greedy"] = 1 - out["proposed"] / out["greedy"]
    out["gap_vs_graham_para"] = 1 - out["proposed"] / out["graham_para"]
    lb.free()
    return out


def run(n_dags: int = 1000, seed: int = 20260226):
    import torch
    ctx = Context(0, torch.cuda.current_stream().cuda_stream)
    rows = []
    for M in (4, 8, 16, 32, 64, 128, 256):
        b = wl.paper_layered_batch(n_dags, 16, M, C_AVG, seed + M)
        rows.append(dict(sweep="M", M=M, P=16, depth="5-8", **_normalised(ctx, b)))
    for P in (4, 5, 6, 7, 8, 9, 10):
        b = wl.paper_layered_batch(n_dags, P, 32, C_AVG, seed + 1000 + P)
        rows.append(dict(sweep="P", M=32, P=P, depth="5-8", **_normalised(ctx, b)))
    for D in (4, 8, 16, 32, 64):
        b = wl.paper_layered_batch(n_dags, 32, 32, C_AVG, seed + 2000 + D, D, D)
        rows.append(dict(sweep="depth", M=32, P=32, depth=D, **_normalised(ctx, b)))
    # schedulability of implicit-deadline tasks
    b = wl.paper_layered_batch(n_dags, 16, 32, C_AVG, seed + 3000)
    lb = ctx.load(b)
    variants = {"paper": VAR_PAPER, "literal": VAR_LITERAL, "no_repair": VAR_NOREPAIR}
    for v in variants.values():
        lb.schedule(v, fields=("status",))
    for U in (0.2, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 1.0):
        dl = wl.implicit_deadlines(b, U)
        share = {name: lb.schedulable(v, dl)[1] / b.n_dags for name, v in variants.items()}
        rows.append(dict(sweep="schedulability", M=32, P=16, U=U, **share))
    lb.free()
    ctx.close()
    return rows


def case_study(reps: int = 100, tick_us: float = 10.0, seed: int = 20260226):
    """The case study's comparison on this GPU: per setting (M in {8, 30} SMs, mean load 4
    or 20 ticks), three of the paper's layered DAGs (P = 8) are realised as CUDA graphs
    (dagrt_realise) `reps` times each, with the proposed schedule under group barriers and
    with Greedy; max / average / standard deviation of the measured makespans in ms, and
    Theorem 1's bound (ticks x tick_us) beside them."""
    import torch
    from .dagrt import REALISE_BARRIER, REALISE_GREEDY
    ctx = Context(0, torch.cuda.current_stream().cuda_stream)
    rows = []
    for c_avg in (4, 20):
        for M in (8, 30):
            b = wl.paper_layered_batch(3, 8, M, c_avg, seed + 17 * M + c_avg)
            for d in range(b.n_dags):
                rp, col, w, k = b.dag(d)
                r = {"sweep": "case_study", "M": M, "c_avg": c_avg, "dag": d, "nodes": len(w), "tick_us": tick_us}
                for name, mode in (("proposed", REALISE_BARRIER), ("greedy", REALISE_GREEDY)):
                    ms, bnd = ctx.realise(rp, col, w, k, M, mode, tick_us=tick_us, reps=reps)
                    ms = ms / 1e3
                    r[name] = {"max_ms": float(ms.max()), "avg_ms": float(ms.mean()), "std_ms": float(ms.std()),
                               "bound_ms": bnd * tick_us / 1e3}
                rows.append(r)
    ctx.close()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dags", type=int, default=1000)
    ap.add_argument("--json", default=None)
    ap.add_argument("--case-study", action="store_true", help="realise schedules as CUDA graphs instead")
    args = ap.parse_args()
    if args.case_study:
        rows = case_study()
        for r in rows:
            p, g = r["proposed"], r["greedy"]
            print(f"M={r['M']:>2} C_avg={r['c_avg']:>2} dag {r['dag']} ({r['nodes']} nodes)  proposed "
                  f"{p['max_ms']:.3f}/{p['avg_ms']:.3f}/{p['std_ms']:.4f} ms (bound {p['bound_ms']:.3f})  greedy "
                  f"{g['max_ms']:.3f}/{g['avg_ms']:.3f}/{g['std_ms']:.4f} ms (bound {g['bound_ms']:.3f})")
        if args.json:
            with open(args.json, "w") as f:
                for r in rows:
                    f.write(json.dumps(r) + "\n")
        return
    rows = run(args.dags)
    for r in rows:
        if r["sweep"] == "schedulability":
            print(f"U={r['U']:.1f}  paper {r['paper']:.3f}  literal {r['literal']:.3f}  no_repair {r['no_repair']:.3f}")
        else:
            print(f"{r['sweep']:>5} M={r['M']:>3} P={r['P']:>2} depth={r['depth']!s:>3}  proposed {r['proposed']:.3f}  "
                  f"greedy {r['greedy']:.3f}  graham_para {r['graham_para']:.3f}  gap vs greedy "
                  f"{100 * r['gap_vs_greedy']:5.1f}%  vs graham_para {100 * r['gap_vs_graham_para']:5.1f}%")
    if args.json:
        with open(args.json, "w") as f:
            for r in rows:
                f.write(json.dumps(r) + "\n")


if __name__ == "__main__":
    main()
