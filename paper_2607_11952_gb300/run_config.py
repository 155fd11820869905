"""One timed alignment on a named workload, for the workloads that are not
the benchmark's (the uneven 100k x 80k pair in particular): Phase 1, the
workload's outer iterations with the chosen warm start and Sinkhorn to the
tolerance, then the top-10 read-out and Hits@1/10 and MRR on the test pairs.

  python -m paper_2607_11952_gb300.run_config [--config cl100k] [--dtype bf16]
      [--warm learned|prev|cold] [--outer T] [--budget-s S] [--out file.json]

A short untimed pass (Phase 1 and one outer iteration of 10 sweeps) runs
first on the same context.  The timed run is bracketed by CUDA events on the
launching stream; it stops early, after the outer iteration in which the
wall clock passes --budget-s, and reports how many outer iterations it ran.
Sweep time per launch comes from CUDA events around every sweep launch.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import torch

from . import _lib as L
from . import api, gnn, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p)).get("hbm_gbs", 6782.1)), "measured"
    return 6800.0, "fallback"


def run(config: str, dtype: str, warm: str, outer: int, tol: float, check_every: int,
        max_sweeps: int, budget_s: float) -> dict:
    g = synth.config_pair(config)
    dev = torch.device("cuda", torch.cuda.current_device())
    G1, G2 = api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2)
    al = api.Aligner(G1, G2, api.Params(dtype=dtype), device=dev)
    model = gnn.WarmStartModel.load(gnn.WEIGHTS_PATH, device=dev) if warm == "learned" else None
    X1 = torch.from_numpy(g.X1).to(dev)
    X2 = torch.from_numpy(g.X2).to(dev)
    stream = torch.cuda.current_stream()
    try:
        al.node_cost(X1, X2, g.anchors)                    # untimed pass
        al.plan_init()
        al.align_iter()
        al.sinkhorn(10)
        al.set_timing(True)
        torch.cuda.synchronize()
        launches0 = L.fa_kernel_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        e0.record(stream)
        al.node_cost(X1, X2, g.anchors)
        al.plan_init()
        ws = gnn.WarmStarter(al, warm, model)
        per_outer = []
        for t in range(outer):
            al.align_iter()
            it, err, st, fell_back = ws.solve(max_sweeps, tol, check_every)
            per_outer.append({"sweeps": it, "err": err, "fell_back": fell_back,
                              "sweep_ms": al.last_sweep_ms()[0]})
            if time.perf_counter() - w0 > budget_s:
                break
        al.topk(10)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = L.fa_kernel_launch_count() - launches0
        hits = al.hits_mrr(g.test_pairs)
    finally:
        al.close()
        G1.close()
        G2.close()
    sweeps = sum(r["sweeps"] for r in per_outer)
    avg_sweep = sum(r["sweeps"] * r["sweep_ms"] for r in per_outer) / max(1, sweeps)
    b = 2 if dtype == "bf16" else 4
    gbs = g.n1 * g.n2 * b / (avg_sweep * 1e-3) / 1e9 if avg_sweep > 0 else None
    peak, kind = _peak_gbs()
    return {"config": config, "n1": g.n1, "n2": g.n2, "dtype": dtype, "warm": warm,
            "outer_requested": outer, "outer_done": len(per_outer), "tol": tol,
            "ms": round(ms, 1), "sweeps": sweeps,
            "sweeps_per_outer": [r["sweeps"] for r in per_outer],
            "fallbacks": sum(r["fell_back"] for r in per_outer),
            "avg_sweep_ms": round(avg_sweep, 4),
            "sweep_GBs": round(gbs, 1) if gbs else None,
            "sweep_frac": round(gbs / peak, 4) if gbs else None, "peak_kind": kind,
            "gpu_launches": int(launches), **{k: round(v, 4) for k, v in hits.items()}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="cl100k")
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "f32"])
    ap.add_argument("--warm", default="learned", choices=["learned", "prev", "cold"])
    ap.add_argument("--outer", type=int, default=None)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--check-every", type=int, default=5)
    ap.add_argument("--max-sweeps", type=int, default=5000)
    ap.add_argument("--budget-s", type=float, default=600.0)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    import __graft_entry__
    __graft_entry__.build()
    outer = a.outer if a.outer is not None else synth.CONFIGS[a.config]["outer"]
    r = run(a.config, a.dtype, a.warm, outer, a.tol, a.check_every, a.max_sweeps, a.budget_s)
    line = json.dumps(r)
    print(line, flush=True)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
