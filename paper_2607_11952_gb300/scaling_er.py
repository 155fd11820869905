"""Scaling sweep on Erdos-Renyi pairs (the paper's synthetic scalability
workload: average degree 10, n from 10k to 110k), BF16 form, one GPU.

  python -m paper_2607_11952_gb300.scaling_er [--sizes 10000,20000,...] [--out file.jsonl]

For every n: a seeded pair (G2 a permuted copy of G1 with 10% of edges
deleted and as many added, 64-dim attributes with sigma = 0.1, 5% anchors),
then Phase 1 (fa_node_cost), one outer iteration (fa_align_iter) and a
fixed number of Sinkhorn sweeps, each timed with CUDA events on the
launching stream.  Prints one JSON line per size with the times, the
sweep's algorithmic bandwidth (one read of K per sweep) and its fraction
of the measured HBM copy peak.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import torch

from . import _lib as L
from . import api, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _peak_gbs() -> float:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                v = d[k]
                return float(v["value"] if isinstance(v, dict) else v)
    except Exception:
        pass
    return 6800.0


def _timed(fn, stream):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    out = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b), out


def run_size(n: int, sweeps: int, dtype: str = "bf16", seed: int = 17) -> dict:
    rng = synth.rng_for(seed + n)
    e1 = synth.erdos_renyi(n, 10.0, rng)
    g = synth.make_pair(e1, n, d=64, sigma=0.1, anchor_frac=0.05, frac_del=0.10,
                        frac_add=0.10, rng=rng, name=f"er{n}", seed=seed)
    al = api.Aligner(api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2),
                     api.Params(dtype=dtype))
    stream = torch.cuda.current_stream()
    X1 = torch.from_numpy(g.X1).cuda()
    X2 = torch.from_numpy(g.X2).cuda()
    try:
        t_p1, _ = _timed(lambda: al.node_cost(X1, X2, g.anchors), stream)
        al.plan_init()
        t_ai, _ = _timed(al.align_iter, stream)
        al.sinkhorn(3)                                      # warm-up
        t_sk, (it, err, st) = _timed(lambda: al.sinkhorn(sweeps), stream)
        al.set_timing(True)
        al.sinkhorn(sweeps)
        ms_sweep, _ = al.last_sweep_ms()
        b = 2 if dtype == "bf16" else 4
        gbs = g.n1 * g.n2 * b / (ms_sweep * 1e-3) / 1e9
        peak = _peak_gbs()
        return {"n": n, "dtype": dtype, "nnz1": int(2 * g.edges1.shape[0]),
                "phase1_ms": round(t_p1, 2), "outer_iteration_ms": round(t_ai, 2),
                "sinkhorn_ms_per_iteration": round(t_sk / sweeps, 4),
                "sweep_kernel_ms": round(ms_sweep, 4), "sweep_GBs": round(gbs, 1),
                "sweep_frac_of_measured_peak": round(gbs / peak, 4),
                "torch_bytes": int(torch.cuda.max_memory_allocated()),
                "workspace_bytes": int(L.fa_ctx_workspace_bytes(al.ctx))}
    finally:
        al.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="10000,20000,30000,40000,50000,60000,70000,80000,"
                                       "90000,100000,110000")
    ap.add_argument("--sweeps", type=int, default=30)
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "f32"])
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    import __graft_entry__  # noqa: F401  (in-tree build)
    __graft_entry__.build()
    f = open(a.out, "w") if a.out else None
    for n in [int(x) for x in a.sizes.split(",")]:
        t0 = time.time()
        r = run_size(n, a.sweeps, a.dtype)
        r["wall_s"] = round(time.time() - t0, 1)
        line = json.dumps(r)
        print(line, flush=True)
        if f:
            f.write(line + "\n")
            f.flush()
        torch.cuda.empty_cache()
    if f:
        f.close()


if __name__ == "__main__":
    main()
