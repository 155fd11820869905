"""Benchmark of the GB300 FastAlign hot path (one JSON line on stdout).

Workload: the 50k-node Chung-Lu pair (exponent 2.1, mean degree 10, 15% edge
noise, 128-dim attributes, 5% anchors), seeded synthetic data.  One step is
an alignment with inputs resident in HBM: Phase 1 (RWR, SDDMM,
node-cost GEMM, propagation), then the workload's 30 outer iterations of
Phase 2 (Pass A, Pass B + Gibbs kernel) and Phase 3 (fused Sinkhorn sweeps,
learned warm start, until the L1 marginal error is <= 1e-4, checked every 5
sweeps), then the top-10 read-out.  The metric is the step time (lower is
better); the same alignment in plain FP32 with a cold start is timed once
beside it.  The Gibbs kernel (5 GB in BF16) is far larger than L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--outer T] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the 5k-node pair with the same generator
parameters, Phase 1 plus the first outer iteration) and scales it to the
metric's unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "50k-node time to 1e-4 marginal err, learned+BF16 vs plain FP32; sweep HBM GB/s"

# Sinkhorn iterations the plain method (FP32 storage, cold start) needs on a
# workload, as measured on GB300 by this script's FP32 comparison; the
# reference arm scales the oracle's per-iteration time by it.
PLAIN_SWEEPS = {("cl50k", 30): 61790, ("cl50k", 4): 1190}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6782.1), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def replica_seed(config: str, rank: int) -> int:
    """Rank r of a replicas run aligns its own pair: the workload's seed + r."""
    from paper_2607_11952_gb300 import synth
    return synth.CONFIGS[config]["seed"] + rank


def max_over_ranks(ms: float, world: int, device) -> float:
    """The job's step time: the slowest rank's (all ranks run the same
    number of independent alignments, so the whole job's time per step is
    the maximum)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_11952_gb300 import api, synth
    from paper_2607_11952_gb300 import _lib as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    # independent replicas: rank r aligns its own pair (seed + r)
    g = synth.config_pair(args.config, seed=replica_seed(args.config, rank))
    G1, G2 = api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2)
    params = api.Params(dtype=args.dtype)
    al = api.Aligner(G1, G2, params, device=dev)
    X1 = torch.from_numpy(g.X1).to(dev)
    X2 = torch.from_numpy(g.X2).to(dev)
    stream = torch.cuda.current_stream()

    # the learned warm start (trained weights committed beside the package)
    from paper_2607_11952_gb300 import gnn
    model = None
    if args.warm == "learned":
        if os.path.exists(gnn.WEIGHTS_PATH):
            model = gnn.WarmStartModel.load(gnn.WEIGHTS_PATH, device=dev)
        else:
            args.warm = "cold"

    def step(aligner, record=None, warm="cold"):
        aligner.node_cost(X1, X2, g.anchors)
        aligner.plan_init()
        ws = gnn.WarmStarter(aligner, warm, model if warm == "learned" else None)
        sweeps = 0
        for _ in range(args.outer):
            aligner.align_iter()
            it, err, st, _ = ws.solve(args.max_sweeps, args.tol, args.check_every)
            sweeps += it
            if record is not None:
                record.append((it, err, aligner.last_sweep_ms()[0]))
        idx, score = aligner.topk(10)
        return sweeps

    al.set_timing(True)
    for _ in range(args.warmup):
        step(al, warm=args.warm)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = L.fa_kernel_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    rec = []
    ev0.record(stream)
    total_sweeps = 0
    for _ in range(args.steps):
        total_sweeps += step(al, rec, warm=args.warm)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = L.fa_kernel_launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(ms, world, dev)
    hits = al.hits_mrr(g.test_pairs)

    # dominant kernel: the fused sweep; time per launch from CUDA events
    # recorded around every sweep launch on the call's stream
    bpe = 2 if args.dtype == "bf16" else 4
    timed = [(r[2], r[0]) for r in rec if r[2] > 0]
    avg_sweep = sum(m * w for m, w in timed) / max(1, sum(w for _, w in timed))
    algo_bytes = g.n1 * g.n2 * bpe
    peak, peak_kind = _peaks()
    achieved = algo_bytes / (avg_sweep * 1e-3) / 1e9 if avg_sweep > 0 else None
    traffic = _ncu_traffic(args)

    # plain FP32 cold start on the same pair, for the metric's comparison
    fp32 = None
    if args.compare_fp32 and args.dtype != "f32":
        al32 = api.Aligner(G1, G2, api.Params(dtype="f32"), device=dev)
        al32.set_timing(True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r32 = []
        e0.record(stream)
        sw32 = step(al32, r32)
        e1.record(stream)
        torch.cuda.synchronize()
        fp32 = {"ms_per_step": e0.elapsed_time(e1), "sweeps": sw32,
                "hits@1": al32.hits_mrr(g.test_pairs)["hits@1"],
                "sweep_ms": sum(r[2] * r[0] for r in r32) / max(1, sum(r[0] for r in r32))}
        al32.close()

    # end to end through the public API from host buffers
    e2e = _e2e(args, g, dev, api, model) if args.e2e else None

    cpu = (_cpu_baseline(args, total_sweeps / args.steps)
           if (rank == 0 and world == 1 and args.cpu_baseline) else None)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(ms, 3), "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
            "data": "synthetic (seeded Chung-Lu pair; no dataset)",
            "config": _config(args, world),
            "sweeps_per_step": total_sweeps / args.steps,
            "warm_start": args.warm,
            "hits@1": hits["hits@1"], "mrr": hits["mrr"],
            "plain_fp32_cold": fp32,
            "roofline": {"kernel": "k_sweep", "bound": "hbm",
                         "achieved": round(achieved, 1) if achieved else None,
                         "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4) if achieved else None,
                         "traffic": traffic, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": algo_bytes,
                         "avg_launch_ms": round(avg_sweep, 4)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


SWEEP_SOURCES = ("paper_2607_11952_gb300/csrc/k_sinkhorn.cu",
                 "paper_2607_11952_gb300/csrc/sweep_dev.cuh")


def sweep_source_hash():
    """sha256 of the sweep kernel's source files, stored with the ncu
    counters so a traffic figure is only reported for the kernel it was
    taken from."""
    import hashlib
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


def _ncu_traffic(args):
    """DRAM bytes per k_sweep launch from the committed ncu summary, if it
    was taken for the current kernel source and dtype (None otherwise)."""
    p = os.path.join(ROOT, "profiles", "k_sweep_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha256") != sweep_source_hash():
        return None
    e = d.get(args.dtype)
    return e.get("dram_bytes_per_launch_full_size") if e else None


def _e2e(args, g, dev, api, model):
    """Same step through the public API from host buffers: graph build
    (host CSR + upload), attribute upload from pinned memory, the whole
    alignment with the same warm start and the read-back of the top-10
    indices."""
    from paper_2607_11952_gb300 import gnn
    import numpy as np
    import torch
    X1h = torch.from_numpy(g.X1).pin_memory()
    X2h = torch.from_numpy(g.X2).pin_memory()
    h2d = X1h.numel() * 4 + X2h.numel() * 4 + (g.edges1.size + g.edges2.size) * 4 + g.anchors.size * 4
    times = []
    for k in range(args.e2e_runs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G1, G2 = api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2)
        al = api.Aligner(G1, G2, api.Params(dtype=args.dtype), device=dev)
        X1 = X1h.to(dev, non_blocking=True)
        X2 = X2h.to(dev, non_blocking=True)
        al.node_cost(X1, X2, g.anchors)
        al.plan_init()
        ws = gnn.WarmStarter(al, args.warm, model if args.warm == "learned" else None)
        for _ in range(args.outer):
            al.align_iter()
            ws.solve(args.max_sweeps, args.tol, args.check_every)
        idx, score = al.topk(10)
        out = idx.cpu().numpy()
        torch.cuda.synchronize()
        times.append((time.perf_counter() - t0) * 1e3)
        al.close()
        G1.close()
        G2.close()
    return {"value": round(min(times[1:] or times), 3), "unit": "ms", "runs": len(times),
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(out.nbytes)}


def _cpu_sample(args):
    """The oracle on the 5k-node pair with the workload's generator
    parameters: Phase 1, then Phase 2 of the first outer iteration and its
    Sinkhorn solve to tol, each timed (FP64)."""
    import math
    import numpy as np
    from oracle import fastalign_ref as R
    from paper_2607_11952_gb300 import synth
    g = synth.config_pair(args.config + "_5k" if args.config == "cl50k" else args.config)
    p = R.Params()
    t0 = time.perf_counter()
    ph = R.phase1(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p)
    t1 = time.perf_counter()
    logS = np.full((g.n1, g.n2), -math.log(g.n1 * g.n2))
    C_eff = R.outer_step(ph, logS, p)
    t2 = time.perf_counter()
    mu, nu = np.full(g.n1, 1 / g.n1), np.full(g.n2, 1 / g.n2)
    _, _, _, iters = R.sinkhorn_log(C_eff, mu, nu, p.eps, 100000, tol=args.tol,
                                    check_every=args.check_every)
    t3 = time.perf_counter()
    return g, dict(phase1=(t1 - t0) * 1e3, phase2=(t2 - t1) * 1e3,
                   sweep=(t3 - t2) * 1e3 / max(1, iters), iters=iters)


def _scale(args, g, t, sweeps):
    """Oracle time for the GPU step's work at n = 50k: Phase 1 grows like
    n1 n2 |L| (|L| ~ n), Phase 2 and one Sinkhorn iteration like n1 n2."""
    s2 = (50_000 / g.n1) * (50_000 / g.n2)
    return (t["phase1"] * s2 * (50_000 / g.n1) + t["phase2"] * s2 * args.outer +
            t["sweep"] * s2 * sweeps)


def _cpu_baseline(args, sweeps):
    g, t = _cpu_sample(args)
    return {"value": round(_scale(args, g, t, sweeps), 1), "unit": "ms",
            "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 oracle on the {g.n1}-node pair with the workload's "
                      f"generator parameters: Phase 1 {t['phase1']:.0f} ms, Phase 2 "
                      f"{t['phase2']:.0f} ms, {t['sweep']:.0f} ms per Sinkhorn iteration "
                      f"({t['iters']} iterations to {args.tol:g}); scaled to n=50k "
                      f"(n^3 Phase 1, n^2 per outer iteration and per Sinkhorn "
                      f"iteration) for {args.outer} outer iterations and the "
                      f"{sweeps:.0f} Sinkhorn iterations the GPU step ran; NumPy "
                      f"elementwise work is single-threaded, BLAS uses all cores"}


def _config(args, world):
    """The workload both arms report (same keys and values)."""
    c = _synth_config(args.config)
    n1 = c["n"]
    n2 = c.get("keep") or n1
    return {"workload": f"{args.config}: Chung-Lu n1={n1} n2={n2}, gamma={c['gamma']}, "
                        f"avg deg {c['avg_deg']:g}, {100 * c['frac_del']:g}% edge noise, "
                        f"d={c['d']}, {100 * c['anchor_frac']:g}% anchors; Phase 1 + "
                        f"{args.outer} outer x Sinkhorn to {args.tol:g} (check every "
                        f"{args.check_every}) + top-10",
            "n1": n1, "n2": n2, "outer": args.outer, "tol": args.tol,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": f"inputs larger than L2 (K is {n1 * n2 * (4 if getattr(args, 'dtype', 'bf16') == 'f32' else 2) / 1e9:.1f} "
                  f"GB), no flush"}


def _synth_config(name):
    from paper_2607_11952_gb300 import synth
    return synth.CONFIGS[name]


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    vals = []
    g = t = None
    for k in range(args.warmup + args.steps):
        g, t = _cpu_sample(args)
        if k >= args.warmup:
            vals.append(_scale(args, g, t, args.ref_sweeps))
    v = sum(vals) / len(vals)
    line = {
        "metric": METRIC, "value": round(v, 1), "unit": "ms", "impl": "reference",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Chung-Lu pair; no dataset)",
        "config": _config(args, world),
        "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": f"FP64 oracle, cold start: Phase 1, Phase 2 and Sinkhorn "
                                   f"iterations timed on the n={g.n1} pair with the "
                                   f"workload's generator parameters, scaled to n=50k "
                                   f"(n^3 Phase 1, n^2 per outer and per Sinkhorn "
                                   f"iteration) for {args.outer} outer iterations and "
                                   f"{args.ref_sweeps} Sinkhorn iterations (the plain "
                                   f"method's count on this workload)"},
        "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="cl50k")
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "f32"])
    # outer iterations per step (default: the workload's own count, 30 at 50k)
    ap.add_argument("--outer", type=int, default=None)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--check-every", type=int, default=5)
    ap.add_argument("--max-sweeps", type=int, default=5000)
    # Sinkhorn iterations of the plain method (FP32, cold start) in one step,
    # for --impl reference (default: the count measured on the GPU for the
    # default workload)
    ap.add_argument("--ref-sweeps", type=int, default=None)
    ap.add_argument("--e2e-runs", type=int, default=1)
    ap.add_argument("--no-fp32", dest="compare_fp32", action="store_false")
    ap.add_argument("--warm", default="learned", choices=["learned", "prev", "cold"])
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu", dest="cpu_baseline", action="store_false")
    args = ap.parse_args()
    if args.outer is None:
        args.outer = _synth_config(args.config)["outer"]
    if args.ref_sweeps is None:
        args.ref_sweeps = PLAIN_SWEEPS.get((args.config, args.outer), 0) or \
            int(round(2060 * args.outer))
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
