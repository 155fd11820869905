"""Benchmark of the GB300 FastAlign hot path (one JSON line on stdout).

Workload: the 50k-node Chung-Lu pair (exponent 2.1, mean degree 10, 15% edge
noise, 128-dim attributes, 5% anchors), seeded synthetic data.  One step is
an alignment with inputs resident in HBM: Phase 1 (RWR, SDDMM,
node-cost GEMM, propagation), then the workload's 30 outer iterations of
Phase 2 (Pass A, Pass B + Gibbs kernel) and Phase 3 (fused Sinkhorn sweeps,
learned warm start, until the L1 marginal error is <= 1e-4, checked every 5
sweeps), then the top-10 read-out.  The metric is the step time (lower is
better); beside it go the same alignment in plain FP32 with a cold start
and, on the same BF16 storage, the cold and previous-correction warm starts
(what the trained network adds).  The Gibbs kernel (5 GB in BF16) is far
larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--outer T] [--impl ours|reference]

The FP64 CPU oracle is timed, as it stands, on bounded samples it finishes
in seconds: the 1k Barabasi-Albert configuration in full (10 outer x 50
Sinkhorn iterations) and the 50k workload's 5k-node run (the same generator
parameters at n = 5000: Phase 1 and the first outer iterations to 1e-4).
The GPU runs the same samples through the same API, so each CPU/GPU ratio
is measured on identical work; the plans of both are compared.
--impl reference times the oracle alone on the 5k-node sample, each step
one run of it.
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

# The oracle's samples: the 1k BA configuration in full, and the 50k
# workload's 5k-node run (Phase 1 + its first outer iterations to 1e-4).
SAMPLE_OUTER = {"ba1k": 10, "cl50k_5k": 3}
SAMPLE_SINK = {"ba1k": 50, "cl50k_5k": 20000}
SAMPLE_TOL = {"ba1k": None, "cl50k_5k": 1e-4}


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
    traffic = _ncu_traffic(args, g.n1, g.n2)
    # the comparison arms below build their own aligners: free this one first
    # (at 100k x 80k one BF16 aligner holds about 144 GB)
    al.close()

    def timed_alignment(dtype, warm, runs=1):
        """The step on a fresh aligner of the given storage type and warm
        start, timed with CUDA events; one untimed outer iteration first
        brings the context's buffers into use."""
        a = api.Aligner(G1, G2, api.Params(dtype=dtype), device=dev)
        a.set_timing(True)
        a.node_cost(X1, X2, g.anchors)
        a.plan_init()
        a.align_iter()
        a.sinkhorn(5)
        out = []
        for _ in range(runs):
            rr = []
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sw = step(a, rr, warm=warm)
            e1.record(stream)
            torch.cuda.synchronize()
            out.append({"ms": round(e0.elapsed_time(e1), 1), "sweeps": sw,
                        "sweep_ms": round(sum(r[2] * r[0] for r in rr) /
                                          max(1, sum(r[0] for r in rr)), 4)})
        h = a.hits_mrr(g.test_pairs)
        a.close()
        ms_all = [o["ms"] for o in out]
        return {"ms_per_step": round(sum(ms_all) / len(ms_all), 1), "runs_ms": ms_all,
                "sweeps": out[-1]["sweeps"], "sweep_ms": out[-1]["sweep_ms"],
                "hits@1": h["hits@1"], "mrr": h["mrr"]}

    # plain FP32 cold start on the same pair, for the metric's comparison
    fp32 = None
    if args.compare_fp32 and args.dtype != "f32":
        fp32 = timed_alignment("f32", "cold", runs=args.fp32_runs)

    # what the trained network adds: the same BF16 alignment from the cold
    # start and from the previous-correction start (the network's base)
    ablation = None
    if args.ablation and args.dtype == "bf16":
        ablation = {"learned": {"ms_per_step": round(ms, 1),
                                "sweeps": total_sweeps / args.steps,
                                "hits@1": hits["hits@1"], "mrr": hits["mrr"]}}
        for w in ("prev", "cold"):
            ablation[w] = timed_alignment("bf16", w)

    # end to end through the public API from host buffers
    e2e = _e2e(args, g, dev, api, model) if args.e2e else None

    cpu = same = None
    if rank == 0 and world == 1 and args.cpu_baseline:
        cpu, same = _cpu_and_same_work(args, dev, model)
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
            "ablation": ablation,
            "roofline": {"kernel": "k_sweep", "bound": "hbm",
                         "achieved": round(achieved, 1) if achieved else None,
                         "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4) if achieved else None,
                         "traffic": traffic, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": algo_bytes,
                         "avg_launch_ms": round(avg_sweep, 4)},
            "cpu_baseline": cpu,
            "same_work": same,
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


def _ncu_traffic(args, n1, n2):
    """DRAM bytes per k_sweep launch from the committed ncu summary, if it
    was taken for the current kernel source, dtype and row width, scaled
    from the captured rows to n1 (None otherwise: another width has another
    launch shape)."""
    p = os.path.join(ROOT, "profiles", "k_sweep_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha256") != sweep_source_hash():
        return None
    e = d.get(args.dtype)
    if not e or e.get("captured_n2") != n2:
        return None
    return int(round(e["dram_bytes_per_launch_captured"] * n1 / e["captured_n1"]))


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


def _oracle_run(name):
    """The FP64 oracle (Algorithm 1 with the scaling form of Eq. 3) on one
    sample, timed on the host cores: Phase 1, then the sample's outer
    iterations (fixed Sinkhorn counts, or to its tolerance checked every
    5).  Returns (pair, wall ms, Sinkhorn iterations, log S)."""
    from oracle import fastalign_ref as R
    from paper_2607_11952_gb300 import synth
    g = synth.config_pair(name)
    t0 = time.perf_counter()
    out = R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, R.Params(),
                      SAMPLE_OUTER[name], SAMPLE_SINK[name], tol=SAMPLE_TOL[name],
                      check_every=5, sinkhorn="scaling")
    ms = (time.perf_counter() - t0) * 1e3
    return g, ms, int(sum(h["iters"] for h in out["hist"])), out["logS"]


def _gpu_run(name, dtype, warm, dev, model):
    """The same sample through the library's API on the GPU (inputs
    resident), timed with CUDA events: (ms, Sinkhorn iterations, plan)."""
    import torch
    from paper_2607_11952_gb300 import api, gnn, synth
    g = synth.config_pair(name)
    G1, G2 = api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2)
    X1 = torch.from_numpy(g.X1).to(dev)
    X2 = torch.from_numpy(g.X2).to(dev)
    tol = SAMPLE_TOL[name]

    def run(al):
        al.node_cost(X1, X2, g.anchors)
        al.plan_init()
        ws = gnn.WarmStarter(al, warm, model if warm == "learned" else None)
        it = 0
        for _ in range(SAMPLE_OUTER[name]):
            al.align_iter()
            it += ws.solve(SAMPLE_SINK[name], -1.0 if tol is None else tol, 5)[0]
        return it

    al = api.Aligner(G1, G2, api.Params(dtype=dtype), device=dev)
    run(al)                                   # warm-up run
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    it = run(al)
    e1.record(s)
    torch.cuda.synchronize()
    T = al.plan_f64()
    al.close()
    return e0.elapsed_time(e1), it, T


def _sample_text(name, g):
    if name == "ba1k":
        return (f"1k Barabasi-Albert configuration in full: Phase 1 + 10 outer x 50 "
                f"Sinkhorn iterations (n={g.n1})")
    return (f"the 50k workload's 5k-node run (same generator parameters at n={g.n1}): "
            f"Phase 1 + {SAMPLE_OUTER[name]} outer iterations, Sinkhorn to "
            f"{SAMPLE_TOL[name]:g} checked every 5")


def _cpu_and_same_work(args, dev, model):
    """cpu_baseline: the oracle as it stands on the 50k workload's 5k-node
    run, measured (not scaled).  same_work: per sample, the oracle's time
    beside the GPU's on identical work (plain FP32, cold start, the same
    iteration rule) and the relative plan error of the GPU's FP32 and
    BF16 + learned forms against the oracle's FP64 plan."""
    import numpy as np
    same = []
    main = None
    for name in ("ba1k", "cl50k_5k"):
        g, ms_o, it_o, logS = _oracle_run(name)
        Tr = np.exp(logS)
        entry = {"workload": _sample_text(name, g), "oracle_ms": round(ms_o, 1),
                 "oracle_sinkhorn_iterations": it_o, "cores": os.cpu_count()}
        for dtype, warm in (("f32", "cold"), ("bf16", "learned")):
            if warm == "learned" and model is None:
                continue
            ms_g, it_g, T = _gpu_run(name, dtype, warm, dev, model)
            key = f"gpu_{dtype}_{warm}"
            entry[key] = {"ms": round(ms_g, 2), "sinkhorn_iterations": it_g,
                          "plan_rel_err_vs_oracle": float(np.linalg.norm(T - Tr) / np.linalg.norm(Tr))}
        entry["ratio_oracle_over_gpu_f32"] = round(ms_o / entry["gpu_f32_cold"]["ms"], 1)
        same.append(entry)
        if name == "cl50k_5k":
            main = (g, ms_o, it_o)
    g, ms_o, it_o = main
    # the step's scale relative to the sample, for context only
    s2 = (50_000 / g.n1) * (50_000 / g.n2)
    cpu = {"value": round(ms_o, 1), "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
           "sample": "FP64 oracle (scaling form of Eq. 3, NumPy/SciPy, BLAS on all cores) on "
                     + _sample_text("cl50k_5k", g) + f"; {it_o} Sinkhorn iterations; measured",
           "sample_vs_workload": {"elements_per_iteration_ratio": round(s2, 1),
                                  "note": "value is the sample's measured time, not scaled: the "
                                          "50k step does ~100x the per-iteration work of the "
                                          "sample and more outer iterations; the oracle is not "
                                          "run at 50k (20 GB per FP64 dense matrix); the GPU "
                                          "is timed on the same sample in same_work"}}
    return cpu, same


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
    """The FP64 oracle as it stands on the host cores, each step one run of
    the 50k workload's 5k-node sample (Phase 1 + its first outer iterations
    to 1e-4); the value is that run's measured wall time."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    vals = []
    g = None
    its = 0
    t_all = time.perf_counter()
    for k in range(args.warmup + args.steps):
        g, ms, its, _ = _oracle_run("cl50k_5k")
        if k >= args.warmup:
            vals.append(ms)
    wall = (time.perf_counter() - t_all) * 1e3
    v = sum(vals) / len(vals)
    sample = ("FP64 oracle (scaling form of Eq. 3, NumPy/SciPy, BLAS on all cores), cold "
              "start, on " + _sample_text("cl50k_5k", g) + f"; {its} Sinkhorn iterations")
    line = {
        "metric": METRIC, "value": round(v, 1), "unit": "ms", "impl": "reference",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Chung-Lu pair; no dataset)",
        "config": _config(args, world),
        "timed_workload": _sample_text("cl50k_5k", g),
        "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_ms_all_runs": round(wall, 1),
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
    ap.add_argument("--e2e-runs", type=int, default=2)
    ap.add_argument("--fp32-runs", type=int, default=2)
    ap.add_argument("--no-fp32", dest="compare_fp32", action="store_false")
    ap.add_argument("--no-ablation", dest="ablation", action="store_false")
    ap.add_argument("--warm", default="learned", choices=["learned", "prev", "cold"])
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu", dest="cpu_baseline", action="store_false")
    args = ap.parse_args()
    if args.outer is None:
        args.outer = _synth_config(args.config)["outer"]
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
