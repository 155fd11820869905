"""Small, self-contained workloads for profiling single kernels with ncu.

  python -m paper_2607_11952_gb300.profile_cases sweep --n1 5000 --n2 50000 --dtype bf16
  python -m paper_2607_11952_gb300.profile_cases gemm  --n 8192 --d 128 --anchors 410
  python -m paper_2607_11952_gb300.profile_cases passb --n 10000 --dtype bf16

sweep: the fused Sinkhorn sweep on an n1 x n2 kernel (one column slab per
       cluster CTA has the same shape as in the n2 x n2 problem); 8 sweeps.
gemm:  the node-similarity cost (RWR, SDDMM, tcgen05 GEMM, propagation)
       on an n x n Chung-Lu pair.
passb: one outer iteration (Pass A, Pass B, normalisation) on a Chung-Lu
       pair.
Each case prints one line with the device time of its main call.
"""
from __future__ import annotations

import argparse

import torch

from . import api, synth


def _timed(fn):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def case_sweep(n1, n2, dtype, sweeps=8):
    rng = synth.rng_for(1)
    e1 = synth.erdos_renyi(n1, 10, rng)
    e2 = synth.erdos_renyi(n2, 10, rng)
    al = api.Aligner(api.Graph(n1, e1), api.Graph(n2, e2), api.Params(dtype=dtype))
    al.plan_init()
    al.set_timing(True)
    al.sinkhorn(sweeps)
    ms, _ = al.last_sweep_ms()
    b = 2 if dtype == "bf16" else 4
    print(f"sweep {n1}x{n2} {dtype}: {ms:.4f} ms per sweep, {n1 * n2 * b / ms / 1e6:.0f} GB/s")


def case_gemm(n, d, anchors, dtype):
    g = synth.config_pair("cl50k", n=n, d=d, anchor_frac=anchors / n)
    al = api.Aligner(api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2),
                     api.Params(dtype=dtype, k_prop=0))
    ms = _timed(lambda: al.node_cost(g.X1, g.X2, g.anchors))
    print(f"node_cost {n}x{n} d={d} |L|={g.anchors.shape[0]} {dtype}: {ms:.2f} ms")


def case_passb(n, dtype):
    g = synth.config_pair("cl50k", n=n)
    al = api.Aligner(api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2), api.Params(dtype=dtype))
    al.node_cost(g.X1, g.X2, g.anchors)
    al.plan_init()
    al.align_iter()
    al.sinkhorn(30)
    ms = _timed(al.align_iter)
    print(f"align_iter {n}x{n} {dtype}: {ms:.2f} ms")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["sweep", "gemm", "passb"])
    ap.add_argument("--n1", type=int, default=5000)
    ap.add_argument("--n2", type=int, default=50000)
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--d", type=int, default=128)
    ap.add_argument("--anchors", type=int, default=410)
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "f32"])
    a = ap.parse_args(argv)
    if a.case == "sweep":
        case_sweep(a.n1, a.n2, a.dtype)
    elif a.case == "gemm":
        case_gemm(a.n, a.d, a.anchors, a.dtype)
    else:
        case_passb(a.n, a.dtype)


if __name__ == "__main__":
    main()
