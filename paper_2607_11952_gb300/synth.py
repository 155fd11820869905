"""Seeded synthetic workloads for network alignment (graph pairs, node
attributes, anchor links).

This module holds input generation only: random graphs, a planted node
permutation, edge noise, Gaussian attributes and an anchor sample.  It
contains none of the alignment method's arithmetic, so both the FP64 oracle
and the CUDA path can draw their inputs from it.

Every generator takes a ``numpy.random.Generator`` built from ``PCG64(seed)``
so a workload is fully determined by its parameters and seed.

Workload shapes follow the alignment problem statement (Section 2: two graphs
G1, G2 with adjacency A1, A2, attributes X1, X2 and an anchor set L of known
correspondences).  The paper's real datasets are not available; synthetic
Barabasi-Albert and Chung-Lu pairs with a planted permutation stand in for
them, and the Erdos-Renyi graphs of the scaling study (Section 4.1.3) are
available through ``erdos_renyi``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "GraphPair",
    "rng_for",
    "barabasi_albert",
    "chung_lu",
    "erdos_renyi",
    "canonical_edges",
    "edge_noise",
    "make_pair",
    "config_pair",
    "CONFIGS",
]


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def canonical_edges(n: int, src, dst) -> np.ndarray:
    """Undirected simple edge list as an (m, 2) int64 array with u < v,
    sorted, duplicates and self-loops removed."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    u = np.minimum(src, dst)
    v = np.maximum(src, dst)
    keep = u != v
    key = np.unique(u[keep] * n + v[keep])
    return np.stack([key // n, key % n], axis=1)


def barabasi_albert(n: int, m: int, rng: np.random.Generator) -> np.ndarray:
    """Preferential attachment: a star on nodes 0..m, then every new node
    attaches to m distinct existing nodes chosen with probability
    proportional to degree.  Gives exactly m*(n-m) edges."""
    if not (1 <= m < n):
        raise ValueError("need 1 <= m < n")
    edges = [(0, t) for t in range(1, m + 1)]
    # endpoint list: each node appears once per incident edge
    ends = np.empty(2 * m * n, dtype=np.int64)
    ne = 0
    for (a, b) in edges:
        ends[ne] = a
        ends[ne + 1] = b
        ne += 2
    for new in range(m + 1, n):
        chosen = set()
        while len(chosen) < m:
            chosen.add(int(ends[rng.integers(0, ne)]))
        for t in chosen:
            edges.append((t, new))
            ends[ne] = t
            ends[ne + 1] = new
            ne += 2
    e = np.asarray(edges, dtype=np.int64)
    return canonical_edges(n, e[:, 0], e[:, 1])


def _chung_lu_weights(n: int, gamma: float, avg_deg: float) -> np.ndarray:
    """Power-law expected degrees w_i ~ (i+1)^(-1/(gamma-1)), rescaled to
    mean avg_deg and capped at sqrt(sum w) so that w_i*w_j/sum(w) <= 1."""
    w = np.power(np.arange(1, n + 1, dtype=np.float64), -1.0 / (gamma - 1.0))
    w *= avg_deg / w.mean()
    for _ in range(50):
        cap = math.sqrt(w.sum())
        capped = w > cap
        if not capped.any():
            break
        w = np.minimum(w, cap)
        free = ~capped
        deficit = avg_deg * n - w.sum()
        if deficit <= 1e-9 * n or not free.any():
            break
        w[free] *= 1.0 + deficit / w[free].sum()
    return w  # non-increasing


def chung_lu(n: int, gamma: float, avg_deg: float,
             rng: np.random.Generator) -> np.ndarray:
    """Chung-Lu random graph with p_uv = min(1, w_u w_v / S) sampled in
    O(n + m) by geometric skipping over the sorted weights (Miller and
    Hagberg, "Efficient generation of networks with given expected
    degrees", 2011)."""
    w = _chung_lu_weights(n, gamma, avg_deg)
    S = float(w.sum())
    us, vs = [], []
    for u in range(n - 1):
        v = u + 1
        p = min(w[u] * w[v] / S, 1.0)
        while v < n and p > 0.0:
            if p < 1.0:
                r = rng.random()
                v += int(math.floor(math.log(r) / math.log1p(-p))) if r > 0 else 0
            if v < n:
                q = min(w[u] * w[v] / S, 1.0)
                if rng.random() < q / p:
                    us.append(u)
                    vs.append(v)
                p = q
                v += 1
    return canonical_edges(n, np.asarray(us, np.int64), np.asarray(vs, np.int64))


def erdos_renyi(n: int, avg_deg: float, rng: np.random.Generator) -> np.ndarray:
    """G(n, m) with m = round(n*avg_deg/2) uniform distinct edges."""
    m = int(round(n * avg_deg / 2))
    got = np.zeros((0, 2), np.int64)
    while got.shape[0] < m:
        k = int((m - got.shape[0]) * 1.1) + 16
        s = rng.integers(0, n, k)
        d = rng.integers(0, n, k)
        got = canonical_edges(n, np.concatenate([got[:, 0], s]),
                              np.concatenate([got[:, 1], d]))
    pick = rng.choice(got.shape[0], m, replace=False)
    return got[np.sort(pick)]


def edge_noise(n: int, edges: np.ndarray, frac_del: float, frac_add: float,
               rng: np.random.Generator) -> np.ndarray:
    """Delete round(frac_del*m) uniform edges, then add round(frac_add*m)
    uniform non-edges (m = the original edge count)."""
    m = edges.shape[0]
    n_del = int(round(frac_del * m))
    n_add = int(round(frac_add * m))
    keep = np.ones(m, bool)
    if n_del:
        keep[rng.choice(m, n_del, replace=False)] = False
    kept = edges[keep]
    existing = set((edges[:, 0] * n + edges[:, 1]).tolist())
    added = []
    while len(added) < n_add:
        a = int(rng.integers(0, n))
        b = int(rng.integers(0, n))
        if a == b:
            continue
        u, v = min(a, b), max(a, b)
        key = u * n + v
        if key in existing:
            continue
        existing.add(key)
        added.append((u, v))
    if added:
        kept = np.concatenate([kept, np.asarray(added, np.int64)])
    return canonical_edges(n, kept[:, 0], kept[:, 1])


@dataclasses.dataclass
class GraphPair:
    """One alignment workload.  Node i of G1 truly corresponds to node
    ``truth[i]`` of G2 (-1 if i has no counterpart)."""
    n1: int
    n2: int
    edges1: np.ndarray          # (m1, 2) int64, u < v
    edges2: np.ndarray          # (m2, 2) int64, u < v
    X1: np.ndarray              # (n1, d) float32
    X2: np.ndarray              # (n2, d) float32
    anchors: np.ndarray         # (|L|, 2) int64 pairs (i, j)
    truth: np.ndarray           # (n1,) int64
    test_pairs: np.ndarray      # (n_test, 2) true pairs that are not anchors
    name: str = ""
    seed: int = 0


def make_pair(edges1: np.ndarray, n1: int, *, d: int, sigma: float,
              anchor_frac: float, frac_del: float, frac_add: float,
              rng: np.random.Generator, keep_nodes: int | None = None,
              name: str = "", seed: int = 0) -> GraphPair:
    """G2 = a uniformly relabelled copy of G1 (optionally the subgraph
    induced by ``keep_nodes`` uniformly kept nodes) with edge noise;
    X1 ~ N(0,1), X2 = relabelled X1 + N(0, sigma^2); anchors are a uniform
    fraction of the true pairs."""
    X1 = rng.standard_normal((n1, d)).astype(np.float32)
    if keep_nodes is None or keep_nodes >= n1:
        kept = np.arange(n1)
    else:
        kept = np.sort(rng.choice(n1, keep_nodes, replace=False))
    n2 = kept.shape[0]
    perm = rng.permutation(n2)            # kept[t] -> perm[t] in G2
    truth = np.full(n1, -1, np.int64)
    truth[kept] = perm
    e = edges1
    sel = (truth[e[:, 0]] >= 0) & (truth[e[:, 1]] >= 0)
    e2 = canonical_edges(n2, truth[e[sel, 0]], truth[e[sel, 1]])
    e2 = edge_noise(n2, e2, frac_del, frac_add, rng)
    X2 = np.empty((n2, d), np.float32)
    X2[perm] = X1[kept] + sigma * rng.standard_normal((n2, d)).astype(np.float32)
    true_pairs = np.stack([kept, perm], axis=1)
    n_anc = int(round(anchor_frac * true_pairs.shape[0]))
    pick = rng.permutation(true_pairs.shape[0])
    anchors = true_pairs[np.sort(pick[:n_anc])]
    test = true_pairs[np.sort(pick[n_anc:])]
    return GraphPair(n1, n2, edges1, e2, X1, X2, anchors.astype(np.int64),
                     truth, test.astype(np.int64), name, seed)


# The five workloads: (graph model, sizes, noise, attributes, anchors).
CONFIGS = {
    # Barabasi-Albert n=1000, m=3; 10% of edges deleted and 5% added;
    # 32-dim attributes, sigma=0.1; 5% anchors; 10 outer x 50 Sinkhorn.
    "ba1k": dict(model="ba", n=1000, m=3, d=32, sigma=0.1, anchor_frac=0.05,
                 frac_del=0.10, frac_add=0.05, seed=1, outer=10, sink=50),
    # Chung-Lu n=10k, exponent 2.5, mean degree 8; 10% noise; 64-dim.
    "cl10k": dict(model="cl", n=10_000, gamma=2.5, avg_deg=8, d=64, sigma=0.1,
                  anchor_frac=0.05, frac_del=0.10, frac_add=0.10, seed=2,
                  outer=20, sink=100),
    # Chung-Lu n=50k, exponent 2.1, mean degree 10; 15% noise; 128-dim.
    "cl50k": dict(model="cl", n=50_000, gamma=2.1, avg_deg=10, d=128,
                  sigma=0.1, anchor_frac=0.05, frac_del=0.15, frac_add=0.15,
                  seed=3, outer=30, sink=None),
    # The same generator parameters at n=5000 (checked against the oracle).
    "cl50k_5k": dict(model="cl", n=5_000, gamma=2.1, avg_deg=10, d=128,
                     sigma=0.1, anchor_frac=0.05, frac_del=0.15,
                     frac_add=0.15, seed=3, outer=30, sink=None),
    # Learned warm start evaluation pairs: n=20k, 64-dim.
    "cl20k": dict(model="cl", n=20_000, gamma=2.5, avg_deg=10, d=64,
                  sigma=0.1, anchor_frac=0.05, frac_del=0.10, frac_add=0.10,
                  seed=4, outer=10, sink=None),
    # Uneven pair: G2 an induced 80k subgraph of a 100k graph.
    "cl100k": dict(model="cl", n=100_000, keep=80_000, gamma=2.2, avg_deg=16,
                   d=256, sigma=0.2, anchor_frac=0.02, frac_del=0.10,
                   frac_add=0.10, seed=5, outer=30, sink=None),
}


def config_pair(name: str, n: int | None = None, seed: int | None = None,
                **over) -> GraphPair:
    """Build a named workload, optionally at another size or seed."""
    c = dict(CONFIGS[name])
    c.update(over)
    if n is not None:
        c["n"] = n
        if "keep" in c:
            c["keep"] = int(round(c["keep"] * n / CONFIGS[name]["n"]))
    if seed is not None:
        c["seed"] = seed
    rng = rng_for(c["seed"])
    if c["model"] == "ba":
        e1 = barabasi_albert(c["n"], c["m"], rng)
    elif c["model"] == "cl":
        e1 = chung_lu(c["n"], c["gamma"], c["avg_deg"], rng)
    elif c["model"] == "er":
        e1 = erdos_renyi(c["n"], c["avg_deg"], rng)
    else:
        raise ValueError(c["model"])
    return make_pair(e1, c["n"], d=c["d"], sigma=c["sigma"],
                     anchor_frac=c["anchor_frac"], frac_del=c["frac_del"],
                     frac_add=c["frac_add"], rng=rng,
                     keep_nodes=c.get("keep"), name=name, seed=c["seed"])


def bf16_representable(x: np.ndarray) -> np.ndarray:
    """float32 values rounded (to nearest, ties to even) onto the bfloat16
    grid, so that a BF16 copy of them is exact.  Used for seeded initial
    weights that both sides of a parity test must see identically."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def random_kernel_rows(n_rows: int, n2: int, rng: np.random.Generator,
                       spread: float = 10.0) -> np.ndarray:
    """A block of rows of a seeded positive n_rows x n2 matrix with entries
    exp(-spread U), U uniform on [0, 1), rounded onto the bfloat16 grid
    (float32 array), so FP32 and BF16 storage of it hold the same values.
    Stands in for a Gibbs kernel where a test needs a general one."""
    u = rng.random((n_rows, n2), dtype=np.float32)
    return bf16_representable(np.exp(-np.float32(spread) * u))


def random_log_scalings(n: int, rng: np.random.Generator, sd: float = 0.5) -> np.ndarray:
    """Seeded log-scalings -log(n) + N(0, sd^2) (float32): a vector whose
    exponentials have the magnitude of a marginal 1/n."""
    return (-math.log(n) + sd * rng.standard_normal(n)).astype(np.float32)
