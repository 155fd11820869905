"""Python front end of the GB300 FastAlign hot path.

``Graph`` and ``Aligner`` own the device buffers (torch tensors, used for
memory and streams only) and call the C ABI through ``_lib``; every step of
the method runs in the CUDA kernels of libfastalign.so.

Typical use (Algorithm 1):

    g1, g2 = Graph(n1, edges1), Graph(n2, edges2)
    al = Aligner(g1, g2, Params(dtype="bf16"))
    al.node_cost(X1, X2, anchors)          # Phase 1 of Algorithm 1
    al.plan_init()                         # S0 = mu nu^T
    for t in range(T):                     # outer iterations
        al.align_iter()                    # Phase 2 + Gibbs kernel
        al.sinkhorn(max_iter=50)           # Phase 3 (Eq. 3)
    idx, score = al.topk(10)               # read-out (Section 4.1.1)
"""
from __future__ import annotations

import dataclasses
import os

import numpy as np
import torch

from . import _lib as L


CHECKPOINT_FORMAT = "fastalign-checkpoint-1"


def write_checkpoint(path: str, state: dict) -> None:
    """Write an outer-loop checkpoint atomically and durably: the file is
    written under a temporary name beside ``path``, flushed to the storage
    device (fsync), renamed over ``path``, and the directory entry is
    flushed too.  An interruption at any point -- the process killed, or
    the machine losing power -- leaves either the previous checkpoint or the
    new one, never a truncated file under ``path``."""
    tmp = f"{path}.tmp.{os.getpid()}"
    try:
        with open(tmp, "wb") as f:
            torch.save({"format": CHECKPOINT_FORMAT, **state}, f)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
        d = os.open(os.path.dirname(os.path.abspath(path)), os.O_RDONLY)
        try:
            os.fsync(d)
        finally:
            os.close(d)
    finally:
        if os.path.exists(tmp):
            os.remove(tmp)


def read_checkpoint(path: str, n1: int, n2: int, ld: int, dtype: str) -> dict:
    """Read a checkpoint written by ``write_checkpoint`` and check that it
    belongs to an aligner of the same shape and kernel storage type."""
    ck = torch.load(path, map_location="cpu", weights_only=True)
    if not isinstance(ck, dict) or ck.get("format") != CHECKPOINT_FORMAT:
        raise ValueError("not a checkpoint of this library")
    if (ck["n1"], ck["n2"], ck["ld"], ck["dtype"]) != (n1, n2, ld, dtype):
        raise ValueError("checkpoint shape or storage type does not match this aligner")
    want = torch.bfloat16 if dtype == "bf16" else torch.float32
    if (tuple(ck["K"].shape) != (n1, ld) or ck["K"].dtype != want
            or tuple(ck["log_u"].shape) != (n1,) or tuple(ck["log_v"].shape) != (n2,)):
        raise ValueError("checkpoint arrays have the wrong shape or type")
    return ck


@dataclasses.dataclass
class Params:
    """Mirror of ``fa_params`` (defaults from ``fa_params_default``)."""
    dtype: str = "f32"              # storage of the Gibbs kernel: "f32" | "bf16"
    eps: float = 0.05
    eps_anc: float = 0.05
    alpha: float = 0.5
    beta: float = 0.15
    k_rwr: int = 10
    k_prop: int = 1
    lam_e: float = 1.0
    lam_n: float = 0.05
    lam_a: float = 0.05
    lam_p: float = 0.05
    delta: float = 1e-30
    normalize_features: bool = True
    gemm: str = "auto"              # "auto" | "tcgen05" | "simt"

    def to_c(self) -> L.fa_params:
        p = L.fa_params_default()
        p.dtype = {"f32": L.FA_F32, "bf16": L.FA_BF16}[self.dtype]
        for f in ("eps", "eps_anc", "alpha", "beta", "lam_e", "lam_n", "lam_a",
                  "lam_p", "delta"):
            setattr(p, f, float(getattr(self, f)))
        p.k_rwr = int(self.k_rwr)
        p.k_prop = int(self.k_prop)
        p.normalize_features = 1 if self.normalize_features else 0
        p.gemm_mode = {"auto": L.FA_GEMM_AUTO, "tcgen05": L.FA_GEMM_TCGEN05,
                       "simt": L.FA_GEMM_SIMT}[self.gemm]
        return p


class Graph:
    """Device CSR of an undirected graph (fa_build_graph)."""

    def __init__(self, n: int, edges: np.ndarray):
        e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
        self.n = int(n)
        self.handle = L.fa_build_graph(self.n, e[:, 0].astype(np.int32),
                                       e[:, 1].astype(np.int32))
        self.nnz = L.fa_graph_info(self.handle)[1]

    def close(self):
        if getattr(self, "handle", None):
            L.fa_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Aligner:
    """Holds one alignment context and the plan T = diag(e^log_u) K diag(e^log_v)."""

    def __init__(self, g1: Graph, g2: Graph, params: Params | None = None,
                 device: str | torch.device = "cuda"):
        self.g1, self.g2 = g1, g2
        self.params = params or Params()
        self.device = torch.device(device)
        self.ctx = L.fa_ctx_create(g1.handle, g2.handle, self.params.to_c())
        self.n1, self.n2 = g1.n, g2.n
        self.ld = L.fa_ctx_ld(self.ctx)
        kdt = torch.bfloat16 if self.params.dtype == "bf16" else torch.float32
        self.K = torch.empty((self.n1, self.ld), dtype=kdt, device=self.device)
        self.C_node = torch.empty((self.n1, self.ld), dtype=torch.float32, device=self.device)
        self.log_u = torch.empty(self.n1, dtype=torch.float32, device=self.device)
        self.log_v = torch.empty(self.n2, dtype=torch.float32, device=self.device)
        self.anchors = None             # the anchor pairs of the last node_cost

    # -- Phase 1
    def node_cost(self, X1, X2, anchors: np.ndarray, stream=None):
        X1 = torch.as_tensor(X1, dtype=torch.float32).to(self.device).contiguous()
        X2 = torch.as_tensor(X2, dtype=torch.float32).to(self.device).contiguous()
        d = X1.shape[1] if X1.ndim == 2 else 0
        self.anchors = np.asarray(anchors).reshape(-1, 2)
        L.fa_node_cost(self.ctx, X1 if d else None, X2 if d else None, d,
                       self.anchors, self.C_node, stream)

    def plan_init(self, stream=None):
        L.fa_plan_init(self.ctx, self.K, self.log_u, self.log_v, stream)

    # -- Phase 2
    def align_iter(self, stream=None):
        L.fa_align_iter(self.ctx, self.K, self.log_u, self.log_v, self.C_node, stream)

    # -- Phase 3
    def sinkhorn(self, max_iter: int, tol: float = -1.0, check_every: int = 1,
                 warm_log_v=None, stream=None):
        """Returns (iterations, marginal error, status)."""
        return L.fa_sinkhorn(self.ctx, self.K, self.log_u, self.log_v, warm_log_v,
                             max_iter, tol, check_every, stream)

    # -- read-out
    def topk(self, k: int, stream=None):
        idx = torch.empty((self.n1, k), dtype=torch.int32, device=self.device)
        score = torch.empty((self.n1, k), dtype=torch.float32, device=self.device)
        L.fa_topk(self.ctx, self.K, self.log_v, k, idx, score, stream)
        return idx, score

    def rank(self, rows, cols, stream=None):
        r = torch.as_tensor(np.asarray(rows), dtype=torch.int32).to(self.device)
        c = torch.as_tensor(np.asarray(cols), dtype=torch.int32).to(self.device)
        out = torch.empty_like(r)
        L.fa_rank(self.ctx, self.K, self.log_v, r, c, out, stream)
        return out

    def hits_mrr(self, test_pairs: np.ndarray, ks=(1, 10)):
        r = self.rank(test_pairs[:, 0], test_pairs[:, 1]).cpu().numpy()
        out = {f"hits@{k}": float(np.mean(r <= k)) for k in ks}
        out["mrr"] = float(np.mean(1.0 / r))
        return out

    def plan_f64(self) -> np.ndarray:
        """The plan as a host float64 array (for checks; n1 x n2)."""
        K = self.K[:, : self.n2].float().cpu().double().numpy()
        u = np.exp(self.log_u.cpu().double().numpy())
        v = np.exp(self.log_v.cpu().double().numpy())
        return u[:, None] * K * v[None, :]

    def set_timing(self, on: bool = True):
        L.fa_ctx_set_timing(self.ctx, on)

    def last_sweep_ms(self):
        return L.fa_ctx_last_sweep_ms(self.ctx)

    def plan_change(self, K, log_u, log_v, stream=None) -> float:
        """sum_ij |T_ij - T'_ij| between the current plan and the plan held
        as (K, log_u, log_v) (fa_plan_change)."""
        return L.fa_plan_change(self.ctx, self.K, self.log_u, self.log_v, K, log_u, log_v,
                                stream)

    # -- checkpoint / resume of the outer loop
    def save_checkpoint(self, path: str, t: int, extra: dict | None = None,
                        warm=None):
        """Write the state an interrupted alignment resumes from: the Gibbs
        kernel K, the log-scalings, the number t of outer iterations done
        and, with a warm starter, its carried state (the previous solve's
        correction), without which a resumed warm-started run would not
        repeat the uninterrupted one.  C_node is not saved (fa_node_cost
        recomputes it deterministically)."""
        state = {"n1": self.n1, "n2": self.n2, "ld": self.ld,
                 "dtype": self.params.dtype, "t": int(t),
                 "K": self.K.cpu(), "log_u": self.log_u.cpu(),
                 "log_v": self.log_v.cpu(), "extra": extra or {}}
        if warm is not None and hasattr(warm, "state"):
            state["warm"] = warm.state()
        write_checkpoint(path, state)

    def load_checkpoint(self, path: str, warm=None) -> int:
        """Restore K and the log-scalings written by save_checkpoint (and a
        warm starter's state, when one is given and was saved); returns the
        number of outer iterations they hold."""
        ck = read_checkpoint(path, self.n1, self.n2, self.ld, self.params.dtype)
        if warm is not None and hasattr(warm, "load_state"):
            if "warm" not in ck:
                raise ValueError("checkpoint holds no warm-start state")
            warm.load_state(ck["warm"])
        self.K.copy_(ck["K"])
        self.log_u.copy_(ck["log_u"])
        self.log_v.copy_(ck["log_v"])
        return int(ck["t"])

    def align(self, X1, X2, anchors, n_outer: int, n_sink: int, tol: float = -1.0,
              check_every: int = 1, warm=None, plan_tol: float | None = None,
              checkpoint: str | None = None, resume: str | None = None):
        """Algorithm 1 end to end; returns per-outer (iterations, error,
        status[, plan change]).

        warm: None (cold start), a warm starter (an object with ``solve``,
        such as gnn.WarmStarter, which runs its own before/after-solve steps
        and the cold-start fallback), or a callable warm(aligner) returning
        the warm column scaling for fa_sinkhorn.
        plan_tol: stop before n_outer once an outer iteration moves the plan
        by at most plan_tol in L1 (the outer loop's convergence test).
        checkpoint: write a checkpoint after every outer iteration (with the
        warm starter's state).
        resume: continue from a checkpoint (Phase 1 is recomputed)."""
        starter = warm if hasattr(warm, "solve") else None
        self.node_cost(X1, X2, anchors)
        t0 = 0
        if resume is not None:
            t0 = self.load_checkpoint(resume, warm=starter)
        else:
            self.plan_init()
        prev = None
        if plan_tol is not None:
            prev = (torch.empty_like(self.K), torch.empty_like(self.log_u),
                    torch.empty_like(self.log_v))
            for dst, src in zip(prev, (self.K, self.log_u, self.log_v)):
                dst.copy_(src)
        hist = []
        for t in range(t0, n_outer):
            self.align_iter()
            if starter is not None:
                it, err, st, _ = starter.solve(n_sink, tol, check_every)
            else:
                w = warm(self) if warm is not None else None
                it, err, st = self.sinkhorn(n_sink, tol, check_every, w)
            if checkpoint is not None:
                self.save_checkpoint(checkpoint, t + 1, warm=starter)
            if prev is None:
                hist.append((it, err, st))
                continue
            change = self.plan_change(*prev)
            hist.append((it, err, st, change))
            if change <= plan_tol:
                break
            for dst, src in zip(prev, (self.K, self.log_u, self.log_v)):
                dst.copy_(src)
        return hist

    def close(self):
        if getattr(self, "ctx", None):
            L.fa_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
