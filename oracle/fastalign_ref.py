"""FP64 CPU oracle for FastAlign's OT-based network alignment.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously
correct restatement of the method that the CUDA path is checked against.
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product path never does.  It shares no code
with the CUDA path: the only common module is the seeded input generator,
which holds none of the method's arithmetic.

Everything is float64 NumPy / SciPy.sparse, written in the order and
notation of the paper:

* Algorithm 1 (linear-algebraic view of OT-based alignment): Phase 1
  (normalisation, RWR, node, anchor and intra-graph costs, initial plan),
  Phase 2 (edge and neighbourhood costs, cost assembly), Phase 3 (Sinkhorn)
  and the alignment output.
* Eq. 1 (entropic OT objective), Eq. 2 (cost decomposition), Eq. 3 (log-domain
  Sinkhorn dual updates), Eq. 4 (plan recovery).
* Section 4.1.1 (Hits@K, MRR).

Where the paper is silent or inconsistent, the following readings are used
(each one is repeated where it is applied):

R-prop   C_node propagation is A1bar C A2bar^T (Section 3.4 text) rather
         than A1bar C A2bar (Algorithm 1): it averages over both
         neighbourhoods.  k_C is its own count.
R-feat   Attributes are L2-normalised per row before X1 X2^T (cosine
         similarity); switchable.
R-init   The plan starts as the independent coupling S0 = mu nu^T.
R-prox   The proximal term lambda_p log(S) enters as the KL-proximal point
         step: C_eff = C - lambda_p log S_prev, so with lambda_p = eps the
         Gibbs kernel is exp(-C/eps) * S_prev.
R-marg   Sinkhorn follows Eq. 3, including eps log nu and eps log mu, with
         mu = 1/n1, nu = 1/n2 (Section 2.1); a in R^{n2} holds column
         potentials and b in R^{n1} row potentials (Eq. 4).
R-b0     The initial row potential of each solve is the row stabiliser
         b0_i = -eps max_j(-C_eff_ij / eps), which makes every row of the
         initial Gibbs kernel peak at 1.  The paper does not state b0.
R-order  One Sinkhorn iteration is the a update then the b update
         (Algorithm 1, Phase 3); the marginal error is measured after the b
         update (rows are then exact): err = |S^T 1 - nu|_1 + |S 1 - mu|_1.
R-clamp  C_nbr = -log(max(Z, delta)) so isolated nodes and underflowed
         entries stay finite.
R-anc    C_anc = -log(eps_anc + OneHot(L)) with its own eps_anc.

Parity pins for every function live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Params",
    "row_normalized",
    "one_hot_anchors",
    "rwr",
    "normalize_features",
    "initial_node_cost",
    "propagate_node_cost",
    "anchor_cost",
    "intra_costs",
    "edge_cost",
    "nbr_cost",
    "total_cost",
    "sinkhorn_log",
    "sinkhorn_scaling",
    "plan_log",
    "entropic_objective",
    "plan_l1",
    "phase1",
    "fastalign",
    "topk",
    "rank_of",
    "hits_mrr",
    "lse",
]


@dataclasses.dataclass
class Params:
    """Hyper-parameters of Algorithm 1.  The paper names them but gives no
    values; these defaults were fixed once on the 1k Barabasi-Albert pair."""
    eps: float = 0.05          # entropic regulariser (Eq. 1)
    eps_anc: float = 0.05      # the eps inside C_anc (Algorithm 1, anchor cost)
    alpha: float = 0.5         # node-cost mix (Algorithm 1, node cost)
    beta: float = 0.15         # restart probability of the RWR (Algorithm 1)
    k_rwr: int = 10            # RWR iterations (Algorithm 1)
    k_prop: int = 1            # C_node propagation steps (Algorithm 1)
    lam_e: float = 1.0         # edge-consistency weight (Eq. 2)
    lam_n: float = 0.05        # neighbourhood-consistency weight (Eq. 2)
    lam_a: float = 0.05        # anchor weight (Eq. 2)
    lam_p: float = 0.05        # proximal weight (Section 3.1; the cost assembly of Algorithm 1)
    delta: float = 1e-30       # clamp inside -log(.) of C_nbr
    normalize_features: bool = True


# ---------------------------------------------------------------- Phase 1

def row_normalized(n: int, edges: np.ndarray) -> sp.csr_matrix:
    """Algorithm 1, row normalisation: symmetric 0/1 adjacency (duplicates and self-loops
    dropped) divided by its degree, Abar = D^{-1} A; degree-0 rows stay 0."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    r = np.concatenate([e[:, 0], e[:, 1]])
    c = np.concatenate([e[:, 1], e[:, 0]])
    A = sp.coo_matrix((np.ones(r.shape[0]), (r, c)), shape=(n, n)).tocsr()
    A.data[:] = 1.0                       # duplicates collapse to one edge
    A.eliminate_zeros()
    deg = np.asarray(A.sum(axis=1)).ravel()
    inv = np.zeros(n)
    inv[deg > 0] = 1.0 / deg[deg > 0]
    return (sp.diags(inv) @ A).tocsr()


def one_hot_anchors(n1: int, n2: int, anchors: np.ndarray):
    """Algorithm 1, anchor encoding: R1^(0)[i_l, l] = 1 and R2^(0)[j_l, l] = 1 for anchor l."""
    L = anchors.shape[0]
    R1 = np.zeros((n1, L))
    R2 = np.zeros((n2, L))
    for l, (i, j) in enumerate(np.asarray(anchors, dtype=np.int64)):
        R1[i, l] = 1.0
        R2[j, l] = 1.0
    return R1, R2


def rwr(Abar: sp.csr_matrix, R0: np.ndarray, beta: float, k: int) -> np.ndarray:
    """Algorithm 1, RWR: k iterations of R <- (1-beta) Abar R + beta R^(0),
    starting from R = R^(0)."""
    R = R0.copy()
    for _ in range(k):
        R = (1.0 - beta) * (Abar @ R) + beta * R0
    return R


def normalize_features(X: np.ndarray) -> np.ndarray:
    """Reading R-feat: unit L2 rows (zero rows stay zero)."""
    X = np.asarray(X, dtype=np.float64)
    nrm = np.sqrt((X * X).sum(axis=1, keepdims=True))
    return np.where(nrm > 0, X / np.where(nrm > 0, nrm, 1.0), 0.0)


def initial_node_cost(R1, R2, X1h, X2h, alpha: float) -> np.ndarray:
    """Algorithm 1, node cost: C_node = alpha exp(-R1 R2^T) + (1-alpha) exp(-X1 X2^T)."""
    return alpha * np.exp(-(R1 @ R2.T)) + (1.0 - alpha) * np.exp(-(X1h @ X2h.T))


def propagate_node_cost(A1bar, A2bar, C: np.ndarray, k: int) -> np.ndarray:
    """Algorithm 1, propagation, with reading R-prop: k times C <- A1bar C A2bar^T,
    evaluated as two sparse-dense products (Section 3.3)."""
    for _ in range(k):
        C = np.asarray(A1bar @ C)                 # left SpMM
        C = np.asarray((A2bar @ C.T).T)           # right SpMM: C A2bar^T
    return C


def anchor_cost(n1: int, n2: int, anchors: np.ndarray, eps_anc: float) -> np.ndarray:
    """Algorithm 1, anchor cost (reading R-anc): C_anc = -log(eps_anc + OneHot(L))."""
    H = np.zeros((n1, n2))
    for i, j in np.asarray(anchors, dtype=np.int64):
        H[i, j] = 1.0
    return -np.log(eps_anc + H)


def intra_costs(R1, R2, A1bar: sp.csr_matrix, A2bar: sp.csr_matrix):
    """Algorithm 1, intra-graph costs: C1 = (R1 R1^T) .* A1bar and C2 = (R2 R2^T) .* A2bar^T,
    evaluated dense-then-masked (the plain definition, not an SDDMM)."""
    M1 = A1bar.toarray()
    M2 = A2bar.T.toarray()
    C1 = (R1 @ R1.T) * M1
    C2 = (R2 @ R2.T) * M2
    return sp.csr_matrix(C1), sp.csr_matrix(C2)


# ---------------------------------------------------------------- Phase 2

def edge_cost(C1: sp.csr_matrix, S: np.ndarray, C2: sp.csr_matrix) -> np.ndarray:
    """Algorithm 1, edge cost: C_edge = C1 S C2^T (two SpMMs)."""
    return np.asarray((C2 @ np.asarray(C1 @ S).T).T)


def nbr_cost(A1bar: sp.csr_matrix, S: np.ndarray, A2bar: sp.csr_matrix,
             delta: float) -> np.ndarray:
    """Algorithm 1, neighbourhood cost (reading R-clamp): C_nbr = -log(max(A1bar^T S A2bar, delta))."""
    Z = np.asarray((A2bar.T @ np.asarray(A1bar.T @ S).T).T)
    return -np.log(np.maximum(Z, delta))


def total_cost(C_node, C_edge, C_nbr, C_anc, p: Params) -> np.ndarray:
    """Algorithm 1, cost assembly / Eq. 2: C = C_node + lam_e C_edge + lam_n C_nbr + lam_a C_anc."""
    return C_node + p.lam_e * C_edge + p.lam_n * C_nbr + p.lam_a * C_anc


# ---------------------------------------------------------------- Phase 3

def lse(x: np.ndarray, axis: int) -> np.ndarray:
    """log-sum-exp with a max shift; rows/columns that are all -inf give -inf."""
    m = np.max(x, axis=axis, keepdims=True)
    mf = np.where(np.isfinite(m), m, 0.0)
    with np.errstate(divide="ignore"):
        out = np.log(np.sum(np.exp(x - mf), axis=axis, keepdims=True)) + mf
    return np.squeeze(out, axis=axis)


def sinkhorn_log(C_eff: np.ndarray, mu: np.ndarray, nu: np.ndarray, eps: float,
                 n_iter: int, b0: np.ndarray | None = None, a_init=None,
                 tol: float | None = None, check_every: int = 1):
    """Log-domain Sinkhorn, Eq. 3, iteration order R-order:

        a_j = eps log nu_j - eps LSE_i((b_i - C_ij)/eps)
        b_i = eps log mu_i - eps LSE_j((a_j - C_ij)/eps)

    ``b0`` defaults to reading R-b0 (row stabiliser).  If ``a_init`` is
    given (a warm start for the column potentials) the first a update is
    skipped and the first b update uses it.  Runs ``n_iter`` iterations, or
    stops early at the first checked iteration whose marginal error is
    <= tol.  Returns (a, b, errs, iterations_run)."""
    logK = -C_eff / eps
    logmu = np.log(mu)
    lognu = np.log(nu)
    if b0 is None:
        b = -eps * np.max(logK, axis=1)
    else:
        b = np.asarray(b0, dtype=np.float64).copy()
    a = None
    errs = []
    it = 0
    for it in range(1, n_iter + 1):
        if it == 1 and a_init is not None:
            a = np.asarray(a_init, dtype=np.float64).copy()
        else:
            a = eps * lognu - eps * lse(b[:, None] / eps + logK, axis=0)
        b = eps * logmu - eps * lse(a[None, :] / eps + logK, axis=1)
        if tol is not None and (it % check_every == 0 or it == n_iter):
            e = marginal_error(logK, a, b, mu, nu, eps)
            errs.append(e)
            if e <= tol:
                break
        elif tol is None:
            errs.append(marginal_error(logK, a, b, mu, nu, eps))
    return a, b, np.asarray(errs), it


def plan_log(C_eff: np.ndarray, a: np.ndarray, b: np.ndarray, eps: float) -> np.ndarray:
    """Eq. 4 in logs: log S_ij = (a_j + b_i - C_ij) / eps."""
    return (a[None, :] + b[:, None] - C_eff) / eps


def marginal_error(logK, a, b, mu, nu, eps) -> float:
    """R-order: |S^T 1 - nu|_1 + |S 1 - mu|_1 with S from Eq. 4."""
    logS = logK + a[None, :] / eps + b[:, None] / eps
    S = np.exp(logS)
    return float(np.abs(S.sum(axis=0) - nu).sum() + np.abs(S.sum(axis=1) - mu).sum())


def sinkhorn_scaling(K: np.ndarray, mu: np.ndarray, nu: np.ndarray, n_iter: int,
                     u0: np.ndarray | None = None, v0: np.ndarray | None = None,
                     tol: float | None = None, check_every: int = 1,
                     track_err: bool = True):
    """Scaling-domain Sinkhorn, the exponentiated form of Eq. 3 with
    u = exp(b/eps), v = exp(a/eps): v = nu / (K^T u), then u = mu / (K v).
    Same iteration order and initial u as ``sinkhorn_log`` when K is the
    row-stabilised kernel and u0 = 1.  If ``v0`` is given (a column scaling
    already updated, like ``a_init`` of ``sinkhorn_log``) the first
    iteration skips its v update.  Stops after n_iter iterations, or at the
    first checked iteration whose marginal error (R-order) is <= tol.
    Returns (u, v, errs) and, when tol is given, the iteration count too."""
    u = np.ones(K.shape[0]) if u0 is None else np.asarray(u0, np.float64).copy()
    v = None
    errs = []
    it = 0
    for it in range(1, n_iter + 1):
        if it == 1 and v0 is not None:
            v = np.asarray(v0, np.float64).copy()
        else:
            v = nu / (K.T @ u)
        u = mu / (K @ v)
        checked = tol is not None and (it % check_every == 0 or it == n_iter)
        if track_err or checked:
            S_col = v * (K.T @ u)
            e = float(np.abs(S_col - nu).sum() + np.abs(u * (K @ v) - mu).sum())
            errs.append(e)
            if checked and e <= tol:
                break
    if tol is None:
        return u, v, np.asarray(errs)
    return u, v, np.asarray(errs), it


def plan_l1(logS_a: np.ndarray, logS_b: np.ndarray) -> float:
    """How far the plan moved between two outer iterations, the test of
    Algorithm 1's outer loop (repeat until the plan converges), read as the L1
    distance sum_ij |S_a,ij - S_b,ij| of the plans given as log S."""
    return float(np.abs(np.exp(logS_a) - np.exp(logS_b)).sum())


def entropic_objective(S: np.ndarray, C: np.ndarray, eps: float) -> float:
    """Eq. 1: <S, C> - eps H(S), with H(S) = -sum S (log S - 1)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        ent = -np.sum(np.where(S > 0, S * (np.log(S) - 1.0), 0.0))
    return float(np.sum(S * C) - eps * ent)


# ---------------------------------------------------------------- whole method

@dataclasses.dataclass
class Phase1:
    A1bar: sp.csr_matrix
    A2bar: sp.csr_matrix
    R1: np.ndarray
    R2: np.ndarray
    C_node: np.ndarray          # after propagation
    C_node0: np.ndarray         # before propagation (node cost of Algorithm 1)
    C_anc: np.ndarray
    C1: sp.csr_matrix
    C2: sp.csr_matrix


def phase1(n1, n2, edges1, edges2, X1, X2, anchors, p: Params) -> Phase1:
    """Phase 1 of Algorithm 1: the S-independent quantities."""
    A1 = row_normalized(n1, edges1)
    A2 = row_normalized(n2, edges2)
    R10, R20 = one_hot_anchors(n1, n2, anchors)
    R1 = rwr(A1, R10, p.beta, p.k_rwr)
    R2 = rwr(A2, R20, p.beta, p.k_rwr)
    if p.normalize_features:
        X1h, X2h = normalize_features(X1), normalize_features(X2)
    else:
        X1h, X2h = np.asarray(X1, np.float64), np.asarray(X2, np.float64)
    C0 = initial_node_cost(R1, R2, X1h, X2h, p.alpha)
    Cn = propagate_node_cost(A1, A2, C0, p.k_prop)
    Ca = anchor_cost(n1, n2, anchors, p.eps_anc)
    C1, C2 = intra_costs(R1, R2, A1, A2)
    return Phase1(A1, A2, R1, R2, Cn, C0, Ca, C1, C2)


def outer_step(ph: Phase1, logS_prev: np.ndarray, p: Params):
    """Phase 2 of Algorithm 1 plus reading R-prox: the effective cost of one outer
    iteration, C_eff = C(S_prev) - lam_p log S_prev."""
    S = np.exp(logS_prev)
    Ce = edge_cost(ph.C1, S, ph.C2)
    Cb = nbr_cost(ph.A1bar, S, ph.A2bar, p.delta)
    C = total_cost(ph.C_node, Ce, Cb, ph.C_anc, p)
    return C - p.lam_p * logS_prev


def fastalign(n1, n2, edges1, edges2, X1, X2, anchors, p: Params,
              n_outer: int, n_sink: int, tol: float | None = None,
              check_every: int = 1, ph: Phase1 | None = None,
              sinkhorn: str = "log"):
    """Algorithm 1 end to end: Phase 1 once, then n_outer rounds of Phase 2
    (S-dependent costs) and Phase 3 (Sinkhorn, Eq. 3), recovering S by Eq. 4.
    The plan is carried as log S in float64 so nothing underflows.

    sinkhorn="log" solves each outer iteration with the log-domain updates
    of Eq. 3; sinkhorn="scaling" with their exponentiated form on the
    row-stabilised kernel exp(log K - max_j log K) (reading R-b0: u = 1 is
    the stabilising b0), the same iterates in exact arithmetic and the form
    timed as the CPU baseline.

    Returns a dict with the final log S, the last potentials (log form)
    and, per outer iteration, the Sinkhorn errors and iteration counts."""
    if ph is None:
        ph = phase1(n1, n2, edges1, edges2, X1, X2, anchors, p)
    if sinkhorn not in ("log", "scaling"):
        raise ValueError(sinkhorn)
    mu = np.full(n1, 1.0 / n1)
    nu = np.full(n2, 1.0 / n2)
    logS = np.full((n1, n2), -math.log(n1 * n2))        # reading R-init
    hist = []
    a = b = None
    for _ in range(n_outer):
        C_eff = outer_step(ph, logS, p)
        if sinkhorn == "log":
            a, b, errs, its = sinkhorn_log(C_eff, mu, nu, p.eps, n_sink, tol=tol,
                                           check_every=check_every)
            logS = plan_log(C_eff, a, b, p.eps)
        else:
            logK = -C_eff / p.eps
            m = np.max(logK, axis=1, keepdims=True)
            Ks = np.exp(logK - m)
            # without tol only the last iteration's error is recorded
            u, v, errs, its = sinkhorn_scaling(
                Ks, mu, nu, n_sink, tol=tol if tol is not None else -1.0,
                check_every=check_every if tol is not None else n_sink,
                track_err=False)
            logS = np.log(u)[:, None] + (logK - m) + np.log(v)[None, :]
            b = p.eps * (np.log(u) - m[:, 0])     # (a_j + b_i)/eps = log u_i - m_i + log v_j
            a = p.eps * np.log(v)
        hist.append(dict(errs=errs, iters=its))
    return dict(logS=logS, a=a, b=b, hist=hist, phase1=ph)


# ---------------------------------------------------------------- read-out

def topk(S: np.ndarray, k: int) -> np.ndarray:
    """Per row, the k columns with the largest S_ij, ties to the lower j
    (stable sort on -S)."""
    order = np.argsort(-S, axis=1, kind="stable")
    return order[:, :k]


def rank_of(S: np.ndarray, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """1-based rank of column cols[t] in row rows[t] under the same order as
    ``topk``: 1 + #{j: S_j > S_c} + #{j < c: S_j == S_c}."""
    out = np.empty(rows.shape[0], np.int64)
    for t, (i, c) in enumerate(zip(rows, cols)):
        s = S[i]
        out[t] = 1 + int(np.sum(s > s[c])) + int(np.sum(s[:c] == s[c]))
    return out


def hits_mrr(S: np.ndarray, test_pairs: np.ndarray, ks=(1, 10)):
    """Section 4.1.1: Hits@K = #hits/n and MRR = mean 1/rank over the test
    pairs (x, x')."""
    r = rank_of(S, test_pairs[:, 0], test_pairs[:, 1])
    out = {f"hits@{k}": float(np.mean(r <= k)) for k in ks}
    out["mrr"] = float(np.mean(1.0 / r))
    return out
