"""FP64 oracle of selected rows of the first outer iteration's Gibbs kernel.

TEST INFRASTRUCTURE ONLY (like ``fastalign_ref``): used by the full-size
parity tests, which cannot hold the dense n1 x n2 matrices of the plain
oracle in host memory.  Each quantity of Phases 1-2 of Algorithm 1 is the plain
definition evaluated at the requested rows i of the n1 x n2 matrices:

* Row normalisation and RWR: Abar = D^{-1} A and the RWR encodings R1, R2 (whole, they
  are n x |L|), from ``fastalign_ref``.
* Node cost: C_node^(0)[k, :] = alpha exp(-R1[k] R2^T) + (1-alpha)
  exp(-X1h[k] X2h^T) for the rows k the propagation needs.
* Propagation (reading R-prop): row i of A1bar C A2bar^T is
  A2bar (A1bar[i, :] C)^T, needing the rows of C at the neighbours of i.
* Edge and neighbourhood products at the first outer iteration, whose plan is the
  independent coupling S0 = mu nu^T (reading R-init), a rank-one matrix:
  C1 S0 C2^T = (C1 mu)(C2 nu)^T and A1bar^T S0 A2bar = (A1bar^T mu)(A2bar^T nu)^T
  (associativity of the matrix products in the definitions).
* Anchor cost and cost assembly (readings R-anc, R-clamp) and the proximal step (R-prox):
  C_eff = C - lam_p log S0, x = -C_eff / eps, and the row-stabilised kernel
  K[i, :] = exp(x[i, :] - max_j x[i, j]) (reading R-b0), which is what the
  library stores.

Pinned in tests/test_oracle_rows.py against ``fastalign_ref`` evaluated on
whole matrices.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import fastalign_ref as R


def _node_cost_rows(ks, R1, R2, X1h, X2h, alpha):
    """Node cost (Algorithm 1) at rows ``ks``."""
    ks = np.asarray(ks, dtype=np.int64)
    return alpha * np.exp(-(R1[ks] @ R2.T)) + (1.0 - alpha) * np.exp(-(X1h[ks] @ X2h.T))


def _propagated_rows(rows, A1, A2, R1, R2, X1h, X2h, alpha, k_prop):
    """Propagation (Algorithm 1, R-prop), k_prop times, at ``rows``: each level needs the
    rows of the previous level at the neighbours of its own rows."""
    levels = [np.unique(np.asarray(rows, dtype=np.int64))]
    for _ in range(k_prop):
        cur = levels[-1]
        nb = [A1.indices[A1.indptr[i]:A1.indptr[i + 1]] for i in cur]
        levels.append(np.unique(np.concatenate([cur] + nb)))
    have = levels[-1]
    C = _node_cost_rows(have, R1, R2, X1h, X2h, alpha)
    pos = {int(k): t for t, k in enumerate(have)}
    for lev in range(k_prop - 1, -1, -1):
        want = levels[lev]
        out = np.zeros((want.shape[0], C.shape[1]))
        for t, i in enumerate(want):
            lo, hi = A1.indptr[i], A1.indptr[i + 1]
            y = np.zeros(C.shape[1])
            for k, w in zip(A1.indices[lo:hi], A1.data[lo:hi]):
                y += w * C[pos[int(k)]]
            out[t] = A2 @ y                      # (A1bar[i,:] C) A2bar^T
        C = out
        pos = {int(k): t for t, k in enumerate(want)}
    return np.stack([C[pos[int(i)]] for i in rows])


def _c1_times_vector(A1: sp.csr_matrix, R1: np.ndarray, m: np.ndarray, rows):
    """(C1 m)[i] for C1 = (R1 R1^T) .* A1bar (Algorithm 1, intra-graph costs), at ``rows``."""
    out = np.zeros(len(rows))
    for t, i in enumerate(rows):
        lo, hi = A1.indptr[i], A1.indptr[i + 1]
        ks = A1.indices[lo:hi]
        out[t] = np.sum(A1.data[lo:hi] * (R1[ks] @ R1[i]) * m[ks])
    return out


def _c2_times_vector(A2: sp.csr_matrix, R2: np.ndarray, v: np.ndarray, chunk=20000):
    """(C2 v)[j] for C2 = (R2 R2^T) .* A2bar^T (Algorithm 1, intra-graph costs), for every j:
    sum over the stored entries (l, j) of A2bar of A2bar[l, j] <R2[j], R2[l]> v[l]."""
    Acoo = A2.tocoo()
    out = np.zeros(A2.shape[0])
    for s in range(0, Acoo.nnz, chunk):
        l = Acoo.row[s:s + chunk]
        j = Acoo.col[s:s + chunk]
        w = Acoo.data[s:s + chunk]
        dots = np.einsum("ij,ij->i", R2[j], R2[l])
        np.add.at(out, j, w * dots * v[l])
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 value (8 significant bits, ties to
    even), returned as float64; the normal range only, which covers the
    RWR encodings and unit feature vectors this is used on."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # x = m 2^e, |m| in [0.5, 1)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


@dataclasses.dataclass
class Phase1Rows:
    """The S-independent whole quantities the rows are evaluated from."""
    n1: int
    n2: int
    A1: sp.csr_matrix
    A2: sp.csr_matrix
    R1: np.ndarray
    R2: np.ndarray
    X1h: np.ndarray
    X2h: np.ndarray


def prepare(n1, n2, edges1, edges2, X1, X2, anchors, p: R.Params) -> Phase1Rows:
    """Row normalisation, RWR and the attribute normalisation (R-feat)."""
    A1 = R.row_normalized(n1, edges1)
    A2 = R.row_normalized(n2, edges2)
    R10, R20 = R.one_hot_anchors(n1, n2, anchors)
    R1 = R.rwr(A1, R10, p.beta, p.k_rwr)
    R2 = R.rwr(A2, R20, p.beta, p.k_rwr)
    if p.normalize_features:
        X1h, X2h = R.normalize_features(X1), R.normalize_features(X2)
    else:
        X1h, X2h = np.asarray(X1, np.float64), np.asarray(X2, np.float64)
    return Phase1Rows(n1, n2, A1, A2, R1, R2, X1h, X2h)


def first_kernel_rows(n1, n2, edges1, edges2, X1, X2, anchors, p: R.Params, rows,
                      operands: str = "f64"):
    """Rows ``rows`` of the row-stabilised Gibbs kernel of the first outer
    iteration (from S0 = mu nu^T), as an len(rows) x n2 float64 array."""
    st = prepare(n1, n2, edges1, edges2, X1, X2, anchors, p)
    return first_kernel_rows_from(st, anchors, p, rows, operands)


def first_kernel_rows_from(st: Phase1Rows, anchors, p: R.Params, rows,
                           operands: str = "f64"):
    """As ``first_kernel_rows`` from prepared quantities.  operands="bf16"
    is the BF16 form of the method: the two node-similarity products of
    the node cost of Algorithm 1 take their operands (R1, R2, X1h, X2h) rounded to bfloat16,
    with exact products and sums; everything else stays float64."""
    rows = [int(i) for i in rows]
    n1, n2, A1, A2 = st.n1, st.n2, st.A1, st.A2
    R1, R2, X1h, X2h = st.R1, st.R2, st.X1h, st.X2h
    if operands == "bf16":
        g1, g2, f1, f2 = bf16_round(R1), bf16_round(R2), bf16_round(X1h), bf16_round(X2h)
    elif operands == "f64":
        g1, g2, f1, f2 = R1, R2, X1h, X2h
    else:
        raise ValueError(operands)
    C_node = _propagated_rows(rows, A1, A2, g1, g2, f1, f2, p.alpha, p.k_prop)

    mu = np.full(n1, 1.0 / n1)
    nu = np.full(n2, 1.0 / n2)
    # C_edge = (C1 mu)(C2 nu)^T at the first outer iteration
    c1m = _c1_times_vector(A1, R1, mu, rows)
    c2n = _c2_times_vector(A2, R2, nu)
    C_edge = c1m[:, None] * c2n[None, :]
    # C_nbr = -log(max((A1bar^T mu)(A2bar^T nu)^T, delta))
    a1m = np.asarray(A1.T @ mu).ravel()[rows]
    a2n = np.asarray(A2.T @ nu).ravel()
    C_nbr = -np.log(np.maximum(a1m[:, None] * a2n[None, :], p.delta))
    # C_anc = -log(eps_anc + OneHot(L))
    H = np.zeros((len(rows), n2))
    pos = {i: t for t, i in enumerate(rows)}
    for i, j in np.asarray(anchors, dtype=np.int64):
        if int(i) in pos:
            H[pos[int(i)], j] = 1.0
    C_anc = -np.log(p.eps_anc + H)
    C = C_node + p.lam_e * C_edge + p.lam_n * C_nbr + p.lam_a * C_anc
    logS0 = np.log(mu)[rows][:, None] + np.log(nu)[None, :]
    x = -(C - p.lam_p * logS0) / p.eps
    return np.exp(x - x.max(axis=1, keepdims=True))


def _c_intra_matrix(A: sp.csr_matrix, R_: np.ndarray, transpose: bool) -> sp.csr_matrix:
    """C1 = (R1 R1^T) .* A1bar, or C2 = (R2 R2^T) .* A2bar^T (transpose=True)
    (Algorithm 1, intra-graph costs), evaluated only on the stored entries
    of the adjacency; the definition is the same as the dense-then-masked
    one of ``fastalign_ref.intra_costs``."""
    M = (A.T if transpose else A).tocoo()
    dots = np.einsum("ij,ij->i", R_[M.row], R_[M.col])
    return sp.csr_matrix((M.data * dots, (M.row, M.col)), shape=M.shape)


def kernel_rows_from_plan(st: Phase1Rows, anchors, p: R.Params, rows,
                          plan_rows, operands: str = "f64"):
    """Rows ``rows`` of the row-stabilised Gibbs kernel of an outer iteration
    whose previous plan S_prev is general (Phases 1-2 of Algorithm 1 with the
    proximal step of reading R-prox).

    ``plan_rows(ks)`` returns the float64 rows ks of S_prev (len(ks) x n2).
    Each quantity is its definition at the requested rows:
      C_edge[i, :] = (sum_k C1[i, k] S_prev[k, :]) C2^T,
      C_nbr[i, :]  = -log(max((sum_k A1bar[k, i] S_prev[k, :]) A2bar, delta)),
      C_eff[i, :]  = C_node + lam_e C_edge + lam_n C_nbr + lam_a C_anc
                     - lam_p log S_prev[i, :],
    then x = -C_eff / eps and K[i, :] = exp(x - max_j x) (reading R-b0).
    A1bar is symmetric in pattern (undirected graphs), so the k with
    A1bar[k, i] != 0 are the neighbours of i, with weight 1/deg(k)."""
    rows = [int(i) for i in rows]
    n1, n2, A1, A2 = st.n1, st.n2, st.A1, st.A2
    R1, R2, X1h, X2h = st.R1, st.R2, st.X1h, st.X2h
    if operands == "bf16":
        g1, g2, f1, f2 = bf16_round(R1), bf16_round(R2), bf16_round(X1h), bf16_round(X2h)
    elif operands == "f64":
        g1, g2, f1, f2 = R1, R2, X1h, X2h
    else:
        raise ValueError(operands)
    C_node = _propagated_rows(rows, A1, A2, g1, g2, f1, f2, p.alpha, p.k_prop)
    C1 = _c_intra_matrix(A1, R1, transpose=False)
    C2 = _c_intra_matrix(A2, R2, transpose=True)
    A1T = A1.T.tocsr()
    out = np.empty((len(rows), n2))
    H = np.zeros(n2)
    anc = np.asarray(anchors, dtype=np.int64).reshape(-1, 2)
    for t, i in enumerate(rows):
        # left products: row i of C1 S_prev and of A1bar^T S_prev
        lo, hi = C1.indptr[i], C1.indptr[i + 1]
        ks = C1.indices[lo:hi]
        Sk = plan_rows(ks) if ks.size else np.zeros((0, n2))
        y_e = C1.data[lo:hi] @ Sk if ks.size else np.zeros(n2)
        lo2, hi2 = A1T.indptr[i], A1T.indptr[i + 1]
        ks2 = A1T.indices[lo2:hi2]
        Sk2 = Sk if np.array_equal(ks2, ks) else (plan_rows(ks2) if ks2.size else np.zeros((0, n2)))
        y_n = A1T.data[lo2:hi2] @ Sk2 if ks2.size else np.zeros(n2)
        # right products: (.) C2^T and (.) A2bar
        z_e = C2 @ y_e
        z_n = A2.T @ y_n
        H[:] = 0.0
        H[anc[anc[:, 0] == i, 1]] = 1.0
        C = (C_node[t] + p.lam_e * z_e - p.lam_n * np.log(np.maximum(z_n, p.delta))
             + p.lam_a * (-np.log(p.eps_anc + H)))
        logS_i = np.log(plan_rows(np.array([i]))[0])
        x = -(C - p.lam_p * logS_i) / p.eps
        out[t] = np.exp(x - x.max())
    return out
