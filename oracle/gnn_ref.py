"""FP64 oracle of the learned warm start (test infrastructure only).

TEST INFRASTRUCTURE ONLY: imported by the tests and nothing on the product
path.  The paper has no learned component; this restates the small model
the CUDA path trains, so its forward pass, gradients and optimiser step can
be checked.

Model (a 2-layer graph network on the column graph G2, hidden width 64):

    AF  = Abar F                       (n x 6, neighbourhood mean of features)
    A1  = AF W1 + b1                   (n x 64)
    H   = max(A1, 0)
    z2  = H w2                         (n)
    a   = Abar z2 + c                  (n, predicted potential correction)

Loss (gauge invariant: potentials are defined up to a constant):

    L = 1/n sum_j ((a_j - mean a) - (y_j - mean y))^2

Optimiser: Adam with bias correction.

The parity pin for the analytic gradient is a central finite difference of
the same FP64 loss (tests/test_gnn_oracle.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

HIDDEN = 64
FIN = 6
N_PARAMS = FIN * HIDDEN + HIDDEN + HIDDEN + 1   # W1, b1, w2, c


def unpack(theta: np.ndarray):
    """Parameter vector layout: W1 (FIN x 64, row-major), b1 (64), w2 (64), c."""
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + FIN * HIDDEN].reshape(FIN, HIDDEN)
    o += FIN * HIDDEN
    b1 = theta[o:o + HIDDEN]
    o += HIDDEN
    w2 = theta[o:o + HIDDEN]
    o += HIDDEN
    c = theta[o]
    return W1, b1, w2, c


def forward(Abar: sp.csr_matrix, F: np.ndarray, theta: np.ndarray):
    W1, b1, w2, c = unpack(theta)
    AF = Abar @ np.asarray(F, np.float64)
    A1 = AF @ W1 + b1
    H = np.maximum(A1, 0.0)
    z2 = H @ w2
    a = Abar @ z2 + c
    return a, dict(AF=AF, A1=A1, H=H, z2=z2)


def loss(a: np.ndarray, y: np.ndarray) -> float:
    r = (a - a.mean()) - (y - y.mean())
    return float(np.mean(r * r))


def backward(Abar: sp.csr_matrix, F, theta, y):
    """Analytic gradient of the loss with respect to theta."""
    W1, b1, w2, c = unpack(theta)
    a, cache = forward(Abar, F, theta)
    n = a.shape[0]
    r = (a - a.mean()) - (np.asarray(y, np.float64) - np.mean(y))
    g = 2.0 * r / n                     # dL/da (centring projects itself)
    gz2 = Abar.T @ g                    # a = Abar z2 + c
    dw2 = cache["H"].T @ gz2
    dH = np.outer(gz2, w2)
    dA1 = dH * (cache["A1"] > 0)
    dW1 = cache["AF"].T @ dA1
    db1 = dA1.sum(axis=0)
    dc = g.sum()                        # zero up to rounding
    grad = np.concatenate([dW1.ravel(), db1, dw2, [dc]])
    return loss(a, y), grad


def adam_step(theta, m, v, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) with bias correction; t >= 1."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def features(Abar_deg: np.ndarray, log_v1: np.ndarray, corr_prev: np.ndarray,
             pot_prev: np.ndarray | None = None, anchor_mask: np.ndarray | None = None,
             outer_index: int = 0) -> np.ndarray:
    """Per-node inputs of column node j: the centred cold first column
    update, the centred previous correction and the centred previous
    converged potential (potentials are defined up to a constant),
    log(1 + degree), the anchor flag and log(1 + outer iterations done)."""
    lv = np.asarray(log_v1, np.float64)
    n = lv.shape[0]
    cp = np.asarray(corr_prev, np.float64)
    pp = np.zeros(n) if pot_prev is None else np.asarray(pot_prev, np.float64)
    am = np.zeros(n) if anchor_mask is None else np.asarray(anchor_mask, np.float64)
    return np.stack([lv - lv.mean(), cp - cp.mean(),
                     np.log1p(np.asarray(Abar_deg, np.float64)),
                     pp - pp.mean(), am, np.full(n, np.log1p(outer_index))], axis=1)


def fit_scale(pred: np.ndarray, y: np.ndarray, max_abs: float, shrink: int = 0) -> float:
    """The trust in a prediction: the least-squares scale alpha minimising
    |(y - mean y) - alpha (p - mean p)|^2 for p = clamp(pred, -max_abs,
    max_abs) (non-finite entries 0), clipped to [0, 1]; 0 when p is
    constant.  shrink 1: alpha times the squared correlation rho^2 of p and
    y; shrink 2: alpha times |rho|; 0 (or any other value): alpha alone."""
    p = np.where(np.isfinite(pred), np.clip(np.asarray(pred, np.float64), -max_abs, max_abs), 0.0)
    yy = np.asarray(y, np.float64)
    dp, dy = p - p.mean(), yy - yy.mean()
    den = float(dp @ dp)
    if den == 0.0:
        return 0.0
    a = float(min(1.0, max(0.0, (dp @ dy) / den)))
    vy = float(dy @ dy)
    r2 = float((dp @ dy) ** 2 / (den * vy)) if vy > 0.0 else 0.0
    if int(shrink) == 1:
        a *= r2
    elif int(shrink) == 2:
        a *= float(np.sqrt(r2))
    return a
