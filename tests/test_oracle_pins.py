"""Pins for the FP64 oracle against facts fixed outside the oracle itself:
hand-computed values, brute-force loops over edges, closed forms, a generic
constrained optimiser and invariances of the method.  CPU only."""
import math

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

from oracle import fastalign_ref as R
from paper_2607_11952_gb300 import synth


def _adj_lists(n, edges):
    nb = [set() for _ in range(n)]
    for u, v in edges:
        if u != v:
            nb[u].add(int(v))
            nb[v].add(int(u))
    return [sorted(s) for s in nb]


# ------------------------------------------------------------ row normalisation

def test_row_normalized_hand_example():
    # path 0-1-2, a duplicate edge, a self-loop and an isolated node 3
    edges = np.array([[0, 1], [1, 2], [1, 0], [2, 2]])
    A = R.row_normalized(4, edges).toarray()
    want = np.array([[0, 1, 0, 0],
                     [0.5, 0, 0.5, 0],
                     [0, 1, 0, 0],
                     [0, 0, 0, 0]], dtype=float)
    np.testing.assert_array_equal(A, want)


def test_row_normalized_rows_sum_to_one_or_zero():
    rng = synth.rng_for(7)
    e = synth.erdos_renyi(300, 3.0, rng)
    A = R.row_normalized(300, e)
    s = np.asarray(A.sum(axis=1)).ravel()
    deg = np.bincount(e.ravel(), minlength=300)
    np.testing.assert_allclose(s[deg > 0], 1.0, rtol=0, atol=1e-15)
    assert np.all(s[deg == 0] == 0)


# ------------------------------------------------------------ RWR

def test_rwr_one_step_hand_value():
    A = R.row_normalized(3, np.array([[0, 1], [1, 2]]))
    R10, _ = R.one_hot_anchors(3, 3, np.array([[0, 0]]))
    got = R.rwr(A, R10, 0.15, 1)
    np.testing.assert_allclose(got[:, 0], [0.15, 0.425, 0.0], atol=1e-15)


def test_rwr_converges_to_ppr_solve():
    rng = synth.rng_for(3)
    n = 80
    e = synth.barabasi_albert(n, 2, rng)
    A = R.row_normalized(n, e)
    anchors = np.array([[3, 0], [17, 1], [40, 2]])
    R10, _ = R.one_hot_anchors(n, 3, anchors)
    beta = 0.15
    got = R.rwr(A, R10, beta, 400)
    want = beta * np.linalg.solve(np.eye(n) - (1 - beta) * A.toarray(), R10)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


# ------------------------------------------------------------ node cost

def test_initial_node_cost_hand_values():
    # R = 0 -> exp(0) = 1; features e_0, e_1 -> cosine matrix = I
    R1 = np.zeros((2, 3))
    R2 = np.zeros((2, 3))
    X = np.array([[2.0, 0.0], [0.0, 5.0]])
    Xh = R.normalize_features(X)
    C = R.initial_node_cost(R1, R2, Xh, Xh, 0.3)
    e1 = math.exp(-1.0)
    want = np.array([[0.3 + 0.7 * e1, 1.0], [1.0, 0.3 + 0.7 * e1]])
    np.testing.assert_allclose(C, want, atol=1e-15)


def test_node_cost_brute_force():
    rng = np.random.default_rng(0)
    R1, R2 = rng.random((5, 4)), rng.random((6, 4))
    X1, X2 = rng.standard_normal((5, 3)), rng.standard_normal((6, 3))
    X1h, X2h = R.normalize_features(X1), R.normalize_features(X2)
    C = R.initial_node_cost(R1, R2, X1h, X2h, 0.5)
    for i in range(5):
        for j in range(6):
            rr = sum(R1[i, t] * R2[j, t] for t in range(4))
            cos = sum(X1[i, t] * X2[j, t] for t in range(3)) / (
                math.sqrt(sum(x * x for x in X1[i])) * math.sqrt(sum(x * x for x in X2[j])))
            assert abs(C[i, j] - (0.5 * math.exp(-rr) + 0.5 * math.exp(-cos))) < 1e-14


# ------------------------------------------------------------ propagation

def test_propagation_is_double_neighbourhood_mean():
    rng = synth.rng_for(11)
    n1, n2 = 30, 25
    e1 = synth.erdos_renyi(n1, 3.0, rng)
    e2 = synth.erdos_renyi(n2, 3.0, rng)
    A1, A2 = R.row_normalized(n1, e1), R.row_normalized(n2, e2)
    C = np.random.default_rng(1).random((n1, n2))
    got = R.propagate_node_cost(A1, A2, C, 1)
    nb1, nb2 = _adj_lists(n1, e1), _adj_lists(n2, e2)
    for i in range(n1):
        for j in range(n2):
            if not nb1[i] or not nb2[j]:
                want = 0.0
            else:
                want = np.mean([[C[k, l] for l in nb2[j]] for k in nb1[i]])
            assert abs(got[i, j] - want) < 1e-14


# ------------------------------------------------------------ anchor cost

def test_anchor_cost_values():
    Ca = R.anchor_cost(3, 4, np.array([[0, 2], [2, 1]]), 0.05)
    assert Ca[0, 2] == pytest.approx(-math.log(1.05))
    assert Ca[2, 1] == pytest.approx(-math.log(1.05))
    mask = np.ones((3, 4), bool)
    mask[0, 2] = mask[2, 1] = False
    np.testing.assert_allclose(Ca[mask], -math.log(0.05))


# ------------------------------------------------------------ intra-graph, edge and neighbourhood costs

def _small_pair(seed=5, n1=24, n2=20):
    rng = synth.rng_for(seed)
    e1 = synth.erdos_renyi(n1, 3.0, rng)
    e2 = synth.erdos_renyi(n2, 3.0, rng)
    return n1, n2, e1, e2


def test_intra_costs_brute_force():
    n1, n2, e1, e2 = _small_pair()
    rng = np.random.default_rng(2)
    R1, R2 = rng.random((n1, 5)), rng.random((n2, 5))
    A1, A2 = R.row_normalized(n1, e1), R.row_normalized(n2, e2)
    C1, C2 = R.intra_costs(R1, R2, A1, A2)
    nb1, nb2 = _adj_lists(n1, e1), _adj_lists(n2, e2)
    for i in range(n1):
        for k in range(n1):
            want = (np.dot(R1[i], R1[k]) / len(nb1[i])) if k in nb1[i] else 0.0
            assert abs(C1[i, k] - want) < 1e-15
    for j in range(n2):
        for l in range(n2):
            # C2 = (R2 R2^T) .* A2bar^T: entry (j, l) carries 1/deg(l)
            want = (np.dot(R2[j], R2[l]) / len(nb2[l])) if l in nb2[j] else 0.0
            assert abs(C2[j, l] - want) < 1e-15


def test_edge_and_nbr_cost_brute_force():
    n1, n2, e1, e2 = _small_pair(6)
    rng = np.random.default_rng(3)
    S = rng.random((n1, n2))
    W1 = sp.csr_matrix(rng.random((n1, n1)) * R.row_normalized(n1, e1).toarray())
    W2 = sp.csr_matrix(rng.random((n2, n2)) * R.row_normalized(n2, e2).toarray())
    A1, A2 = R.row_normalized(n1, e1), R.row_normalized(n2, e2)
    Ce = R.edge_cost(W1, S, W2)
    Cn = R.nbr_cost(A1, S, A2, 1e-30)
    W1d, W2d, A1d, A2d = W1.toarray(), W2.toarray(), A1.toarray(), A2.toarray()
    for i in range(0, n1, 3):
        for j in range(0, n2, 2):
            ze = 0.0
            zn = 0.0
            for k in range(n1):
                for l in range(n2):
                    ze += W1d[i, k] * S[k, l] * W2d[j, l]
                    zn += A1d[k, i] * S[k, l] * A2d[l, j]
            assert abs(Ce[i, j] - ze) < 1e-13 * max(1.0, abs(ze))
            assert abs(Cn[i, j] + math.log(max(zn, 1e-30))) < 1e-12


# ------------------------------------------------------------ Eq. 1, Eq. 3, Eq. 4

def _closed_form_2x2(C, mu, nu, eps):
    q = math.exp(-(C[0, 0] + C[1, 1] - C[0, 1] - C[1, 0]) / eps)
    A = 1.0 - q
    B = mu[1] - nu[0] + q * (mu[0] + nu[0])
    Cc = -q * mu[0] * nu[0]
    lo, hi = max(0.0, nu[0] - mu[1]), min(mu[0], nu[0])
    if abs(A) < 1e-15:
        roots = [-Cc / B]
    else:
        disc = math.sqrt(B * B - 4 * A * Cc)
        roots = [(-B + disc) / (2 * A), (-B - disc) / (2 * A)]
    t = [r for r in roots if lo - 1e-15 <= r <= hi + 1e-15][0]
    return np.array([[t, mu[0] - t], [nu[0] - t, mu[1] - nu[0] + t]])


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_sinkhorn_2x2_closed_form(seed):
    rng = np.random.default_rng(seed)
    C = rng.random((2, 2))
    mu = rng.random(2) + 0.2
    mu /= mu.sum()
    nu = rng.random(2) + 0.2
    nu /= nu.sum()
    eps = 0.3
    a, b, errs, _ = R.sinkhorn_log(C, mu, nu, eps, 2000)
    S = np.exp(R.plan_log(C, a, b, eps))
    np.testing.assert_allclose(S, _closed_form_2x2(C, mu, nu, eps), rtol=0, atol=1e-13)


def test_sinkhorn_marginals_reach_1e10():
    rng = np.random.default_rng(4)
    n1, n2 = 40, 30
    C = rng.random((n1, n2))
    mu, nu = np.full(n1, 1 / n1), np.full(n2, 1 / n2)
    a, b, errs, its = R.sinkhorn_log(C, mu, nu, 0.1, 5000, tol=1e-10)
    S = np.exp(R.plan_log(C, a, b, 0.1))
    assert errs[-1] <= 1e-10
    assert np.abs(S.sum(0) - nu).sum() + np.abs(S.sum(1) - mu).sum() <= 1e-10
    assert its < 5000


def test_sinkhorn_minimises_entropic_objective():
    # Eq. 1 solved by a generic constrained optimiser on a 3x3 problem.
    rng = np.random.default_rng(5)
    C = rng.random((3, 3))
    mu = np.array([0.2, 0.3, 0.5])
    nu = np.array([0.4, 0.4, 0.2])
    eps = 0.2
    a, b, _, _ = R.sinkhorn_log(C, mu, nu, eps, 3000)
    S = np.exp(R.plan_log(C, a, b, eps))

    def f(x):
        Sx = x.reshape(3, 3)
        return float(np.sum(Sx * C) + eps * np.sum(Sx * (np.log(Sx) - 1.0)))

    cons = [{"type": "eq", "fun": lambda x, i=i: x.reshape(3, 3)[i].sum() - mu[i]} for i in range(3)]
    cons += [{"type": "eq", "fun": lambda x, j=j: x.reshape(3, 3)[:, j].sum() - nu[j]} for j in range(2)]
    res = so.minimize(f, np.outer(mu, nu).ravel(), method="SLSQP", constraints=cons,
                      bounds=[(1e-12, 1)] * 9, options=dict(ftol=1e-15, maxiter=1000))
    np.testing.assert_allclose(S, res.x.reshape(3, 3), atol=2e-6)
    assert R.entropic_objective(S, C, eps) <= f(res.x) + 1e-12


def test_sinkhorn_kkt_additive_form_and_zero_duality_gap():
    """Optimality of Eq. 1 under the marginal constraints, checked through
    its dual rather than the iteration: (i) the stationarity condition
    eps log S + C = a (+) b, an additive rank-2 form, leaves a zero
    double-centring residual; (ii) the dual
    D(a, b) = <a, nu> + <b, mu> - eps sum exp((a_j + b_i - C_ij) / eps)
    equals the primal objective at the returned potentials; (iii) D is
    concave and (a, b) maximises it, so no perturbation raises it.  Uneven
    masses and n1 != n2, so a swapped index or a dropped log-marginal term
    fails (ii)."""
    rng = np.random.default_rng(11)
    n1, n2 = 7, 5
    C = rng.random((n1, n2))
    mu = rng.random(n1)
    mu /= mu.sum()
    nu = rng.random(n2)
    nu /= nu.sum()
    eps = 0.3
    a, b, errs, _ = R.sinkhorn_log(C, mu, nu, eps, 5000, tol=1e-14)
    assert errs[-1] <= 1e-14
    logS = R.plan_log(C, a, b, eps)
    M = logS + C / eps
    resid = M - M.mean(axis=1, keepdims=True) - M.mean(axis=0, keepdims=True) + M.mean()
    assert np.abs(resid).max() <= 1e-12

    def dual(a_, b_):
        return float(a_ @ nu + b_ @ mu
                     - eps * np.exp((a_[None, :] + b_[:, None] - C) / eps).sum())

    primal = R.entropic_objective(np.exp(logS), C, eps)
    assert abs(primal - dual(a, b)) <= 1e-12
    d0 = dual(a, b)
    for _ in range(200):
        assert dual(a + rng.normal(0, 0.05, n2), b + rng.normal(0, 0.05, n1)) <= d0 + 1e-14


def test_log_and_scaling_sinkhorn_agree():
    rng = np.random.default_rng(6)
    n1, n2 = 12, 9
    C = rng.random((n1, n2))
    mu, nu = np.full(n1, 1 / n1), np.full(n2, 1 / n2)
    eps = 0.25
    a, b, errs, _ = R.sinkhorn_log(C, mu, nu, eps, 37)
    logK = -C / eps
    Ks = np.exp(logK - logK.max(axis=1, keepdims=True))     # row-stabilised
    u, v, errs2 = R.sinkhorn_scaling(Ks, mu, nu, 37)
    S1 = np.exp(R.plan_log(C, a, b, eps))
    S2 = u[:, None] * Ks * v[None, :]
    np.testing.assert_allclose(S1, S2, rtol=1e-12, atol=0)
    np.testing.assert_allclose(errs, errs2, rtol=1e-9, atol=1e-15)


def test_fixed_point_independent_of_b0():
    rng = np.random.default_rng(8)
    C = rng.random((15, 11))
    mu, nu = np.full(15, 1 / 15), np.full(11, 1 / 11)
    a1, b1, _, _ = R.sinkhorn_log(C, mu, nu, 0.2, 3000)
    a2, b2, _, _ = R.sinkhorn_log(C, mu, nu, 0.2, 3000, b0=rng.standard_normal(15))
    np.testing.assert_allclose(np.exp(R.plan_log(C, a1, b1, 0.2)),
                               np.exp(R.plan_log(C, a2, b2, 0.2)), atol=1e-14)


# ------------------------------------------------------------ Section 4.1.1

def test_topk_rank_hits_hand_example():
    S = np.array([[0.1, 0.5, 0.5, 0.2],
                  [0.9, 0.0, 0.3, 0.9]])
    np.testing.assert_array_equal(R.topk(S, 3), [[1, 2, 3], [0, 3, 2]])
    np.testing.assert_array_equal(R.rank_of(S, np.array([0, 0, 1, 1]), np.array([2, 0, 3, 1])),
                                  [2, 4, 2, 4])
    hm = R.hits_mrr(S, np.array([[0, 2], [1, 0]]))
    assert hm["hits@1"] == 0.5 and hm["hits@10"] == 1.0
    assert hm["mrr"] == pytest.approx((0.5 + 1.0) / 2)


# ------------------------------------------------------------ whole method

def test_first_outer_iteration_from_independent_coupling():
    # With S0 = mu nu^T constant, the proximal term is a constant shift, so
    # the first solve equals a Sinkhorn solve on C alone.
    g = synth.config_pair("ba1k", n=60, m=2, d=8)
    p = R.Params()
    ph = R.phase1(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p)
    out = R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p, 1, 300, ph=ph)
    S0 = np.full((g.n1, g.n2), 1.0 / (g.n1 * g.n2))
    C = R.total_cost(ph.C_node, R.edge_cost(ph.C1, S0, ph.C2),
                     R.nbr_cost(ph.A1bar, S0, ph.A2bar, p.delta), ph.C_anc, p)
    mu, nu = np.full(g.n1, 1 / g.n1), np.full(g.n2, 1 / g.n2)
    a, b, _, _ = R.sinkhorn_log(C, mu, nu, p.eps, 300)
    np.testing.assert_allclose(np.exp(out["logS"]), np.exp(R.plan_log(C, a, b, p.eps)),
                               rtol=1e-9, atol=1e-15)


def test_permutation_equivariance():
    g = synth.config_pair("ba1k", n=70, m=2, d=8)
    p = R.Params()
    out = R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p, 3, 20)
    rng = np.random.default_rng(9)
    pi = rng.permutation(g.n2)                      # relabel G2: j -> pi[j]
    e2 = pi[g.edges2]
    X2 = np.empty_like(g.X2)
    X2[pi] = g.X2
    anc = g.anchors.copy()
    anc[:, 1] = pi[anc[:, 1]]
    out2 = R.fastalign(g.n1, g.n2, g.edges1, e2, g.X1, X2, anc, p, 3, 20)
    S, S2 = np.exp(out["logS"]), np.exp(out2["logS"])
    np.testing.assert_allclose(S2[:, pi], S, rtol=1e-12, atol=1e-15)


def test_planted_permutation_is_recovered():
    # Aligning a graph to an exactly relabelled copy (identical attributes):
    # without propagation the attribute term alone singles out the true
    # match, so every test node must be recovered.
    rng = synth.rng_for(21)
    n = 200
    e1 = synth.barabasi_albert(n, 3, rng)
    g = synth.make_pair(e1, n, d=16, sigma=0.0, anchor_frac=0.1, frac_del=0.0,
                        frac_add=0.0, rng=rng)
    out = R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors,
                      R.Params(k_prop=0), 5, 50)
    assert R.hits_mrr(np.exp(out["logS"]), g.test_pairs)["hits@1"] == 1.0
    # With the propagation step of Algorithm 1 each node's own attribute cost
    # is replaced by its neighbourhood mean, so nodes with (nearly)
    # identical neighbourhoods can swap; every miss must still rank 2-3.
    out = R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors,
                      R.Params(), 5, 50)
    S = np.exp(out["logS"])
    r = R.rank_of(S, g.test_pairs[:, 0], g.test_pairs[:, 1])
    assert np.mean(r == 1) >= 0.98 and r.max() <= 3


def test_plan_l1_definition():
    # identical plans: 0; moving mass m between two entries: 2m; symmetric;
    # matches the double loop; two probability plans are at most 2 apart
    rng = np.random.default_rng(4)
    S = rng.random((3, 4))
    S /= S.sum()
    assert R.plan_l1(np.log(S), np.log(S)) == 0.0
    m = 0.05
    S2 = S.copy()
    S2[0, 0] -= m
    S2[2, 3] += m
    assert abs(R.plan_l1(np.log(S), np.log(S2)) - 2 * m) < 1e-15
    assert R.plan_l1(np.log(S), np.log(S2)) == R.plan_l1(np.log(S2), np.log(S))
    T = rng.random((3, 4))
    T /= T.sum()
    brute = sum(abs(S[i, j] - T[i, j]) for i in range(3) for j in range(4))
    assert abs(R.plan_l1(np.log(S), np.log(T)) - brute) < 1e-15
    assert R.plan_l1(np.log(S), np.log(T)) <= 2.0


# ------------------------------------------------------------ proximal outer loop

def _pure_node_cost_run(n1, n2, e1, e2, X1, X2, eps, lam_p, n_outer):
    """The oracle's outer loop with the structural, neighbourhood and anchor
    weights switched off, so every outer iteration sees the same cost
    C = C_node and only the proximal term links consecutive solves."""
    p = R.Params(eps=eps, lam_p=lam_p, lam_e=0.0, lam_n=0.0, lam_a=0.0, k_prop=0)
    anchors = np.zeros((0, 2), np.int64)
    out = R.fastalign(n1, n2, e1, e2, X1, X2, anchors, p, n_outer, 40000,
                      tol=1e-14, check_every=1)
    assert all(h["errs"][-1] <= 1e-14 for h in out["hist"])   # every solve converged
    return out, out["phase1"].C_node


def _prox_temperature(eps, lam_p, t):
    """Effective temperature after t proximal steps on a fixed cost.  Section
    3.1's proximal point step with the KL term of reading R-prox gives
    S_t = diag(x) exp(-C/eps - (lam_p/eps) (C/eta_{t-1})) diag(y), i.e.
    1/eta_t = 1/eps + (lam_p/eps) / eta_{t-1}, starting from the constant
    plan (1/eta_0 = 0).  With lam_p = eps this is eta_t = eps / t."""
    inv = 0.0
    for _ in range(t):
        inv = 1.0 / eps + (lam_p / eps) * inv
    return 1.0 / inv


@pytest.mark.parametrize("lam_ratio", [1.0, 0.5, 2.0])
def test_proximal_outer_loop_matches_2x2_closed_form(lam_ratio):
    """Fixed cost, 2 x 2: after t outer iterations the plan is the entropic
    optimum of C at the temperature eta_t of the proximal recursion, whose
    closed form is the 2 x 2 root above.  A flipped sign of the proximal
    term, or lam_p entering without its 1/eps weight, changes eta_t."""
    rng = np.random.default_rng(40)
    X1 = rng.standard_normal((2, 3))
    X2 = rng.standard_normal((2, 3))
    e = np.array([[0, 1]])
    eps = 0.5
    mu = nu = np.array([0.5, 0.5])
    for t in (1, 2, 3, 4):
        out, C = _pure_node_cost_run(2, 2, e, e, X1, X2, eps, lam_ratio * eps, t)
        eta = _prox_temperature(eps, lam_ratio * eps, t)
        want = _closed_form_2x2(C, mu, nu, eta)
        np.testing.assert_allclose(np.exp(out["logS"]), want, rtol=0, atol=1e-12)


def test_proximal_outer_loop_is_one_solve_at_eps_over_t():
    """Fixed cost on a 9 x 7 pair with lam_p = eps: t outer iterations equal
    a single entropic OT solve of C at eps / t (and differ from the solve at
    eps, so the pin is not vacuous)."""
    rng = synth.rng_for(41)
    n1, n2 = 9, 7
    e1 = synth.erdos_renyi(n1, 2.5, rng)
    e2 = synth.erdos_renyi(n2, 2.5, rng)
    X1 = rng.standard_normal((n1, 4))
    X2 = rng.standard_normal((n2, 4))
    eps = 0.1
    mu, nu = np.full(n1, 1 / n1), np.full(n2, 1 / n2)
    for t in (2, 3, 5):
        out, C = _pure_node_cost_run(n1, n2, e1, e2, X1, X2, eps, eps, t)
        a, b, errs, _ = R.sinkhorn_log(C, mu, nu, eps / t, 40000, tol=1e-14)
        want = np.exp(R.plan_log(C, a, b, eps / t))
        got = np.exp(out["logS"])
        np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-14)
        a1, b1, _, _ = R.sinkhorn_log(C, mu, nu, eps, 40000, tol=1e-14)
        assert np.abs(got - np.exp(R.plan_log(C, a1, b1, eps))).max() > 1e-3


@pytest.mark.parametrize("tol", [None, 1e-6])
def test_scaling_form_of_the_whole_method_matches_log_form(tol):
    """The two Sinkhorn forms of Eq. 3 inside the full outer loop: with the
    same iteration counts (or the same stopping rule) they give the same
    plans, potentials and iteration counts, on an uneven pair over several
    outer iterations (the proximal term then carries each solve into the
    next)."""
    rng = synth.rng_for(43)
    e1 = synth.chung_lu(80, 2.4, 5.0, rng)
    g = synth.make_pair(e1, 80, d=8, sigma=0.1, anchor_frac=0.1, frac_del=0.1,
                        frac_add=0.1, rng=rng, keep_nodes=64)
    p = R.Params()
    ph = R.phase1(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p)
    kw = dict(tol=tol, check_every=3, ph=ph)
    lg = R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p, 4, 60, **kw)
    sc = R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p, 4, 60,
                     sinkhorn="scaling", **kw)
    np.testing.assert_allclose(np.exp(sc["logS"]), np.exp(lg["logS"]), rtol=1e-10, atol=1e-16)
    assert [h["iters"] for h in sc["hist"]] == [h["iters"] for h in lg["hist"]]
    np.testing.assert_allclose(sc["hist"][-1]["errs"][-1], lg["hist"][-1]["errs"][-1],
                               rtol=1e-8, atol=1e-15)
    # potentials up to the gauge (a + k, b - k)
    k = np.mean(sc["a"] - lg["a"])
    np.testing.assert_allclose(sc["a"] - k, lg["a"], atol=1e-10)
    np.testing.assert_allclose(sc["b"] + k, lg["b"], atol=1e-10)
