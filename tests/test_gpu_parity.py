"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 path): plan ||T - T_ref||_F / ||T_ref||_F <= 1e-4;
column marginals within 1e-6 relative to 1/n2; top-k indices identical in
every row whose relative score margin exceeds 1e-5.  Intermediate quantities
use bounds derived from FP32 rounding of the same arithmetic."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastalign_ref as R  # noqa: E402
from paper_2607_11952_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

PLAN_TOL = 1e-4
# The device computes |T^T 1 - nu|_1 in FP64 from FP32 column sums, each
# carrying a relative rounding error of a few ulp, so the reported error
# cannot go below about n2 * nu * 2^-23 ~ 1e-7; compare above that floor.
ERR_FLOOR = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _api():
    from paper_2607_11952_gb300 import api
    return api


def _oparams(p):
    return R.Params(eps=p.eps, eps_anc=p.eps_anc, alpha=p.alpha, beta=p.beta,
                    k_rwr=p.k_rwr, k_prop=p.k_prop, lam_e=p.lam_e,
                    lam_n=p.lam_n, lam_a=p.lam_a, lam_p=p.lam_p, delta=p.delta,
                    normalize_features=p.normalize_features)


def _aligner(g, p):
    api = _api()
    return api.Aligner(api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2), p)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _induced(n, keep, d, seed):
    rng = synth.rng_for(seed)
    e1 = synth.chung_lu(n, 2.3, 6.0, rng)
    return synth.make_pair(e1, n, d=d, sigma=0.2, anchor_frac=0.04,
                           frac_del=0.1, frac_add=0.1, rng=rng, keep_nodes=keep)


CASES = {
    "ba300": lambda: synth.config_pair("ba1k", n=300),
    "ragged700x530": lambda: _induced(700, 530, 24, 12),
}


# ------------------------------------------------------------ Phase 1

@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("gemm", ["simt", "auto"])
def test_node_cost_matches_oracle(case, gemm):
    g = CASES[case]()
    api = _api()
    p = api.Params(gemm=gemm)
    al = _aligner(g, p)
    al.node_cost(g.X1, g.X2, g.anchors)
    C = al.C_node.cpu().numpy()
    ph = R.phase1(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, _oparams(p))
    assert np.all(C[:, g.n2:] == 0.0)
    err = np.abs(C[:, : g.n2] - ph.C_node).max()
    assert err <= 5e-6 * np.abs(ph.C_node).max(), err


# ------------------------------------------------------------ Phase 2 + 3

def _oracle_first_kernel(ph, p, logS_prev):
    C_eff = R.outer_step(ph, logS_prev, p)
    logK = -C_eff / p.eps
    m = logK.max(axis=1, keepdims=True)
    Ks = np.exp(logK - m)
    n2 = logK.shape[1]
    log_v1 = -math.log(n2) - R.lse(logK - m, axis=0)
    return C_eff, Ks, log_v1


@pytest.mark.parametrize("case", sorted(CASES))
def test_outer_iteration_matches_oracle(case):
    g = CASES[case]()
    api = _api()
    # a large edge weight makes the C1 T C2^T term visible in the kernel
    p = api.Params(lam_e=2e5, lam_n=0.1)
    op = _oparams(p)
    al = _aligner(g, p)
    al.node_cost(g.X1, g.X2, g.anchors)
    al.plan_init()
    ph = R.phase1(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, op)
    logS = np.full((g.n1, g.n2), -math.log(g.n1 * g.n2))
    mu, nu = np.full(g.n1, 1 / g.n1), np.full(g.n2, 1 / g.n2)
    for outer in range(2):
        al.align_iter()
        torch.cuda.synchronize()
        C_eff, Ks, log_v1 = _oracle_first_kernel(ph, op, logS)
        K = al.K[:, : g.n2].cpu().numpy()
        assert np.all(al.K[:, g.n2:].cpu().numpy() == 0.0)
        assert _rel(K, Ks) <= 2e-5, (outer, _rel(K, Ks))
        np.testing.assert_allclose(K, Ks, rtol=2e-3, atol=2e-6)
        np.testing.assert_allclose(al.log_v.cpu().numpy(), log_v1, rtol=0, atol=2e-4)
        it, err, st = al.sinkhorn(30)
        a, b, errs, _ = R.sinkhorn_log(C_eff, mu, nu, op.eps, 30)
        logS = R.plan_log(C_eff, a, b, op.eps)
        T, Tr = al.plan_f64(), np.exp(logS)
        assert _rel(T, Tr) <= PLAN_TOL, (outer, _rel(T, Tr))
        assert it == 30
        assert abs(err - errs[-1]) <= 1e-3 * errs[-1] + ERR_FLOOR


def _top_agree(T, Tr, k):
    """Top-k indices identical wherever the relative margin exceeds 1e-5."""
    gi = np.argsort(-T, axis=1, kind="stable")[:, :k]
    ri = R.topk(Tr, k)
    srt = -np.sort(-Tr, axis=1)
    bad = 0
    for i in range(Tr.shape[0]):
        for r in range(k):
            margin = (srt[i, r] - srt[i, r + 1]) / max(srt[i, 0], 1e-300)
            if margin > 1e-5 and gi[i, r] != ri[i, r]:
                bad += 1
            if margin <= 1e-5:
                break
    return bad


@pytest.mark.parametrize("case,outer,sink", [("ba1k", 10, 50), ("ragged700x530", 4, 40)])
def test_end_to_end_matches_oracle(case, outer, sink):
    g = synth.config_pair("ba1k") if case == "ba1k" else CASES[case]()
    api = _api()
    p = api.Params()
    al = _aligner(g, p)
    hist = al.align(g.X1, g.X2, g.anchors, n_outer=outer, n_sink=sink)
    torch.cuda.synchronize()
    ref = R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors,
                      _oparams(p), outer, sink)
    T, Tr = al.plan_f64(), np.exp(ref["logS"])
    assert _rel(T, Tr) <= PLAN_TOL, _rel(T, Tr)
    # marginals
    m, mr = T.sum(axis=0), Tr.sum(axis=0)
    assert np.abs(m - mr).max() <= 1e-6 / g.n2 * 1.0 + 1e-6 * np.abs(mr).max()
    assert np.abs(T.sum(axis=1) - 1 / g.n1).max() <= 1e-6 / g.n1
    # errors per outer iteration
    for (it, err, st), h in zip(hist, ref["hist"]):
        assert it == sink
        assert abs(err - h["errs"][-1]) <= 1e-3 * h["errs"][-1] + ERR_FLOOR
    # top-k and the alignment metrics
    idx, score = al.topk(10)
    idx = idx.cpu().numpy()
    assert _top_agree(T, Tr, 10) == 0
    gi = np.argsort(-T, axis=1, kind="stable")[:, :10]
    srt = -np.sort(-Tr, axis=1)
    clear = ((srt[:, :10] - srt[:, 1:11]) / srt[:, :1] > 1e-5).all(axis=1)
    assert np.array_equal(idx[clear], gi[clear])
    hm = al.hits_mrr(g.test_pairs)
    hr = R.hits_mrr(Tr, g.test_pairs)
    assert abs(hm["hits@1"] - hr["hits@1"]) <= 1.0 / len(g.test_pairs) + 1e-12
    assert abs(hm["mrr"] - hr["mrr"]) <= 2e-3


def test_bf16_form_error_against_oracle():
    g = synth.config_pair("ba1k")
    api = _api()
    res = {}
    for dt in ("f32", "bf16"):
        al = _aligner(g, api.Params(dtype=dt))
        al.align(g.X1, g.X2, g.anchors, n_outer=10, n_sink=50)
        res[dt] = (al.plan_f64(), al.hits_mrr(g.test_pairs))
    ref = R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors,
                      R.Params(), 10, 50)
    Tr = np.exp(ref["logS"])
    e32, e16 = _rel(res["f32"][0], Tr), _rel(res["bf16"][0], Tr)
    print(f"plan error vs oracle: f32 {e32:.2e}, bf16 {e16:.2e}")
    assert e32 <= PLAN_TOL
    assert e16 <= 5e-2
    assert abs(res["bf16"][1]["hits@1"] - res["f32"][1]["hits@1"]) <= 0.005


# ------------------------------------------------------------ edge cases

def test_no_anchors_isolated_nodes_and_no_attributes():
    rng = synth.rng_for(5)
    n1, n2 = 130, 97
    e1 = synth.erdos_renyi(n1 - 10, 3.0, rng)      # nodes 120..129 isolated
    e2 = synth.erdos_renyi(n2, 2.0, rng)
    api = _api()
    p = api.Params()
    al = api.Aligner(api.Graph(n1, e1), api.Graph(n2, e2), p)
    X1 = np.zeros((n1, 0), np.float32)
    X2 = np.zeros((n2, 0), np.float32)
    anchors = np.zeros((0, 2), np.int64)
    al.node_cost(X1, X2, anchors)
    al.plan_init()
    ph = R.phase1(n1, n2, e1, e2, np.zeros((n1, 0)), np.zeros((n2, 0)), anchors, _oparams(p))
    np.testing.assert_allclose(al.C_node[:, :n2].cpu().numpy(), ph.C_node, atol=1e-6)
    for _ in range(2):
        al.align_iter()
        al.sinkhorn(20)
    ref = R.fastalign(n1, n2, e1, e2, np.zeros((n1, 0)), np.zeros((n2, 0)), anchors,
                      _oparams(p), 2, 20, ph=ph)
    assert _rel(al.plan_f64(), np.exp(ref["logS"])) <= PLAN_TOL


def test_edgeless_graph():
    """G2 without a single edge: every CSR is empty, so RWR keeps only the
    restart term, C2 and both right products vanish, the propagation of
    C_node gives 0 and C_nbr is the clamp -log(delta) everywhere."""
    rng = synth.rng_for(8)
    n1, n2 = 60, 45
    e1 = synth.erdos_renyi(n1, 3.0, rng)
    e2 = np.zeros((0, 2), np.int64)
    X1 = rng.standard_normal((n1, 8)).astype(np.float32)
    X2 = rng.standard_normal((n2, 8)).astype(np.float32)
    anchors = np.array([[0, 0], [5, 7], [9, 44]])
    api = _api()
    al = api.Aligner(api.Graph(n1, e1), api.Graph(n2, e2), api.Params())
    assert al.g2.nnz == 0
    al.align(X1, X2, anchors, n_outer=2, n_sink=20)
    ref = R.fastalign(n1, n2, e1, e2, X1, X2, anchors, R.Params(), 2, 20)
    assert _rel(al.plan_f64(), np.exp(ref["logS"])) <= PLAN_TOL


def test_two_node_graphs():
    api = _api()
    e = np.array([[0, 1]])
    X = np.array([[1.0, 0.0], [0.0, 1.0]], np.float32)
    al = api.Aligner(api.Graph(2, e), api.Graph(2, e), api.Params())
    hist = al.align(X, X, np.array([[0, 0]]), n_outer=2, n_sink=10)
    ref = R.fastalign(2, 2, e, e, X, X, np.array([[0, 0]]), R.Params(), 2, 10)
    assert _rel(al.plan_f64(), np.exp(ref["logS"])) <= PLAN_TOL


def test_warm_start_and_status_codes():
    from paper_2607_11952_gb300 import _lib as L
    g = synth.config_pair("ba1k", n=250)
    al = _aligner(g, _api().Params())
    al.node_cost(g.X1, g.X2, g.anchors)
    al.plan_init()
    al.align_iter()
    K0 = al.K.clone()
    v0 = al.log_v.clone()
    # FP32 column sums bound the reachable L1 marginal error near 1e-7
    it, err, st = al.sinkhorn(2000, tol=1e-6, check_every=10)
    assert st == L.FA_OK and err <= 1e-6 and it < 2000
    v_star = al.log_v.clone()
    # not converged is a status, not a crash; the state stays valid
    al.K.copy_(K0)
    al.log_v.copy_(v0)
    it, err, st = al.sinkhorn(3, tol=1e-12, check_every=1)
    assert st == L.FA_ERR_NOT_CONVERGED and it == 3 and err > 1e-12
    # a warm start at the fixed point converges at once
    it, err, st = al.sinkhorn(50, tol=1e-6, check_every=1, warm_log_v=v_star)
    assert st == L.FA_OK and it <= 2


def test_topk_and_rank_are_consistent():
    g = synth.config_pair("ba1k", n=400)
    al = _aligner(g, _api().Params())
    al.align(g.X1, g.X2, g.anchors, n_outer=3, n_sink=30)
    idx, _ = al.topk(5)
    idx = idx.cpu().numpy()
    rows = np.repeat(np.arange(g.n1), 5)
    r = al.rank(rows, idx.ravel()).cpu().numpy().reshape(g.n1, 5)
    assert np.array_equal(r, np.tile(np.arange(1, 6), (g.n1, 1)))
