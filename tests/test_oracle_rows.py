"""Pins of the row-restricted oracle (oracle/rows_ref.py) against the
whole-matrix oracle: the first outer iteration's row-stabilised Gibbs
kernel, Phases 1-2 of Algorithm 1 from the independent coupling, must agree row by row
to rounding (1e-12), for k_C = 0, 1, 2 and with anchors on the sampled rows."""
import numpy as np
import pytest

from oracle import fastalign_ref as R
from oracle import rows_ref
from paper_2607_11952_gb300 import synth


def _full_first_kernel(g, p):
    ph = R.phase1(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p)
    logS0 = np.full((g.n1, g.n2), -np.log(g.n1 * g.n2))
    x = -R.outer_step(ph, logS0, p) / p.eps
    return np.exp(x - x.max(axis=1, keepdims=True))


@pytest.mark.parametrize("k_prop", [0, 1, 2])
def test_rows_match_whole_matrix_oracle(k_prop):
    rng = synth.rng_for(77)
    e1 = synth.chung_lu(90, 2.4, 5.0, rng)
    g = synth.make_pair(e1, 90, d=8, sigma=0.1, anchor_frac=0.1, frac_del=0.1,
                        frac_add=0.1, rng=rng, keep_nodes=70)
    p = R.Params(k_prop=k_prop, lam_e=200.0)   # make the edge term visible
    K = _full_first_kernel(g, p)
    rows = [0, 5, int(g.anchors[0, 0]), g.n1 - 1]
    Kr = rows_ref.first_kernel_rows(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2,
                                    g.anchors, p, rows)
    assert Kr.shape == (len(rows), g.n2)
    np.testing.assert_allclose(Kr, K[rows], rtol=1e-12, atol=1e-14)
    # the anchor term is present on the anchor row
    assert np.isclose(Kr.max(axis=1), 1.0).all()


def test_rows_with_isolated_node_and_no_features():
    rng = synth.rng_for(3)
    n = 40
    e1 = synth.erdos_renyi(n - 3, 3.0, rng)          # nodes 37..39 isolated
    e2 = synth.erdos_renyi(n, 3.0, rng)
    X1 = rng.standard_normal((n, 4))
    X2 = rng.standard_normal((n, 4))
    anchors = np.array([[1, 2], [38, 5]])
    p = R.Params(normalize_features=False)
    ph = R.phase1(n, n, e1, e2, X1, X2, anchors, p)
    logS0 = np.full((n, n), -np.log(n * n))
    x = -R.outer_step(ph, logS0, p) / p.eps
    K = np.exp(x - x.max(axis=1, keepdims=True))
    rows = [38, 39, 1]
    Kr = rows_ref.first_kernel_rows(n, n, e1, e2, X1, X2, anchors, p, rows)
    np.testing.assert_allclose(Kr, K[rows], rtol=1e-12, atol=1e-14)


def test_bf16_round_definition():
    # 8 significant bits, ties to even, sign kept; exact values unchanged
    x = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-9, -3.0 - 2**-7, 0.15625, 1.0 + 2**-9])
    got = rows_ref.bf16_round(x)
    want = np.array([1.0, 1.0, 1.0 + 2**-7, -3.0 - 2**-7 + 0.0, 0.15625, 1.0])
    # 1 + 2^-8: halfway between 1 and 1 + 2^-7 -> even (1); 1 + 3*2^-9 -> 1 + 2^-7
    np.testing.assert_array_equal(got[[0, 1, 2, 4]], want[[0, 1, 2, 4]])
    assert got[3] == -3.0 - 2**-6 or got[3] == -3.0   # |x| in [2, 4): spacing 2^-6
    assert got[5] == 1.0
    r = np.random.default_rng(0).standard_normal(1000)
    b = rows_ref.bf16_round(r)
    assert np.all(np.abs(b - r) <= np.abs(r) * 2.0**-8)
    # idempotent and exactly 8 significant bits
    np.testing.assert_array_equal(rows_ref.bf16_round(b), b)
    m, _ = np.frexp(b)
    np.testing.assert_array_equal(m * 256, np.rint(m * 256))


def test_bf16_operands_change_only_the_node_products():
    rng = synth.rng_for(78)
    e1 = synth.chung_lu(60, 2.4, 5.0, rng)
    g = synth.make_pair(e1, 60, d=8, sigma=0.1, anchor_frac=0.1, frac_del=0.1,
                        frac_add=0.1, rng=rng)
    p = R.Params()
    st = rows_ref.prepare(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p)
    rows = [0, 1, 2]
    K64 = rows_ref.first_kernel_rows_from(st, g.anchors, p, rows, "f64")
    K16 = rows_ref.first_kernel_rows_from(st, g.anchors, p, rows, "bf16")
    d = np.abs(K16 - K64).max()
    assert 0 < d < 0.1
    # the whole-matrix oracle with bf16-rounded operands gives the same rows
    ph = R.phase1(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p)
    C0 = R.initial_node_cost(rows_ref.bf16_round(ph.R1), rows_ref.bf16_round(ph.R2),
                             rows_ref.bf16_round(R.normalize_features(g.X1)),
                             rows_ref.bf16_round(R.normalize_features(g.X2)), p.alpha)
    ph.C_node = R.propagate_node_cost(ph.A1bar, ph.A2bar, C0, p.k_prop)
    logS0 = np.full((g.n1, g.n2), -np.log(g.n1 * g.n2))
    x = -R.outer_step(ph, logS0, p) / p.eps
    K = np.exp(x - x.max(axis=1, keepdims=True))
    np.testing.assert_allclose(K16, K[rows], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("k_prop", [0, 1])
def test_rows_from_a_general_plan_match_whole_matrix_oracle(k_prop):
    """The row oracle of an outer iteration whose previous plan is general
    (not the rank-one first plan), against fastalign_ref's whole-matrix
    outer step on the same plan; rows with anchors, the highest-degree
    row and the last row included."""
    rng = synth.rng_for(79)
    e1 = synth.chung_lu(90, 2.2, 6.0, rng)
    g = synth.make_pair(e1, 90, d=8, sigma=0.1, anchor_frac=0.1, frac_del=0.1,
                        frac_add=0.1, rng=rng, keep_nodes=75)
    p = R.Params(k_prop=k_prop, lam_e=200.0)
    ph = R.phase1(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p)
    prng = np.random.default_rng(3)
    S = np.exp(-6.0 * prng.random((g.n1, g.n2)))
    S /= S.sum()
    logS = np.log(S)
    x = -R.outer_step(ph, logS, p) / p.eps
    K = np.exp(x - x.max(axis=1, keepdims=True))
    st = rows_ref.prepare(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p)
    deg = np.diff(st.A1.indptr)
    rows = [0, int(np.argmax(deg)), int(g.anchors[0, 0]), g.n1 - 1]
    Kr = rows_ref.kernel_rows_from_plan(st, g.anchors, p, rows, lambda ks: S[np.asarray(ks)])
    np.testing.assert_allclose(Kr, K[rows], rtol=1e-11, atol=1e-14)
