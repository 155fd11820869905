"""Sanity of the seeded workload generators (CPU only)."""
import numpy as np
import pytest

from paper_2607_11952_gb300 import synth


def test_ba_edge_count_and_determinism():
    e = synth.barabasi_albert(1000, 3, synth.rng_for(1))
    assert e.shape[0] == 3 * (1000 - 3)
    e2 = synth.barabasi_albert(1000, 3, synth.rng_for(1))
    np.testing.assert_array_equal(e, e2)
    assert np.all(e[:, 0] < e[:, 1])


def test_chung_lu_mean_degree():
    for n, g, d in [(20000, 2.5, 8.0), (20000, 2.1, 10.0)]:
        e = synth.chung_lu(n, g, d, synth.rng_for(3))
        mean = 2 * e.shape[0] / n
        assert abs(mean - d) / d < 0.05, mean
        deg = np.bincount(e.ravel(), minlength=n)
        assert deg.max() > 20 * d          # heavy tail


def test_pair_truth_and_anchors():
    g = synth.config_pair("ba1k")
    assert g.n1 == g.n2 == 1000
    assert g.anchors.shape[0] == 50
    assert np.all(g.truth[g.anchors[:, 0]] == g.anchors[:, 1])
    assert np.all(g.truth[g.test_pairs[:, 0]] == g.test_pairs[:, 1])
    assert g.anchors.shape[0] + g.test_pairs.shape[0] == 1000
    m1 = g.edges1.shape[0]
    # 10% deleted and 5% added
    assert g.edges2.shape[0] == m1 - round(0.10 * m1) + round(0.05 * m1)


def test_induced_uneven_pair():
    g = synth.config_pair("cl100k", n=2000)
    assert g.n1 == 2000 and g.n2 == 1600
    kept = np.nonzero(g.truth >= 0)[0]
    assert kept.shape[0] == 1600
    assert np.array_equal(np.sort(g.truth[kept]), np.arange(1600))


def test_ba_degrees_match_networkx():
    """Same model as networkx's preferential-attachment generator (a star
    on m+1 nodes, then m distinct degree-proportional targets per new
    node): pooled degree distributions over five seeds are
    indistinguishable by a two-sample Kolmogorov-Smirnov test."""
    nx = pytest.importorskip("networkx")
    ss = pytest.importorskip("scipy.stats")
    ours, theirs = [], []
    for s in range(5):
        e = synth.barabasi_albert(2000, 3, synth.rng_for(100 + s))
        ours.append(np.bincount(e.ravel(), minlength=2000))
        G = nx.barabasi_albert_graph(2000, 3, seed=100 + s)
        theirs.append(np.array([d for _, d in G.degree()]))
    o, t = np.concatenate(ours), np.concatenate(theirs)
    assert o.min() == t.min() == 3
    assert o.sum() == t.sum()
    assert ss.ks_2samp(o, t).pvalue > 0.05


@pytest.mark.parametrize("gamma", [2.1, 2.5, 2.8])
def test_chung_lu_tail_exponent(gamma):
    """P(deg >= k) ~ k^-(gamma-1) in the tail: the discrete Hill estimate
    1 + n_tail / sum log(d / (k_min - 1/2)) over degrees >= 20 recovers
    gamma (its standard error here is about 0.05; the finite-size cap at
    sqrt(sum w) biases it slightly upward)."""
    n = 30000
    e = synth.chung_lu(n, gamma, 8.0, synth.rng_for(3))
    deg = np.bincount(e.ravel(), minlength=n)
    tail = deg[deg >= 20]
    assert tail.size > 1000
    g_hat = 1.0 + tail.size / np.log(tail / 19.5).sum()
    assert abs(g_hat - gamma) < 0.2, g_hat


def test_chung_lu_pair_noise_attributes_and_anchors():
    """N11 noise for the Chung-Lu workloads (delete x% of G2's edges, add as
    many non-edges: the edge count is kept), the relabelling carries every
    kept edge that was not deleted, X2 = relabelled X1 + N(0, sigma^2), and
    5% anchors."""
    g = synth.config_pair("cl50k", n=4000)
    e1 = {(int(u), int(v)) for u, v in g.edges1}
    e2 = {(int(u), int(v)) for u, v in g.edges2}
    assert len(e2) == len(e1)
    mapped = {tuple(sorted((int(g.truth[u]), int(g.truth[v])))) for u, v in e1}
    kept = len(mapped & e2)
    assert kept == len(e1) - round(0.15 * len(e1))
    diff = g.X2[g.truth] - g.X1
    assert abs(float(diff.std()) - 0.1) < 0.005 and abs(float(diff.mean())) < 0.005
    assert g.anchors.shape[0] == round(0.05 * 4000)
    assert len({int(i) for i, _ in g.anchors} & {int(i) for i, _ in g.test_pairs}) == 0


def test_seeded_generators_are_reproducible():
    a = synth.config_pair("cl10k", n=1500)
    b = synth.config_pair("cl10k", n=1500)
    for f in ("edges1", "edges2", "X1", "X2", "anchors", "truth", "test_pairs"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    c = synth.config_pair("cl10k", n=1500, seed=99)
    assert not np.array_equal(a.edges1, c.edges1)
