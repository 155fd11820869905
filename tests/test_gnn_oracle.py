"""Pins for the FP64 oracle of the learned warm start: analytic gradients
against central finite differences, gauge invariance, a hand-sized forward
pass and the Adam closed form for a constant gradient.  CPU only."""
import numpy as np

from oracle import fastalign_ref as R
from oracle import gnn_ref as G
from paper_2607_11952_gb300 import synth


def _setup(n=40, seed=0):
    rng = np.random.default_rng(seed)
    e = synth.erdos_renyi(n, 3.0, synth.rng_for(seed))
    A = R.row_normalized(n, e)
    F = rng.standard_normal((n, G.FIN))
    y = rng.standard_normal(n)
    theta = 0.3 * rng.standard_normal(G.N_PARAMS)
    return A, F, y, theta


def test_gradient_matches_central_differences():
    A, F, y, theta = _setup()
    L, g = G.backward(A, F, theta, y)
    h = 1e-6
    num = np.empty_like(theta)
    for k in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        num[k] = (G.loss(G.forward(A, F, tp)[0], y) - G.loss(G.forward(A, F, tm)[0], y)) / (2 * h)
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-8)
    assert abs(g[-1]) < 1e-12          # the bias c does not change a centred loss


def test_loss_is_gauge_invariant():
    A, F, y, theta = _setup(seed=1)
    a, _ = G.forward(A, F, theta)
    assert abs(G.loss(a, y) - G.loss(a + 3.7, y - 1.2)) < 1e-12


def test_forward_hand_example():
    # path 0-1-2; W1 picks feature 0 into unit 0; w2 = e_0; c = 0.5
    A = R.row_normalized(3, np.array([[0, 1], [1, 2]]))
    F = np.zeros((3, G.FIN))
    F[:, 0] = [1.0, -2.0, 3.0]
    theta = np.zeros(G.N_PARAMS)
    theta[0] = 1.0                       # W1[0, 0]
    theta[G.FIN * G.HIDDEN + G.HIDDEN] = 1.0   # w2[0]
    theta[-1] = 0.5
    a, c = G.forward(A, F, theta)
    # AF[:,0] = (-2, 2, -2); relu -> (0, 2, 0); a = Abar z2 + .5 = (2.5, .5, 2.5)
    np.testing.assert_allclose(a, [2.5, 0.5, 2.5])


def test_adam_constant_gradient_closed_form():
    theta = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    g = np.array([1.0, -2.0, 0.5, 0.0])
    for t in range(1, 6):
        theta, m, v = G.adam_step(theta, m, v, g, t, lr=0.1)
    # with a constant gradient the bias-corrected step is lr * sign(g)
    np.testing.assert_allclose(theta, -0.5 * np.sign(g) * (g != 0), atol=1e-7)


def test_features_hand_values():
    # degrees (0, 1, 3); log v1 (1, 2, 6) has mean 3; c_prev (0.5, 0.5, 2)
    # has mean 1; previous potential (-1, 0, 4) has mean 1; node 1 is an
    # anchor's partner; two outer iterations done
    F = G.features(np.array([0, 1, 3]), np.array([1.0, 2.0, 6.0]),
                   np.array([0.5, 0.5, 2.0]), np.array([-1.0, 0.0, 4.0]),
                   np.array([0.0, 1.0, 0.0]), 2)
    want = np.array([[-2.0, -0.5, 0.0, -2.0, 0.0, np.log(3.0)],
                     [-1.0, -0.5, np.log(2.0), -1.0, 1.0, np.log(3.0)],
                     [3.0, 1.0, np.log(4.0), 3.0, 0.0, np.log(3.0)]])
    np.testing.assert_allclose(F, want, rtol=0, atol=1e-15)
    # the first solve: no previous correction, potential or anchors given
    F0 = G.features(np.array([2]), np.array([5.0]), np.array([0.0]))
    np.testing.assert_array_equal(F0, [[0.0, 0.0, np.log(3.0), 0.0, 0.0, 0.0]])


def test_fit_scale_hand_values():
    p = np.array([1.0, 2.0, 3.0, 6.0])
    # y = k p + c: the centred fit recovers k, clipped to [0, 1]
    assert G.fit_scale(p, 0.5 * p + 7.0, 20.0) == 0.5
    assert G.fit_scale(p, 3.0 * p, 20.0) == 1.0
    assert G.fit_scale(p, -p, 20.0) == 0.0
    assert G.fit_scale(np.full(4, 2.0), p, 20.0) == 0.0          # constant prediction
    # the clamp applies first: p = (1, 2, 2, 2) against y = p
    assert abs(G.fit_scale(p, np.array([1.0, 2.0, 2.0, 2.0]), 2.0) - 1.0) < 1e-15
    # a non-finite prediction counts as 0
    q = np.array([1.0, np.nan, 3.0, -1.0])
    want = G.fit_scale(np.array([1.0, 0.0, 3.0, -1.0]), np.array([0.2, 0.0, 0.6, -0.2]), 20.0)
    assert abs(G.fit_scale(q, np.array([0.2, 0.0, 0.6, -0.2]), 20.0) - want) < 1e-15
    assert abs(want - 0.2) < 1e-15


def test_fit_scale_shrink_is_alpha_times_a_power_of_the_correlation():
    p = np.array([1.0, 2.0, 3.0, 6.0])
    noise = np.array([0.3, -0.6, 0.3, 0.0])          # centred, orthogonal to the centred p
    y = 0.5 * p + noise
    dp = p - p.mean()
    rho2 = (dp @ (y - y.mean())) ** 2 / ((dp @ dp) * ((y - y.mean()) @ (y - y.mean())))
    assert abs(G.fit_scale(p, y, 20.0) - 0.5) < 1e-15
    assert abs(G.fit_scale(p, y, 20.0, shrink=1) - 0.5 * rho2) < 1e-15
    assert abs(G.fit_scale(p, y, 20.0, shrink=2) - 0.5 * np.sqrt(rho2)) < 1e-15
    assert 0.0 < rho2 < 1.0
    # hand value: dp = (-2, -1, 0, 3), dp.dp = 14, dy = 0.5 dp + noise,
    # dy.dy = 3.5 + 0.54 = 4.04, (dp.dy)^2 = 49, rho^2 = 49 / (14 * 4.04)
    assert abs(rho2 - 49.0 / (14.0 * 4.04)) < 1e-14
    for mode in (1, 2):
        assert G.fit_scale(p, 0.5 * p, 20.0, shrink=mode) == 0.5   # exact fit: rho^2 = 1
