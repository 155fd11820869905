"""The learned warm start's kernels (through the C ABI) against the FP64
oracle: forward pass, gradient, one Adam step; and the gain of a trained
model over the cold start."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastalign_ref as R  # noqa: E402
from oracle import gnn_ref as G  # noqa: E402
from paper_2607_11952_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _case(n=700, seed=3):
    from paper_2607_11952_gb300 import api, gnn
    rng = synth.rng_for(seed)
    e = synth.chung_lu(n, 2.3, 6.0, rng)
    F = rng.standard_normal((n, G.FIN)).astype(np.float32)
    y = rng.standard_normal(n).astype(np.float32)
    theta = gnn.init_params(seed)
    return api.Graph(n, e), e, F, y, theta


def test_forward_and_gradient_match_oracle():
    from paper_2607_11952_gb300 import gnn
    graph, e, F, y, theta = _case()
    n = graph.n
    m = gnn.WarmStartModel(theta)
    Fd, yd = torch.from_numpy(F).cuda(), torch.from_numpy(y).cuda()
    a = m.predict(graph, Fd)
    from paper_2607_11952_gb300 import _lib as L
    L.fa_gnn_backward(m.h, graph.handle, m.ws(n), a, yd, m.grad, m.loss)
    torch.cuda.synchronize()
    A = R.row_normalized(n, e)
    a_ref, _ = G.forward(A, F.astype(np.float64), theta.astype(np.float64))
    loss_ref, g_ref = G.backward(A, F.astype(np.float64), theta.astype(np.float64), y)
    np.testing.assert_allclose(a.cpu().numpy(), a_ref, rtol=1e-5, atol=1e-5)
    assert abs(m.loss.item() - loss_ref) <= 1e-5 * loss_ref
    g = m.grad.cpu().numpy().astype(np.float64)
    scale = np.abs(g_ref[:-1]).max()
    np.testing.assert_allclose(g[:-1], g_ref[:-1], rtol=0, atol=2e-5 * scale)
    assert abs(g[-1]) < 1e-4


def test_adam_step_matches_oracle():
    from paper_2607_11952_gb300 import gnn
    graph, e, F, y, theta = _case(seed=4)
    m = gnn.WarmStartModel(theta)
    Fd, yd = torch.from_numpy(F).cuda(), torch.from_numpy(y).cuda()
    m.train_step(graph, Fd, yd, lr=1e-2)
    torch.cuda.synchronize()
    g = m.grad.cpu().numpy().astype(np.float64)
    th_ref, _, _ = G.adam_step(theta.astype(np.float64), np.zeros(G.N_PARAMS), np.zeros(G.N_PARAMS),
                               g, 1, lr=1e-2)
    np.testing.assert_allclose(m.params(), th_ref, rtol=0, atol=1e-6)


def test_training_reduces_loss():
    from paper_2607_11952_gb300 import gnn
    graph, e, F, y, theta = _case(seed=5)
    # a target the model can represent: a smooth function of the features
    A = R.row_normalized(graph.n, e)
    y = (A @ np.tanh(F[:, 0] + 0.5 * F[:, 2])).astype(np.float32)
    m = gnn.WarmStartModel(theta)
    Fd, yd = torch.from_numpy(F).cuda(), torch.from_numpy(y).cuda()
    first = m.train_step(graph, Fd, yd, lr=5e-3).item()
    for _ in range(300):
        last = m.train_step(graph, Fd, yd, lr=5e-3)
    assert last.item() < 0.5 * first


def test_trained_warm_start_beats_cold_start():
    """The committed trained model, on a fresh 5k pair it never saw: the
    same Gibbs kernel of every outer iteration is solved to 1e-4 from the
    cold start and from the learned warm start; the learned start must need
    fewer Sinkhorn iterations in total."""
    import os
    from paper_2607_11952_gb300 import api, gnn
    if not os.path.exists(gnn.WEIGHTS_PATH):
        pytest.skip("no trained weights")
    model = gnn.WarmStartModel.load(gnn.WEIGHTS_PATH)
    g = synth.config_pair("cl50k_5k", seed=11)
    al = api.Aligner(api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2), api.Params(dtype="bf16"))
    al.node_cost(g.X1, g.X2, g.anchors)
    al.plan_init()
    ws = gnn.WarmStarter(al, "learned", model)
    K0, u0, v0 = torch.empty_like(al.K), torch.empty_like(al.log_u), torch.empty_like(al.log_v)
    tot = {"cold": 0, "learned": 0}
    for t in range(6):
        al.align_iter()
        K0.copy_(al.K), u0.copy_(al.log_u), v0.copy_(al.log_v)
        it_c, _, st_c = al.sinkhorn(20000, 1e-4, 5)
        al.K.copy_(K0), al.log_u.copy_(u0), al.log_v.copy_(v0)
        it_l, _, st_l, _ = ws.solve(20000, 1e-4, 5)
        tot["cold"] += it_c
        tot["learned"] += it_l
    print("sweeps to 1e-4 over 6 outer iterations:", tot)
    assert tot["learned"] < tot["cold"]


def test_trained_network_beats_previous_correction_start():
    """What the trained network adds over the method without it: on a fresh
    5k pair, every outer iteration's Gibbs kernel is solved to 1e-4 three
    times -- cold start, the previous-correction start (the network's base,
    log v1 + c_prev, with f = 0) and the learned start (base + f) -- and the
    learned start must need fewer Sinkhorn iterations in total than the
    previous-correction start."""
    import os
    from paper_2607_11952_gb300 import api, gnn
    if not os.path.exists(gnn.WEIGHTS_PATH):
        pytest.skip("no trained weights")
    model = gnn.WarmStartModel.load(gnn.WEIGHTS_PATH)
    g = synth.config_pair("cl50k_5k", seed=11)
    al = api.Aligner(api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2), api.Params(dtype="bf16"))
    al.node_cost(g.X1, g.X2, g.anchors)
    al.plan_init()
    prev = gnn.WarmStarter(al, "prev")
    learned = gnn.WarmStarter(al, "learned", model)
    K0, u0, v0 = torch.empty_like(al.K), torch.empty_like(al.log_u), torch.empty_like(al.log_v)
    tot = {"cold": 0, "prev": 0, "learned": 0}
    per = []
    for t in range(10):
        al.align_iter()
        K0.copy_(al.K), u0.copy_(al.log_u), v0.copy_(al.log_v)
        it_c, _, _ = al.sinkhorn(20000, 1e-4, 5)
        al.K.copy_(K0), al.log_u.copy_(u0), al.log_v.copy_(v0)
        it_p, _, _, _ = prev.solve(20000, 1e-4, 5)
        al.K.copy_(K0), al.log_u.copy_(u0), al.log_v.copy_(v0)
        it_l, _, _, _ = learned.solve(20000, 1e-4, 5)
        tot["cold"] += it_c
        tot["prev"] += it_p
        tot["learned"] += it_l
        per.append((it_c, it_p, it_l))
    al.close()
    print("sweeps to 1e-4 over 10 outer iterations:", tot, "per outer (cold, prev, learned):", per)
    assert tot["learned"] < tot["prev"] < tot["cold"]


@pytest.mark.parametrize("first", [False, True])
def test_features_match_oracle(first):
    """Inputs of the model: the centred cold column update, previous
    correction and previous potential, log(1 + degree), the anchor flag and
    the outer-iteration index, against the oracle's; first = True is the
    first solve (no previous state given)."""
    from paper_2607_11952_gb300 import gnn
    graph, e, F, y, theta = _case(n=900, seed=6)
    rng = np.random.default_rng(6)
    lv1 = (rng.standard_normal(graph.n) - 9.0).astype(np.float32)
    corr = (rng.standard_normal(graph.n) + 3.0).astype(np.float32)
    pot = (rng.standard_normal(graph.n) - 4.0).astype(np.float32)
    mask = (rng.random(graph.n) < 0.05).astype(np.float32)
    m = gnn.WarmStartModel(theta)
    dev = lambda x: torch.from_numpy(x).cuda()   # noqa: E731
    if first:
        got = m.features(graph, dev(lv1), None, None, None, 0)
        want = G.features(np.bincount(e.ravel(), minlength=graph.n), lv1, np.zeros(graph.n))
    else:
        got = m.features(graph, dev(lv1), dev(corr), dev(pot), dev(mask), 7)
        want = G.features(np.bincount(e.ravel(), minlength=graph.n), lv1, corr, pot, mask, 7)
    np.testing.assert_allclose(got.cpu().numpy(), want, rtol=1e-5, atol=1e-5)


def test_fit_scale_matches_oracle():
    """The trust fit of the learned warm start (the clamped prediction's
    least-squares scale against the observed change, clipped to [0, 1])."""
    from paper_2607_11952_gb300 import _lib as L
    rng = np.random.default_rng(12)
    n = 5001
    pred = (3.0 * rng.standard_normal(n)).astype(np.float32)
    pred[7] = np.inf
    for k in (0.3, 1.7, -0.4):
        y = (k * np.clip(pred, -2.0, 2.0) * np.isfinite(pred) + 0.7 * rng.standard_normal(n)
             + 5.0).astype(np.float32)
        for shrink in (0, 1, 2):
            out = torch.zeros(1, device="cuda")
            L.fa_gnn_fit_scale(n, torch.from_numpy(pred).cuda(), torch.from_numpy(y).cuda(), 2.0,
                               out, shrink=shrink)
            want = G.fit_scale(pred.astype(np.float64), y.astype(np.float64), 2.0, shrink=shrink)
            assert abs(out.item() - want) <= 1e-6, (k, shrink, out.item(), want)
