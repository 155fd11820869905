"""The outer loop's convergence test and checkpoint/resume, through the C
ABI on the GPU.

* fa_plan_change on two plans the FP64 oracle produced (consecutive outer
  iterations, uploaded as K = exp(log S - row max), log u = row max,
  log v = 0) against the oracle's plan_l1 of the same plans.  Each element
  is formed in float32 (relative error a few 2^-24) and the differences are
  summed in float64: |error| <= 1e-5 of the sum + 1e-7.
* align(plan_tol=...) stops at the first outer iteration whose plan change
  is <= plan_tol; the plan it returns matches the oracle run for that many
  outer iterations (1e-4), and the changes it reports match the oracle's
  plan changes (1e-3 relative, the plans' own parity tolerance propagated).
* An alignment interrupted after 2 of 4 outer iterations and resumed from
  its checkpoint ends with exactly the plan of the uninterrupted run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastalign_ref as R  # noqa: E402
from paper_2607_11952_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    return synth.config_pair("ba1k", n=300)


def _aligner(g, dtype="f32"):
    from paper_2607_11952_gb300 import api
    return api.Aligner(api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2),
                       api.Params(dtype=dtype))


def _upload(al, logS, K):
    """A plan given as log S in the library's (K, log u, log v) form."""
    m = logS.max(axis=1)
    Kh = np.zeros((al.n1, al.ld))
    Kh[:, : al.n2] = np.exp(logS - m[:, None])
    K.copy_(torch.from_numpy(Kh).to(K.dtype))
    lu = torch.from_numpy(m.astype(np.float32)).cuda()
    lv = torch.zeros(al.n2, dtype=torch.float32, device="cuda")
    return lu, lv


def test_plan_change_matches_oracle(small):
    g = small
    p = R.Params()
    ph = R.phase1(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p)
    a = R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p, 2, 30, ph=ph)
    b = R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p, 3, 30, ph=ph)
    want = R.plan_l1(a["logS"], b["logS"])
    al = _aligner(g)
    try:
        Kb = torch.empty_like(al.K)
        lu_a, lv_a = _upload(al, a["logS"], al.K)
        lu_b, lv_b = _upload(al, b["logS"], Kb)
        al.log_u.copy_(lu_a)
        al.log_v.copy_(lv_a)
        got = al.plan_change(Kb, lu_b, lv_b)
        same = al.plan_change(al.K, al.log_u, al.log_v)
    finally:
        al.close()
    print(f"plan change: device {got:.9e}, oracle {want:.9e}")
    assert abs(got - want) <= 1e-5 * want + 1e-7
    assert same == 0.0


def test_convergence_driven_outer_loop(small):
    g = small
    p = R.Params()
    al = _aligner(g)
    try:
        hist = al.align(g.X1, g.X2, g.anchors, n_outer=40, n_sink=30, plan_tol=2e-3)
        T = al.plan_f64()
    finally:
        al.close()
    changes = [h[3] for h in hist]
    n = len(hist)
    print("plan changes:", ["%.2e" % c for c in changes])
    assert 1 < n < 40
    assert changes[-1] <= 2e-3 and all(c > 2e-3 for c in changes[:-1])
    ph = R.phase1(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p)
    ref = [R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p, k, 30,
                       ph=ph)["logS"] for k in range(n + 1)[-3:]]
    Tr = np.exp(ref[-1])
    assert np.linalg.norm(T - Tr) / np.linalg.norm(Tr) <= 1e-4
    for k in (1, 2):
        want = R.plan_l1(ref[k - 1], ref[k])
        got = changes[n - 3 + k]
        assert abs(got - want) <= 1e-3 * want + 1e-6, (k, got, want)


@pytest.mark.parametrize("mode", ["cold", "prev", "learned"])
def test_checkpoint_resume_reproduces_the_run(small, tmp_path, mode):
    """A run interrupted after 2 of 4 outer iterations and resumed from its
    checkpoint ends with the uninterrupted run's plan, bit for bit, with
    the cold start and with both warm starts (whose carried correction is
    part of the checkpoint)."""
    from paper_2607_11952_gb300 import gnn
    g = small
    path = str(tmp_path / "align.ckpt")
    model = gnn.WarmStartModel.load(gnn.WEIGHTS_PATH) if mode == "learned" else None

    def starter(al):
        return None if mode == "cold" else gnn.WarmStarter(al, mode, model)

    a = _aligner(g, "bf16")
    try:
        a.align(g.X1, g.X2, g.anchors, n_outer=2, n_sink=20, tol=1e-6, check_every=5,
                warm=starter(a), checkpoint=path)
    finally:
        a.close()
    b = _aligner(g, "bf16")
    try:
        hist = b.align(g.X1, g.X2, g.anchors, n_outer=4, n_sink=20, tol=1e-6,
                       check_every=5, warm=starter(b), resume=path)
        Tb = b.plan_f64()
    finally:
        b.close()
    c = _aligner(g, "bf16")
    try:
        hc = c.align(g.X1, g.X2, g.anchors, n_outer=4, n_sink=20, tol=1e-6,
                     check_every=5, warm=starter(c))
        Tc = c.plan_f64()
    finally:
        c.close()
    assert len(hist) == 2
    assert [h[0] for h in hist] == [h[0] for h in hc[2:]]
    np.testing.assert_array_equal(Tb, Tc)
