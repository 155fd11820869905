"""Launch shapes of the fused sweep (256 threads with two CTAs per SM or 512
threads with one; clusters of 1 to 16 CTAs) against the FP64 oracle on a ragged pair
(n1 = 5000, n2 = 4700 after inducing a subgraph, so the padded columns and
a partial last vector slot are exercised): two outer iterations of ten
Sinkhorn iterations each, FP32 storage (plan tolerance 1e-4) and BF16
storage (5e-2, the BF16 form's tolerance).  The shape is forced through
the planner's FA_SWEEP_NT / FA_SWEEP_Q switches, which it reads at every
call."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastalign_ref as R  # noqa: E402
from paper_2607_11952_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    rng = synth.rng_for(91)
    e1 = synth.chung_lu(5000, 2.3, 8.0, rng)
    g = synth.make_pair(e1, 5000, d=32, sigma=0.1, anchor_frac=0.05, frac_del=0.1,
                        frac_add=0.1, rng=rng, keep_nodes=4700)
    ref = R.fastalign(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors,
                      R.Params(), 2, 10)
    return g, np.exp(ref["logS"])


@pytest.mark.parametrize("nt", [256, 512])
@pytest.mark.parametrize("q", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_sweep_shape_matches_oracle(case, monkeypatch, nt, q, dtype):
    from paper_2607_11952_gb300 import api
    g, Tr = case
    monkeypatch.setenv("FA_SWEEP_NT", str(nt))
    monkeypatch.setenv("FA_SWEEP_Q", str(q))
    al = api.Aligner(api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2),
                     api.Params(dtype=dtype))
    try:
        al.align(g.X1, g.X2, g.anchors, n_outer=2, n_sink=10)
        torch.cuda.synchronize()
        T = al.plan_f64()
    finally:
        al.close()
    rel = float(np.linalg.norm(T - Tr) / np.linalg.norm(Tr))
    assert rel <= (1e-4 if dtype == "f32" else 5e-2), rel
