"""Launch shapes of the fused sweep against the FP64 oracle on a ragged pair
(the CUDA-core sweep: 256 threads with two CTAs per SM or 512 threads with
one; the tensor-core row pass: two 128-thread or one 256-thread CTA per SM,
4 to 8 rows per step; clusters of 1 to 16 CTAs)
(n1 = 5000, n2 = 4700 after inducing a subgraph, so the padded columns and
a partial last vector slot are exercised): two outer iterations of ten
Sinkhorn iterations each, FP32 storage (plan tolerance 1e-4) and BF16
storage (5e-2, the BF16 form's tolerance).  The shape is forced through
the planner's FA_SWEEP_* switches, which it reads at every call."""
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


SHAPES = (
    # the CUDA-core sweep (FP32 and BF16): threads per CTA x cluster size
    [("f32", {"FA_SWEEP_NT": nt, "FA_SWEEP_Q": q}) for nt in (256, 512) for q in (1, 2, 4, 8, 16)]
    + [("bf16", {"FA_SWEEP_KIND": 0, "FA_SWEEP_NT": nt, "FA_SWEEP_Q": q})
       for nt in (256, 512) for q in (1, 2, 4, 8, 16)]
    # clusters of any size: uneven column slabs
    + [("bf16", {"FA_SWEEP_KIND": 0, "FA_SWEEP_Q": q}) for q in (3, 5, 7, 9, 13)]
    + [("f32", {"FA_SWEEP_ANYQ": 1, "FA_SWEEP_Q": q}) for q in (3, 6, 11)]
    # the tensor-core row pass (BF16): CTAs per SM x cluster size x rows per step
    + [("bf16", {"FA_SWEEP_KIND": 2, "FA_SWEEP_MB": mb, "FA_SWEEP_Q": q}) for mb in (1, 2) for q in (1, 2, 4, 8, 16)]
    + [("bf16", {"FA_SWEEP_KIND": 2, "FA_SWEEP_MB": 2, "FA_SWEEP_Q": 4, "FA_SWEEP_R": r}) for r in (6, 7)]
    + [("bf16", {"FA_SWEEP_KIND": 2, "FA_SWEEP_MB": 1, "FA_SWEEP_Q": 2, "FA_SWEEP_R": r}) for r in (4, 5)]
)


@pytest.mark.parametrize("dtype,env", SHAPES,
                         ids=[f"{d}-" + "-".join(f"{k[9:]}{v}" for k, v in e.items()) for d, e in SHAPES])
def test_sweep_shape_matches_oracle(case, monkeypatch, dtype, env):
    from paper_2607_11952_gb300 import _lib as L
    from paper_2607_11952_gb300 import api
    g, Tr = case
    for k, v in env.items():
        monkeypatch.setenv(k, str(v))
    plan = L.fa_sweep_plan(g.n1, (g.n2 + 127) // 128 * 128, L.FA_BF16 if dtype == "bf16" else L.FA_F32)
    if "FA_SWEEP_MB" in env:
        if plan["kind"] != 2:
            pytest.skip(f"no tensor-core shape {env} at this width (planner chose {plan})")
        assert plan["NT"] == (128 if env["FA_SWEEP_MB"] == 2 else 256), plan
    for k, f in (("FA_SWEEP_Q", "Q"), ("FA_SWEEP_R", "R")):
        if k in env:
            assert plan[f] == env[k], plan
    al = api.Aligner(api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2),
                     api.Params(dtype=dtype))
    try:
        al.align(g.X1, g.X2, g.anchors, n_outer=2, n_sink=10)
        torch.cuda.synchronize()
        T = al.plan_f64()
    finally:
        al.close()
    rel = float(np.linalg.norm(T - Tr) / np.linalg.norm(Tr))
    assert rel <= (1e-4 if dtype == "f32" else 5e-2), (rel, plan)
