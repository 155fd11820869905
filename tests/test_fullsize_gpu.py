"""Full-size checks at the 50k Chung-Lu workload, in the launch
configuration bench.py times (default sweep shape, BF16 kernel storage, the
learned warm start), through the C ABI.

* Sampled rows (the five highest-degree hubs among them) of the first
  outer iteration's row-stabilised Gibbs kernel (Phases 1-2 of Algorithm 1
  from the independent coupling) against the FP64 row oracle
  (oracle/rows_ref.py), FP32 and BF16 storage.
* The same rows of an outer iteration whose previous plan is a seeded
  general one (T_prev = diag(u) K diag(v) with K spanning e^-10 .. 1), so
  Pass A and Pass B gather a full-rank plan, against the row oracle's
  general-plan form.
* Sinkhorn to 1e-4 (Eq. 3): row and column marginals recomputed
  independently in float64 from the stored K and the potentials; the
  reported error must match them and meet the tolerance.
* Top-10 of sampled rows against an exact float64 sort of the same plan rows.
* The learned warm start converges to the plan the cold start reaches.

Tolerances (derived from the arithmetic, not fitted):
* FP32 storage: |x| = |C_eff / eps| <= ~100 computed in FP32 with a 3xTF32
  node-similarity GEMM, |dC| <= 1e-5, so |dx| <= 2e-4 and
  |dK| <= 5e-4 K + 1e-6 (the absolute term covers FP32 underflow of exp).
* BF16 storage: the oracle takes the node-similarity operands rounded to
  bfloat16 (the BF16 form), leaving FP32 accumulation of exact bf16
  products and the bf16 rounding of K (2^-9 relative): |dK| <= 5e-3 K + 1e-6.
* Marginals: the device sums K v in FP32, so each row sum carries a
  relative error of a few 1e-6: |S 1 - mu|_1 <= 1e-5; the reported column
  error equals the float64 one to 1e-3 relative + 1e-6 (ERR_FLOOR).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastalign_ref as R  # noqa: E402
from oracle import rows_ref  # noqa: E402
from paper_2607_11952_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
ERR_FLOOR = 1e-6


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    g = synth.config_pair("cl50k")
    p = R.Params()
    st = rows_ref.prepare(g.n1, g.n2, g.edges1, g.edges2, g.X1, g.X2, g.anchors, p)
    deg = np.diff(st.A1.indptr)
    rng = np.random.default_rng(5)
    rows = list(rng.choice(np.flatnonzero(deg <= 40), 6, replace=False))
    anc = [int(i) for i, _ in g.anchors if deg[int(i)] <= 40][:1]
    # the five highest-degree rows: the hubs of the heavy-tailed degree
    # distribution, where the edge-balanced split of the sparse products
    # spreads one row's neighbours over many warps
    hubs = [int(i) for i in np.argsort(-deg, kind="stable")[:5]]
    rows = [int(r) for r in rows] + anc + hubs + [g.n1 - 1]
    return g, p, st, rows


def _aligner(g, dtype):
    from paper_2607_11952_gb300 import api
    return api.Aligner(api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2),
                       api.Params(dtype=dtype))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_first_iteration_kernel_rows_50k(setup, dtype):
    g, p, st, rows = setup
    al = _aligner(g, dtype)
    try:
        al.node_cost(g.X1, g.X2, g.anchors)
        al.plan_init()
        al.align_iter()
        idx = torch.tensor(rows, device=al.device)
        Kg = al.K.index_select(0, idx)[:, : g.n2].double().cpu().numpy()
    finally:
        al.close()
    Kr = rows_ref.first_kernel_rows_from(st, g.anchors, p, rows,
                                         "f64" if dtype == "f32" else "bf16")
    rel = 5e-4 if dtype == "f32" else 5e-3
    err = np.abs(Kg - Kr)
    worst = float((err / (rel * Kr + 1e-6)).max())
    print(f"{dtype}: max |dK| {err.max():.3e}, worst / bound {worst:.3f}")
    assert worst <= 1.0
    # every row is stabilised: its largest entry is exactly 1
    np.testing.assert_array_equal(Kg.max(axis=1), 1.0)


@pytest.fixture(scope="module")
def general_plan(setup):
    """A seeded general previous plan at full size: K (bf16 grid, 5 GB as
    bfloat16 on the host) and the log-scalings."""
    g, p, st, rows = setup
    ld = (g.n2 + 127) // 128 * 128
    rng = synth.rng_for(4242)
    K = torch.zeros((g.n1, ld), dtype=torch.bfloat16)
    for i0 in range(0, g.n1, 2000):
        blk = synth.random_kernel_rows(min(2000, g.n1 - i0), g.n2, rng)
        K[i0:i0 + blk.shape[0], : g.n2] = torch.from_numpy(blk).to(torch.bfloat16)
    lu = synth.random_log_scalings(g.n1, rng)
    lv = synth.random_log_scalings(g.n2, rng)
    return K, lu, lv


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_general_plan_kernel_rows_50k(setup, general_plan, dtype):
    g, p, st, rows = setup
    K, lu, lv = general_plan
    al = _aligner(g, dtype)
    try:
        al.node_cost(g.X1, g.X2, g.anchors)
        for i0 in range(0, g.n1, 5000):
            al.K[i0:i0 + 5000].copy_(K[i0:i0 + 5000].to(al.device).to(al.K.dtype))
        al.log_u.copy_(torch.from_numpy(lu))
        al.log_v.copy_(torch.from_numpy(lv))
        al.align_iter()
        idx = torch.tensor(rows, device=al.device)
        Kg = al.K.index_select(0, idx)[:, : g.n2].double().cpu().numpy()
    finally:
        al.close()
    u = np.exp(lu.astype(np.float64))
    v = np.exp(lv.astype(np.float64))

    def plan_rows(ks):
        ks = np.asarray(ks, dtype=np.int64)
        Kk = K[torch.from_numpy(ks), : g.n2].double().numpy()
        return u[ks, None] * Kk * v[None, :]

    Kr = rows_ref.kernel_rows_from_plan(st, g.anchors, p, rows, plan_rows,
                                        "f64" if dtype == "f32" else "bf16")
    rel = 5e-4 if dtype == "f32" else 5e-3
    err = np.abs(Kg - Kr)
    worst = float((err / (rel * Kr + 1e-6)).max())
    print(f"{dtype}: max |dK| {err.max():.3e}, worst / bound {worst:.3f}")
    assert worst <= 1.0
    np.testing.assert_array_equal(Kg.max(axis=1), 1.0)


@pytest.fixture(scope="module")
def solved(setup):
    """The bench step's path on the 50k pair: BF16 storage, Phase 1, two
    outer iterations with the learned warm start, Sinkhorn to 1e-4."""
    from paper_2607_11952_gb300 import gnn
    g, p, st, rows = setup
    al = _aligner(g, "bf16")
    model = gnn.WarmStartModel.load(gnn.WEIGHTS_PATH, device=al.device)
    al.node_cost(g.X1, g.X2, g.anchors)
    al.plan_init()
    ws = gnn.WarmStarter(al, "learned", model)
    res = None
    for _ in range(2):
        al.align_iter()
        res = ws.solve(5000, 1e-4, 5)
    torch.cuda.synchronize()
    yield g, al, res
    al.close()


def _marginals(al, block=2048):
    """Row and column sums of S = diag(u) K diag(v) in float64."""
    u = torch.exp(al.log_u.double())
    v = torch.exp(al.log_v.double())
    rsum = torch.empty(al.n1, dtype=torch.float64, device=al.device)
    csum = torch.zeros(al.n2, dtype=torch.float64, device=al.device)
    for i0 in range(0, al.n1, block):
        Kb = al.K[i0:i0 + block, : al.n2].double()
        rsum[i0:i0 + block] = u[i0:i0 + block] * (Kb @ v)
        csum += (u[i0:i0 + block, None] * Kb).sum(dim=0)
    csum *= v
    return rsum, csum


def test_sinkhorn_marginals_50k(solved):
    g, al, (it, err, st, fell_back) = solved
    rsum, csum = _marginals(al)
    row_err = float((rsum - 1.0 / al.n1).abs().sum())
    col_err = float((csum - 1.0 / al.n2).abs().sum())
    print(f"iterations {it}, reported {err:.3e}, column {col_err:.3e}, row {row_err:.3e}")
    assert st == 0 and not fell_back
    assert row_err <= 1e-5
    assert abs(err - col_err) <= 1e-3 * col_err + ERR_FLOOR
    assert col_err <= 1e-4 + ERR_FLOOR


def test_topk_sampled_rows_50k(solved):
    g, al, _ = solved
    idx, score = al.topk(10)
    rows = torch.tensor([0, 17, 4242, 31337, al.n1 - 1], device=al.device)
    v = torch.exp(al.log_v.double())
    T = al.K.index_select(0, rows)[:, : al.n2].double() * v[None, :]
    srt, order = torch.sort(T, dim=1, descending=True, stable=True)
    got = idx.index_select(0, rows).long()
    for r in range(rows.shape[0]):
        gap = ((srt[r, :10] - srt[r, 1:11]) / srt[r, 0] > 1e-5)
        before = torch.cat([torch.ones(1, dtype=torch.bool, device=gap.device), gap[:9]])
        # every position separated from both neighbours holds the exact column
        clear = gap & before
        ok = (got[r] == order[r, :10]) | ~clear
        assert bool(ok.all()), (int(rows[r]), got[r].tolist(), order[r, :10].tolist())


def test_learned_and_cold_reach_the_same_plan_50k(setup):
    """Eq. 3 has one fixed point: the warm start only changes the path to
    it.  After the same outer iteration solved to 1e-5 from the learned and
    from the cold start, the plans' sampled rows agree to the stopping
    tolerance."""
    from paper_2607_11952_gb300 import gnn, _lib as L
    g, p, st, rows = setup
    al = _aligner(g, "bf16")
    try:
        model = gnn.WarmStartModel.load(gnn.WEIGHTS_PATH, device=al.device)
        al.node_cost(g.X1, g.X2, g.anchors)
        al.plan_init()
        al.align_iter()
        v1 = al.log_v.clone()
        ws = gnn.WarmStarter(al, "learned", model)
        it_l, err_l, _, _ = ws.solve(8000, 1e-5, 5)
        lu_l, lv_l = al.log_u.clone(), al.log_v.clone()
        L.fa_vec_axpby(al.n2, 1.0, v1, 0.0, None, al.log_v)
        it_c, err_c, _ = al.sinkhorn(8000, 1e-5, 5)
        lu_c, lv_c = al.log_u.clone(), al.log_v.clone()
        sel = torch.tensor(rows, device=al.device)
        K = al.K.index_select(0, sel)[:, : al.n2].double()
        Tl = torch.exp(lu_l.double()[sel, None]) * K * torch.exp(lv_l.double())[None, :]
        Tc = torch.exp(lu_c.double()[sel, None]) * K * torch.exp(lv_c.double())[None, :]
        d = float((Tl - Tc).abs().sum() / Tc.abs().sum())
        print(f"learned {it_l} sweeps, cold {it_c} sweeps, relative plan difference {d:.2e}")
        assert err_l <= 1e-5 + ERR_FLOOR and err_c <= 1e-5 + ERR_FLOOR
        assert d <= 1e-3
    finally:
        al.close()


def test_largest_uneven_pair_100k_by_80k():
    """The largest workload (G2 an induced 80k subgraph of a 100k graph,
    256-dim attributes, 2% anchors): Phase 1, one outer iteration and
    Sinkhorn to 1e-4 with BF16 storage; row and column marginals of the
    unequal masses mu = 1/n1, nu = 1/n2 recomputed in float64."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    g = synth.config_pair("cl100k")
    assert (g.n1, g.n2) == (100_000, 80_000)
    al = _aligner(g, "bf16")
    try:
        al.node_cost(g.X1, g.X2, g.anchors)
        al.plan_init()
        al.align_iter()
        it, err, st = al.sinkhorn(5000, 1e-4, 5)
        torch.cuda.synchronize()
        rsum, csum = _marginals(al)
        row_err = float((rsum - 1.0 / al.n1).abs().sum())
        col_err = float((csum - 1.0 / al.n2).abs().sum())
        print(f"100k x 80k: {it} sweeps, reported {err:.3e}, column {col_err:.3e}, row {row_err:.3e}")
        assert st == 0
        assert row_err <= 1e-5
        assert abs(err - col_err) <= 1e-3 * col_err + ERR_FLOOR
        assert col_err <= 1e-4 + ERR_FLOOR
        assert bool(torch.isfinite(al.log_u).all()) and bool(torch.isfinite(al.log_v).all())
    finally:
        al.close()
