"""The fused Sinkhorn sweep (Algorithm 1, Phase 3; Eq. 3) in the launch
shape of the 50k workload, against the FP64 oracle's scaling-domain
iteration on the same kernel.

The row width is the workload's (n2 = 50,000 columns, ld = 50,048), so the
planner picks the shape bench.py times (the cluster size, column slab,
vectors per thread and the slab's ragged last vector round depend on ld,
not on n1); 2,000 rows keep the FP64 oracle quick.  K is a seeded general
kernel (entries spanning e^-10 .. 1, on the bfloat16 grid so FP32 and BF16
storage hold the same values), the start v0 a seeded column scaling.  Ten
iterations from v0: u = mu / (K v), v = nu / (K^T u).

Tolerance: the device sums each row and column in FP32 (products of exact
bf16 values with FP32 scalings): a relative error of a few 1e-6 per
iteration, which ten iterations of the contraction do not amplify
past 1e-4 -- the plan tolerance of the FP32 path (||dT||_F/||T||_F
<= 1e-4) applied to u and v themselves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastalign_ref as R  # noqa: E402
from paper_2607_11952_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

N1, N2, ITERS = 2000, 50_000, 10


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    rng = synth.rng_for(2024)
    K = synth.random_kernel_rows(N1, N2, rng)
    lv0 = synth.random_log_scalings(N2, rng)
    mu, nu = np.full(N1, 1.0 / N1), np.full(N2, 1.0 / N2)
    u, v, _ = R.sinkhorn_scaling(K.astype(np.float64), mu, nu, ITERS,
                                 v0=np.exp(lv0.astype(np.float64)), track_err=False)
    return K, lv0, u, v


def _run(K, lv0, dtype):
    from paper_2607_11952_gb300 import api
    empty = np.zeros((0, 2), np.int64)
    al = api.Aligner(api.Graph(N1, empty), api.Graph(N2, empty), api.Params(dtype=dtype))
    try:
        kt = torch.from_numpy(K).to(al.device)
        al.K.zero_()
        al.K[:, :N2].copy_(kt.to(al.K.dtype))
        al.log_v.copy_(torch.from_numpy(lv0))
        it, err, st = al.sinkhorn(ITERS)
        torch.cuda.synchronize()
        return (al.log_u.double().cpu().numpy(), al.log_v.double().cpu().numpy(),
                it, st, al.ld)
    finally:
        al.close()


@pytest.mark.parametrize("q", [0, 8, 16])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_workload_sweep_shape_matches_oracle(case, monkeypatch, dtype, q):
    """q = 0: the planner's own shape for this width (the bench's); q = 8:
    the power-of-two cluster; q = 16: the largest cluster."""
    from paper_2607_11952_gb300 import _lib as L
    K, lv0, u, v = case
    if q:
        monkeypatch.setenv("FA_SWEEP_Q", str(q))
    plan = L.fa_sweep_plan(N1, 50_048, L.FA_BF16 if dtype == "bf16" else L.FA_F32)
    lu, lv, it, st, ld = _run(K, lv0, dtype)
    assert ld == 50_048 and it == ITERS and st == 0
    du = np.abs(lu - np.log(u)).max()
    dv = np.abs(lv - np.log(v)).max()
    print(f"{dtype} plan {plan}: max |d log u| {du:.2e}, max |d log v| {dv:.2e}")
    assert du <= 1e-4 and dv <= 1e-4


# every tensor-core sweep shape on a ragged kernel: 1003 rows (a partial
# last step for every R), 4700 columns (ld 4736: a partial last column pair
# and padding columns in the last slab)
M1, M2 = 1003, 4700
MMA_SHAPES = ([{"FA_SWEEP_KIND": 2, "FA_SWEEP_MB": mb, "FA_SWEEP_Q": q} for mb in (1, 2) for q in (1, 2, 4, 8, 16)]
              + [{"FA_SWEEP_KIND": 2, "FA_SWEEP_MB": 2, "FA_SWEEP_Q": 4, "FA_SWEEP_R": r} for r in (6, 7)]
              + [{"FA_SWEEP_KIND": 2, "FA_SWEEP_MB": 1, "FA_SWEEP_Q": 2, "FA_SWEEP_R": r} for r in (4, 5)])


@pytest.fixture(scope="module")
def ragged():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    rng = synth.rng_for(2025)
    K = synth.random_kernel_rows(M1, M2, rng)
    lv0 = synth.random_log_scalings(M2, rng)
    mu, nu = np.full(M1, 1.0 / M1), np.full(M2, 1.0 / M2)
    u, v, _ = R.sinkhorn_scaling(K.astype(np.float64), mu, nu, ITERS,
                                 v0=np.exp(lv0.astype(np.float64)), track_err=False)
    return K, lv0, u, v


@pytest.mark.parametrize("env", MMA_SHAPES,
                         ids=["-".join(f"{k[9:]}{v}" for k, v in e.items()) for e in MMA_SHAPES])
def test_tensor_core_sweep_shapes_match_oracle(ragged, monkeypatch, env):
    from paper_2607_11952_gb300 import _lib as L
    from paper_2607_11952_gb300 import api
    K, lv0, u, v = ragged
    for k, val in env.items():
        monkeypatch.setenv(k, str(val))
    plan = L.fa_sweep_plan(M1, 4736, L.FA_BF16)
    if plan["kind"] != 2:
        pytest.skip(f"no tensor-core shape {env} at this width (planner chose {plan})")
    assert plan["Q"] == env["FA_SWEEP_Q"], plan
    empty = np.zeros((0, 2), np.int64)
    al = api.Aligner(api.Graph(M1, empty), api.Graph(M2, empty), api.Params(dtype="bf16"))
    try:
        al.K.zero_()
        al.K[:, :M2].copy_(torch.from_numpy(K).to(al.device).to(al.K.dtype))
        al.log_v.copy_(torch.from_numpy(lv0))
        it, err, st = al.sinkhorn(ITERS)
        torch.cuda.synchronize()
        lu, lv = al.log_u.double().cpu().numpy(), al.log_v.double().cpu().numpy()
    finally:
        al.close()
    du = np.abs(lu - np.log(u)).max()
    dv = np.abs(lv - np.log(v)).max()
    print(f"plan {plan}: max |d log u| {du:.2e}, max |d log v| {dv:.2e}")
    assert it == ITERS and st == 0
    assert du <= 1e-4 and dv <= 1e-4


# the planner's own shapes at other widths (its cluster rule picks a
# power-of-two cluster with two rows per step at 30k and 70k columns, ten
# CTAs with one row at 100k): 700 rows (a partial last step), FP64 oracle
PLANNER_WIDTHS = (30_000, 70_000, 100_000)


@pytest.mark.parametrize("n2", PLANNER_WIDTHS)
def test_planner_shapes_at_other_widths_match_oracle(monkeypatch, n2):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_11952_gb300 import _lib as L
    from paper_2607_11952_gb300 import api
    for k in ("FA_SWEEP_Q", "FA_SWEEP_R", "FA_SWEEP_NS", "FA_SWEEP_ANYQ", "FA_SWEEP_KIND"):
        monkeypatch.delenv(k, raising=False)
    n1 = 700
    rng = synth.rng_for(3000 + n2 // 1000)
    K = synth.random_kernel_rows(n1, n2, rng)
    lv0 = synth.random_log_scalings(n2, rng)
    mu, nu = np.full(n1, 1.0 / n1), np.full(n2, 1.0 / n2)
    u, v, _ = R.sinkhorn_scaling(K.astype(np.float64), mu, nu, ITERS,
                                 v0=np.exp(lv0.astype(np.float64)), track_err=False)
    empty = np.zeros((0, 2), np.int64)
    al = api.Aligner(api.Graph(n1, empty), api.Graph(n2, empty), api.Params(dtype="bf16"))
    try:
        plan = L.fa_sweep_plan(n1, al.ld, L.FA_BF16)
        al.K.zero_()
        al.K[:, :n2].copy_(torch.from_numpy(K).to(al.device).to(al.K.dtype))
        al.log_v.copy_(torch.from_numpy(lv0))
        it, err, st = al.sinkhorn(ITERS)
        torch.cuda.synchronize()
        lu, lv = al.log_u.double().cpu().numpy(), al.log_v.double().cpu().numpy()
    finally:
        al.close()
    expect = {30_000: (4, 2), 70_000: (8, 2), 100_000: (10, 1)}[n2]
    assert (plan["Q"], plan["R"]) == expect, plan
    assert it == ITERS and st == 0
    du = np.abs(lu - np.log(u)).max()
    dv = np.abs(lv - np.log(v)).max()
    print(f"n2 {n2} plan {plan}: max |d log u| {du:.2e}, max |d log v| {dv:.2e}")
    assert du <= 1e-4 and dv <= 1e-4
