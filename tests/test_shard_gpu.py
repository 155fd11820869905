"""The column-sharded Sinkhorn iteration (the data path of a sweep whose
columns are split over devices), on one device: the same seeded kernel run
as one column range, two ranges and three ranges gives bit-identical
scalings; they match the FP64 oracle's scaling-domain iteration to the FP32
path's tolerance and the fused sweep to FP32 rounding.  FP32 and BF16
storage; 1,500 rows, 9,000 columns (ld 9,088: a last block of 896 columns
and padding)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastalign_ref as R  # noqa: E402
from paper_2607_11952_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
N1, N2, ITERS = 1500, 9000, 8


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    rng = synth.rng_for(2026)
    K = synth.random_kernel_rows(N1, N2, rng)
    lv0 = synth.random_log_scalings(N2, rng)
    mu, nu = np.full(N1, 1.0 / N1), np.full(N2, 1.0 / N2)
    u, v, _ = R.sinkhorn_scaling(K.astype(np.float64), mu, nu, ITERS,
                                 v0=np.exp(lv0.astype(np.float64)), track_err=False)
    return K, lv0, u, v


def _aligner(dtype, K, lv0):
    from paper_2607_11952_gb300 import api
    empty = np.zeros((0, 2), np.int64)
    al = api.Aligner(api.Graph(N1, empty), api.Graph(N2, empty), api.Params(dtype=dtype))
    al.K.zero_()
    al.K[:, :N2].copy_(torch.from_numpy(K).to(al.device).to(al.K.dtype))
    al.log_v.copy_(torch.from_numpy(lv0))
    return al


def _sharded(dtype, K, lv0, cuts):
    """ITERS iterations through the sharded calls; cuts: the range bounds."""
    from paper_2607_11952_gb300 import _lib as L
    al = _aligner(dtype, K, lv0)
    try:
        ld = al.ld
        bounds = [0] + list(cuts) + [ld]
        parts = torch.full((L.fa_shard_blocks(ld), N1), float("nan"), device=al.device)
        lv, lv_next = al.log_v.clone(), torch.empty_like(al.log_v)
        for _ in range(ITERS):
            for j0, j1 in zip(bounds[:-1], bounds[1:]):
                L.fa_sinkhorn_shard_rows(al.ctx, al.K, lv, j0, j1, parts)
            L.fa_sinkhorn_shard_combine(al.ctx, parts, al.log_u)
            for j0, j1 in zip(bounds[:-1], bounds[1:]):
                L.fa_sinkhorn_shard_cols(al.ctx, al.K, al.log_u, lv, j0, j1, lv_next)
            lv, lv_next = lv_next, lv
        torch.cuda.synchronize()
        # (log_u, the v that produced it): the state fa_sinkhorn returns
        return al.log_u.cpu().numpy(), lv_next.cpu().numpy()
    finally:
        al.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_sharded_iteration_is_split_invariant_and_matches_oracle(case, dtype):
    K, lv0, u, v = case
    one = _sharded(dtype, K, lv0, [])
    two = _sharded(dtype, K, lv0, [4096])
    three = _sharded(dtype, K, lv0, [2048, 6144])
    for other in (two, three):
        np.testing.assert_array_equal(one[0], other[0])
        np.testing.assert_array_equal(one[1], other[1])
    du = np.abs(one[0] - np.log(u)).max()
    dv = np.abs(one[1] - np.log(v)).max()
    print(f"{dtype}: max |d log u| {du:.2e}, |d log v| {dv:.2e} against the oracle")
    assert du <= 1e-4 and dv <= 1e-4
    # the fused sweep computes the same iteration in another summation order
    al = _aligner(dtype, K, lv0)
    try:
        al.sinkhorn(ITERS)
        torch.cuda.synchronize()
        fu, fv = al.log_u.cpu().numpy(), al.log_v.cpu().numpy()
    finally:
        al.close()
    assert np.abs(fu - one[0]).max() <= 2e-5 and np.abs(fv - one[1]).max() <= 2e-5


def test_range_arguments_are_checked(case):
    from paper_2607_11952_gb300 import _lib as L
    K, lv0, u, v = case
    al = _aligner("f32", K, lv0)
    try:
        parts = torch.zeros((L.fa_shard_blocks(al.ld), N1), device=al.device)
        for j0, j1 in [(100, 2048), (0, 3000), (2048, 2048), (0, al.ld + 128), (-2048, 2048)]:
            with pytest.raises(L.FastAlignError) as ei:
                L.fa_sinkhorn_shard_rows(al.ctx, al.K, al.log_v, j0, j1, parts)
            assert ei.value.status == L.FA_ERR_ARG
        L.fa_sinkhorn_shard_rows(al.ctx, al.K, al.log_v, 8192, al.ld, parts)   # ld ends a range
    finally:
        al.close()
