"""Host logic of the library, checked on the CPU through its C ABI (no
device work is involved in either entry point).

* fa_graph_csr_host, the host half of fa_build_graph (Algorithm 1, row normalisation), against
  the oracle's row-normalised adjacency built by SciPy: identical row
  pointers and column indices, Abar values equal to float32(1/deg_i) and
  Abar^T values equal to float32(1/deg_k), on edge lists with duplicates,
  reversed pairs, self-loops and isolated nodes.
* fa_sweep_plan, the planner of the fused Sinkhorn sweep: the shapes the
  measured workloads run with, and at every row width a multiple of 128 up
  to the largest supported one, a shape that covers the row exactly, fits
  its threads' vectors, keeps at least two ring stages and fits the
  per-SM shared memory at the CTAs per SM its launch bounds promise.
"""
import numpy as np
import pytest

from oracle import fastalign_ref as R
from paper_2607_11952_gb300 import _lib as L
from paper_2607_11952_gb300 import synth

SMEM_PER_SM = 228 * 1024        # GB300 shared memory per SM
SMEM_RESERVED_PER_CTA = 1024    # reserved by the system for every resident CTA
MAX_ROW = 196_608               # widest row a sweep shape exists for


def _edge_soup(n, m, rng):
    src = rng.integers(0, n - 5, m)          # the last 5 nodes stay isolated
    dst = rng.integers(0, n - 5, m)
    dup = rng.integers(0, m, m // 5)
    src = np.concatenate([src, dst[dup], src[:7]])   # reversed duplicates
    dst = np.concatenate([dst, src[dup], src[:7]])   # ... and self-loops
    return src.astype(np.int32), dst.astype(np.int32)


@pytest.mark.parametrize("n,m,seed", [(1, 0, 0), (12, 30, 1), (500, 2500, 2), (3000, 40000, 3)])
def test_csr_matches_oracle_adjacency(n, m, seed):
    rng = np.random.default_rng(seed)
    if n > 5:
        src, dst = _edge_soup(n, m, rng)
    else:
        src = dst = np.zeros(0, np.int32)
    rp, col, vr, vc = L.fa_graph_csr_host(n, src, dst)
    A = R.row_normalized(n, np.stack([src, dst], axis=1).astype(np.int64))
    A.sort_indices()
    np.testing.assert_array_equal(rp, A.indptr)
    np.testing.assert_array_equal(col, A.indices)
    np.testing.assert_array_equal(vr, A.data.astype(np.float32))
    At = A.T.tocsr()
    At.sort_indices()
    np.testing.assert_array_equal(At.indptr, A.indptr)       # symmetric pattern
    np.testing.assert_array_equal(vc, At.data.astype(np.float32))
    deg = np.diff(rp)
    if n > 5:
        assert np.all(deg[-5:] == 0)


def test_csr_of_a_generated_graph():
    e = synth.chung_lu(2000, 2.3, 6.0, synth.rng_for(4))
    rp, col, vr, vc = L.fa_graph_csr_host(2000, e[:, 0], e[:, 1])
    assert rp[-1] == 2 * e.shape[0]
    A = R.row_normalized(2000, e)
    A.sort_indices()
    np.testing.assert_array_equal(rp, A.indptr)
    np.testing.assert_array_equal(col, A.indices)


def test_csr_argument_errors():
    with pytest.raises(L.FastAlignError) as ei:
        L.fa_graph_csr_host(4, np.array([0, 4]), np.array([1, 2]))
    assert ei.value.status == L.FA_ERR_ARG
    with pytest.raises(L.FastAlignError) as ei:
        L.fa_graph_csr_host(0, np.zeros(0), np.zeros(0))
    assert ei.value.status == L.FA_ERR_ARG
    with pytest.raises(L.FastAlignError) as ei:
        L.fa_graph_csr_host(3, np.array([0, -1]), np.array([1, 2]))
    assert ei.value.status == L.FA_ERR_ARG


def test_sweep_shapes_of_the_measured_workloads():
    # BF16 rule: the smallest power-of-two cluster (<= 8) whose slab takes at
    # most 5 vectors per thread with the last round >= 80% full; else the
    # smallest cluster (<= 10) with at most 5 vectors; else any that fits.
    # 50k: 4 CTAs need 7 vectors and 8 CTAs fill their 4th round to 76%, so
    # 5 CTAs (slabs of 1252 or 1251 vectors), one row per step
    got = L.fa_sweep_plan(50_000, 50_048, L.FA_BF16)
    assert (got["Q"], got["W"], got["S"], got["R"], got["NS"], got["NT"], got["kind"]) == \
        (5, 10016, 5, 1, 5, 256, 0)
    got = L.fa_sweep_plan(50_000, 50_048, L.FA_F32)
    assert (got["Q"], got["S"], got["R"], got["NS"], got["NT"], got["kind"]) == (8, 7, 1, 4, 256, 0)
    # 80k columns: 8 CTAs of 1250 vectors (98% of 5 rounds)
    got = L.fa_sweep_plan(100_000, 80_000, L.FA_BF16)
    assert (got["Q"], got["W"], got["S"], got["R"]) == (8, 10_000, 5, 1)
    # 30k and 70k columns: power-of-two clusters with two rows per step
    got = L.fa_sweep_plan(50_000, 30_080, L.FA_BF16)
    assert (got["Q"], got["W"], got["S"], got["R"], got["NS"]) == (4, 7520, 4, 2, 3)
    got = L.fa_sweep_plan(50_000, 70_016, L.FA_BF16)
    assert (got["Q"], got["W"], got["S"], got["R"], got["NS"]) == (8, 8752, 5, 2, 3)
    # 100k columns: rule 2 (10 CTAs); 110k: rule 3 (9 CTAs, 6 vectors)
    got = L.fa_sweep_plan(50_000, 100_096, L.FA_BF16)
    assert (got["Q"], got["S"]) == (10, 5)
    got = L.fa_sweep_plan(50_000, 110_080, L.FA_BF16)
    assert (got["Q"], got["S"]) == (9, 6)


def test_any_size_clusters_behind_their_switch(monkeypatch):
    monkeypatch.setenv("FA_SWEEP_ANYQ", "1")
    got = L.fa_sweep_plan(100_000, 80_000, L.FA_BF16)
    assert (got["Q"], got["W"], got["S"], got["R"]) == (7, 11_432, 6, 1)


def test_power_of_two_clusters_behind_their_switch(monkeypatch):
    monkeypatch.setenv("FA_SWEEP_ANYQ", "0")
    got = L.fa_sweep_plan(50_000, 50_048, L.FA_BF16)
    assert (got["Q"], got["W"], got["S"], got["R"], got["NS"], got["NT"], got["kind"]) == \
        (8, 6256, 4, 2, 4, 256, 0)


def test_tensor_core_sweep_shape_behind_its_switch(monkeypatch):
    # two 128-thread CTAs per SM, clusters of 16 and 7 rows per step at the
    # 50k workload's width
    monkeypatch.setenv("FA_SWEEP_KIND", "2")
    got = L.fa_sweep_plan(50_000, 50_048, L.FA_BF16)
    assert (got["Q"], got["W"], got["S"], got["R"], got["NS"], got["NT"], got["kind"]) == \
        (16, 3128, 4, 7, 2, 128, 2)
    got = L.fa_sweep_plan(100_000, 80_000, L.FA_BF16)
    assert (got["Q"], got["W"], got["S"], got["R"], got["NT"], got["kind"]) == \
        (16, 5000, 3, 8, 256, 2)


def _smem(p, b):
    """Dynamic shared memory of one CTA of the CUDA-core sweep: the ring of
    NS x R slab rows, the 8 ring and 4 exchange mbarriers, the row-partial
    reduction and the cluster exchange slots (4 x 16 clusters x R)."""
    return p["NS"] * p["R"] * p["W"] * b + 12 * 8 + (2 * p["R"] * (p["NT"] // 32) + 4 * 16 * p["R"]) * 4


def _smem_mma(p):
    """Dynamic shared memory of one CTA of the tensor-core sweep: NS x R ring
    rows and the three bfloat16 parts of v, each row of W columns padded to
    a multiple of 32 plus 16 bytes; a 16-byte zero chunk; 4 ring and 4
    exchange mbarriers; the row partials (8 per warp) and the exchange
    slots (4 x 16 clusters x 8)."""
    rs = (p["W"] + 31) // 32 * 32 * 2 + 16
    return (p["NS"] * p["R"] + 3) * rs + 16 + 8 * 8 + (p["NT"] // 32 * 8 + 4 * 16 * 8) * 4


@pytest.mark.parametrize("kind", [0, 2])
@pytest.mark.parametrize("dtype", [L.FA_BF16, L.FA_F32])
def test_sweep_plan_invariants_at_every_width(dtype, kind, monkeypatch):
    monkeypatch.setenv("FA_SWEEP_KIND", str(kind))
    V, b = (8, 2) if dtype == L.FA_BF16 else (4, 4)
    n_mma = 0
    for ld in range(128, MAX_ROW + 1, 128):
        p = L.fa_sweep_plan(4096, ld, dtype)
        assert p["kind"] in ((0, 2) if dtype == L.FA_BF16 else (0,))
        if p["kind"] == 0 and dtype == L.FA_BF16:
            # any cluster size; slabs of ceil or floor of ld / V / Q vectors
            assert 1 <= p["Q"] <= 16
            assert p["W"] == V * -(-(ld // V) // p["Q"]) and (p["W"] * b) % 16 == 0
        else:
            assert p["Q"] in (1, 2, 4, 8, 16)
            assert p["Q"] * p["W"] == ld and (p["W"] * b) % 16 == 0
        assert (p["S"] - 1) * p["NT"] * V < p["W"] <= p["S"] * p["NT"] * V
        assert 1 <= p["G"] <= (4096 + p["R"] - 1) // p["R"]
        if p["kind"] == 2:
            n_mma += 1
            per_sm = 2 if p["NT"] == 128 else 1
            assert p["NT"] in (128, 256) and p["NS"] == 2 and 4 <= p["R"] <= 8
            assert per_sm * (_smem_mma(p) + SMEM_RESERVED_PER_CTA) <= SMEM_PER_SM, (ld, p)
            assert _smem_mma(p) <= 227 * 1024
            continue
        assert p["R"] in (1, 2, 4) and 2 <= p["NS"] <= 8
        per_sm = (4 if p["S"] * V <= 16 else 2) if p["NT"] == 256 else 1
        assert per_sm * (_smem(p, b) + SMEM_RESERVED_PER_CTA) <= SMEM_PER_SM, (ld, p)
    if dtype == L.FA_BF16 and kind == 2:
        assert n_mma > 0.8 * (MAX_ROW // 128)     # every width up to ~167k
    else:
        assert n_mma == 0
    with pytest.raises(L.FastAlignError) as ei:
        L.fa_sweep_plan(4096, MAX_ROW + 128, dtype)
    assert ei.value.status == L.FA_ERR_UNSUPPORTED


def test_sweep_plan_switches_and_errors(monkeypatch):
    monkeypatch.setenv("FA_SWEEP_Q", "2")
    assert L.fa_sweep_plan(10_000, 10_112, L.FA_BF16)["Q"] == 2
    monkeypatch.setenv("FA_SWEEP_Q", "")
    monkeypatch.setenv("FA_SWEEP_KIND", "2")
    monkeypatch.setenv("FA_SWEEP_MB", "1")
    assert L.fa_sweep_plan(10_000, 10_112, L.FA_BF16)["NT"] == 256
    monkeypatch.delenv("FA_SWEEP_MB")
    monkeypatch.delenv("FA_SWEEP_KIND")
    monkeypatch.setenv("FA_SWEEP_NT", "512")
    assert L.fa_sweep_plan(10_000, 10_112, L.FA_BF16)["NT"] == 512
    monkeypatch.delenv("FA_SWEEP_NT")
    for args in [(0, 128, L.FA_BF16), (10, 100, L.FA_BF16), (10, 128, 7)]:
        with pytest.raises(L.FastAlignError) as ei:
            L.fa_sweep_plan(*args)
        assert ei.value.status == L.FA_ERR_ARG
