"""fa_sinkhorn_step_static, the Sinkhorn iteration that allocates no device
memory, against fa_sinkhorn (the context-based entry) on the same Gibbs
kernel: two calls in a row, each compared with the context path's result
after as many iterations.  Collected last so that it runs both after the
other GPU tests and, on its own, in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2607_11952_gb300 import synth  # noqa: E402

ERR_FLOOR = 1e-6          # FP32 floor of the reported marginal error
LOG_TOL = 1e-5            # log scalings: FP32 rounding of the same sums
MAX_LD = 65536            # static scratch limit stated in include/fastalign.h


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_11952_gb300 import _lib
    return _lib


def test_rejects_columns_beyond_the_static_limit(L):
    # host-side check: answers before any CUDA call
    fake = 256
    with pytest.raises(L.FastAlignError) as ei:
        st = L.lib().fa_sinkhorn_step_static(fake, L.FA_F32, 10, MAX_LD + 1, MAX_LD + 128,
                                             fake, fake, fake, fake, None, None)
        L._check(st, "fa_sinkhorn_step_static")
    assert ei.value.status == L.FA_ERR_UNSUPPORTED
    assert "static scratch maximum" in str(ei.value)
    st = L.lib().fa_sinkhorn_step_static(None, L.FA_F32, 10, 10, 128, fake, fake, fake, fake,
                                         None, None)
    assert st == L.FA_ERR_ARG


CASES = [("f32", 700, 530), ("bf16", 700, 530), ("f32", 2000, 60000),
         ("bf16", 1500, 65500)]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,n1,n2", CASES)
def test_static_step_matches_context_sinkhorn(L, dtype, n1, n2):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_11952_gb300 import api
    rng = synth.rng_for(31 + n1)
    g1 = api.Graph(n1, synth.erdos_renyi(n1, 3.0, rng))
    g2 = api.Graph(n2, synth.erdos_renyi(n2, 3.0, rng))
    al = api.Aligner(g1, g2, api.Params(dtype=dtype))
    ld = al.ld
    assert ld <= MAX_LD
    gen = torch.Generator(device="cuda").manual_seed(7 + n2)
    K = 0.05 + 0.95 * torch.rand((n1, ld), generator=gen, device="cuda")
    K[:, n2:] = 0.0
    al.K.copy_(K.to(al.K.dtype))
    v0 = 0.5 * torch.randn(n2, generator=gen, device="cuda")

    # context path: one and two iterations from v0
    _, err_ref1, st = al.sinkhorn(1, tol=-1.0, warm_log_v=v0)
    assert st == L.FA_OK
    u_ref1 = al.log_u.clone()
    _, err_ref2, st = al.sinkhorn(2, tol=-1.0, warm_log_v=v0)
    assert st == L.FA_OK
    v_ref1, u_ref2 = al.log_v.clone(), al.log_u.clone()

    # allocation-free path: two calls in a row, the second consuming the first
    code = L.FA_BF16 if dtype == "bf16" else L.FA_F32
    u = torch.empty(n1, device="cuda")
    v1 = torch.empty(n2, device="cuda")
    v2 = torch.empty(n2, device="cuda")
    err = torch.empty(2, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    L.fa_sinkhorn_step_static(al.K, code, n1, n2, ld, v0, u, v1, err[0:1], status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    torch.testing.assert_close(u, u_ref1, rtol=LOG_TOL, atol=LOG_TOL)
    L.fa_sinkhorn_step_static(al.K, code, n1, n2, ld, v1, u, v2, err[1:2], None)
    torch.cuda.synchronize()
    torch.testing.assert_close(v1, v_ref1, rtol=LOG_TOL, atol=LOG_TOL)
    torch.testing.assert_close(u, u_ref2, rtol=LOG_TOL, atol=LOG_TOL)
    e = err.cpu().numpy()
    for got, ref in ((e[0], err_ref1), (e[1], err_ref2)):
        assert np.isfinite(got)
        assert abs(got - ref) <= 1e-3 * ref + ERR_FLOOR, (got, ref)
