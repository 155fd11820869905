"""Failure detection without a GPU fault.

fa_ctx_selftest_wait runs one kernel whose bounded mbarrier wait (the one
every wait of the fused sweep uses) waits on a phase that nothing
completes.  It must give up after its time limit (about 2 s), return
normally and leave the timeout bit in the context's status.  The next
fa_sinkhorn reports FA_ERR_TIMEOUT, clears the bit, and the context stays
usable: a following solve on it converges as usual.
"""
import time

import pytest

torch = pytest.importorskip("torch")

from paper_2607_11952_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_context_recovers():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_11952_gb300 import api, _lib as L
    g = synth.config_pair("ba1k", n=300)
    al = api.Aligner(api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2),
                     api.Params(dtype="f32"))
    try:
        al.node_cost(g.X1, g.X2, g.anchors)
        al.plan_init()
        al.align_iter()
        v1 = al.log_v.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.fa_ctx_selftest_wait(al.ctx)
        with pytest.raises(L.FastAlignError) as ei:
            al.sinkhorn(50, 1e-4, 5)
        waited = time.perf_counter() - t0
        print(f"status {ei.value.status}, waited {waited:.2f} s")
        assert ei.value.status == L.FA_ERR_TIMEOUT
        assert 1.5 <= waited <= 60.0           # the wait ran to its limit and no further
        # the bit was cleared once reported: the same context solves normally
        L.fa_vec_axpby(al.n2, 1.0, v1, 0.0, None, al.log_v)
        it, err, st = al.sinkhorn(2000, 1e-4, 5)
        assert st == L.FA_OK and err <= 1e-4
        assert bool(torch.isfinite(al.log_u).all()) and bool(torch.isfinite(al.log_v).all())
    finally:
        al.close()
