"""__graft_entry__.smoke() runs on the GPU: the FP32 path against the
oracle and the BF16 form with the learned warm start."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_smoke():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.smoke()
