"""The bounded wait of the tensor-core kernels: a wait on an mbarrier that receives no arrival gives
up after its limit and returns, leaving the context usable; a wait after the arrival completes."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kf():
    import __graft_entry__ as ge
    ge.build_library()
    import paper_1906_02253_gb300 as k
    k.load_library()
    return k


@pytest.mark.parametrize("limit_us", [2000, 20000])
def test_bounded_wait_gives_up_and_the_context_stays_usable(kf, limit_us):
    out = kf.wait_probe(limit_us).cpu().numpy()
    assert out[0] == 0, "a wait with no arrival must give up"
    assert out[1] == 1, "a wait after the arrival must complete"
    assert limit_us * 1000 <= out[2] < limit_us * 1000 + 5_000_000, out[2]
    # the context still runs the tensor-core kernels
    import synth
    w = synth.mlp_init(3)
    buf = kf.mlp_buffer(w, np.zeros(14, np.float32), np.ones(14, np.float32))
    got = kf.mlp_forward(buf, torch.ones((300, 14), device="cuda"))
    assert torch.isfinite(got).all()

