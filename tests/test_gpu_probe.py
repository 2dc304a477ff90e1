"""The FP32 throughput probe used as context for the ALU-bound kernels' roofline: it reaches a
large part of the nominal FP32 rate (SMs x 128 lanes x 2 flop x the maximum SM clock) and not more."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_fp32_fma_probe_rate():
    import __graft_entry__ as ge
    ge.build_library()
    import paper_1906_02253_gb300 as kf
    props = torch.cuda.get_device_properties(0)
    max_mhz = getattr(props, "clock_rate", 0) / 1000.0 or 2070.0  # kHz in the properties when present
    nominal = props.multi_processor_count * 128 * 2 * max_mhz * 1e6 / 1e12
    rate = kf.fp32_fma_rate(iters=1024)
    assert 0.4 * nominal < rate < 1.05 * nominal, (rate, nominal)
    with pytest.raises(kf.KfError):
        kf.fp32_fma_rate(iters=0)
