"""The FP32 FMA-rate probe: the measured rate sits below the derived peak
(SMs x 128 lanes x 2 flops x clock at the maximum SM clock) and well above
half of it (the search kernels' roofline takes the derived peak)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_fma_rate_is_near_the_derived_peak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_11313_gb300 as px
    ctx = px.Context()
    tflops, ms = px.xcf_fp32_fma_rate(ctx)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived_at_2070 = sms * 128 * 2 * 2.070e9 / 1e12
    assert 0.5 * derived_at_2070 < tflops < 1.02 * derived_at_2070, (tflops, derived_at_2070)
    assert ms > 0.5
    ctx.close()
