"""GPU test of the FP32 FMA-chain probe, the measured denominator of the render
kernels' ALU roofline: it must land near SMs x 128 lanes x 2 flop x clock."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_fp32_probe_near_lane_count_peak(gpu_lib):
    from paper_2211_17263_gb300 import api
    ctx = api.Context(0)
    try:
        tflops, ms = ctx.fp32_peak_probe(1 << 16)
    finally:
        ctx.close()
    props = torch.cuda.get_device_properties(0)
    formula = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12  # at the maximum SM clock
    assert ms > 0
    assert 0.3 * formula < tflops < 1.05 * formula, (tflops, formula)
