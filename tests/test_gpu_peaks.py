"""The peak measurement used as the ALU roofline denominators (GPU)."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_02888_gb300 import ewald
    p = ewald.measure_peaks()
    # a GB300 has 152 SMs x 128 FP32 lanes at up to ~2 GHz (~80 TFLOP/s FMA)
    # and a far narrower FP64 pipe; the measurement must land in that range
    assert 10 < p["fp32_tflops"] < 120
    assert 0.05 < p["fp64_tflops"] < p["fp32_tflops"] / 4
    assert p["rsqrt_tops"] > 0.5
