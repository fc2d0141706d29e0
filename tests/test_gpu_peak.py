"""The in-process FP64 rate measurement (the denominator of the FP64 step's
arithmetic roofline) returns a plausible figure: GB300's FP64 rate is
nominally 1.25 TFLOP/s (152 SMs x 2 FMA per clock x 2.07 GHz)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2208_01339_gb300.polyprec")


def test_fp64_fma_rate_is_plausible():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tf = P.fp64_fma_rate(reps=3)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # between a quarter of and twice 2 FMA/clock/SM at 2.1 GHz
    nominal = sms * 4 * 2.1e9 / 1e12
    assert 0.25 * nominal < tf < 2.0 * nominal, tf
