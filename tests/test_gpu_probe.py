"""The measured FP32 FMA throughput (volks_measure_fp32_peak), the
denominator of the FP32 search kernel's roofline."""
import pytest

torch = pytest.importorskip("torch")

from paper_2108_05602_b300 import build
from paper_2108_05602_b300 import volks as V

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_plausible():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    props = torch.cuda.get_device_properties(0)
    t = [V.volks_measure_fp32_peak(torch.cuda.current_stream().cuda_stream) for _ in range(3)]
    # 128 FP32 lanes per SM, 2 flops per FMA, at 1-2.2 GHz
    lo, hi = props.multi_processor_count * 128 * 2 * 1.0e9 / 1e12, props.multi_processor_count * 256 * 2.2e9 / 1e12
    print(f"measured FP32 FMA peak: {max(t):.2f} TFLOP/s (runs {', '.join(f'{x:.2f}' for x in t)})")
    assert lo < max(t) < hi
