"""The benchmark's measured FP32 FMA throughput (bench_fp32_fma_tflops in
the benchmark-only helper library), the denominator of the FP32 search
kernel's roofline."""
import pytest

torch = pytest.importorskip("torch")

import bench
from paper_2108_05602_b300 import build

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_plausible():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    props = torch.cuda.get_device_properties(0)
    t = [bench.measured_fp32_tflops(torch.cuda.current_stream().cuda_stream) for _ in range(3)]
    # 128 FP32 lanes per SM, 2 flops per FMA, at 1-2.2 GHz
    lo, hi = props.multi_processor_count * 128 * 2 * 1.0e9 / 1e12, props.multi_processor_count * 256 * 2.2e9 / 1e12
    print(f"measured FP32 FMA peak: {max(t):.2f} TFLOP/s (runs {', '.join(f'{x:.2f}' for x in t)})")
    assert lo < max(t) < hi
