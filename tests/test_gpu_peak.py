"""The FP64 throughput probe that states the FP64 kernels' roofline."""
import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_fp64_peak_is_measured_and_stable():
    sv = need_gpu()
    a = sv.measure_fp64_peak()
    b = sv.measure_fp64_peak()
    # a double-precision FMA rate: well above zero, well below the float rate
    assert 0.1 < a < 20.0
    assert abs(a - b) <= 0.05 * max(a, b)
