"""The FMA-throughput probe (blcoc_probe_peak) that gives the ALU roofline its peak."""
import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def test_probe_peak_is_plausible():
    need_gpu()
    from paper_1601_05362_gb300 import blcoc
    fp64 = blcoc.probe_peak("fp64")
    fp32 = blcoc.probe_peak("fp32")
    # a GB300 issues 2 DFMA and 128 FFMA per clock per SM (152 SMs, <= 2.07 GHz): at most
    # 1.26 and 80.6 TFLOP/s; the probe must land below those and not far below
    assert 0.5e12 < fp64 < 1.3e12, fp64
    assert 30e12 < fp32 < 81e12, fp32
    assert blcoc.load_library().blcoc_probe_peak(2, None) == blcoc.BLCOC_ERR_INVALID_ARG
