"""The peak microbenchmarks behind the benchmark's roofline fractions.

Each kernel keeps one arithmetic pipe busy; its rate per SM clock must lie
below the unit counts of the part (128 FP32 lanes x 2 flops per SM and clock)
and the pipes must order as the hardware does (tensor cores above FP32 above
FP64).  The values themselves are measurements, not asserted.
"""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_09900_gb300 import build
    build.build()
    import paper_2205_09900_gb300 as fpm
    fpm.load()
    return fpm


def test_peak_rates_are_physical(fp):
    r = {w: fp.measure_peak(w) for w in (fp.PEAK_FFMA, fp.PEAK_FFMA2, fp.PEAK_DFMA, fp.PEAK_TC_TF32,
                                         fp.PEAK_TC_BF16)}
    for w, v in r.items():
        assert v["tflops"] > 0 and v["sm_mhz"] > 100 and v["sms"] > 0, (w, v)
    # 128 FP32 lanes per SM: at most 256 flops per clock (a few % of clock skew allowed)
    assert r[fp.PEAK_FFMA]["flops_per_clk_sm"] < 256 * 1.05
    assert r[fp.PEAK_FFMA2]["flops_per_clk_sm"] < 256 * 1.05
    assert r[fp.PEAK_DFMA]["tflops"] < r[fp.PEAK_FFMA]["tflops"]
    assert r[fp.PEAK_TC_TF32]["tflops"] > r[fp.PEAK_FFMA2]["tflops"]
    assert r[fp.PEAK_TC_BF16]["tflops"] > r[fp.PEAK_TC_TF32]["tflops"]
