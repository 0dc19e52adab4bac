"""The FP32 fma probe that gives the blend's roofline denominator (fdgs_measure_fp32_peak):
its figures must be positive and physically possible, i.e. at most what 128 FP32 lanes per SM
at the maximum SM clock can do (twice that for the paired form, which issues two fmas per
lane), and the call rejects bad arguments."""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu

SM_MAX_MHZ = 2070.0


@pytest.fixture(scope="module")
def fd():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_16422_gb300 import build, fdgs
    build.build()
    fdgs.lib()
    return fdgs


def test_fp32_probe_is_within_the_unit_count_bound(fd):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound = sms * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    scalar = fd.measure_fp32_peak(False)
    paired = fd.measure_fp32_peak(True)
    print(f"PROBE scalar {scalar:.1f} paired {paired:.1f} unit-count bound {bound:.1f} TFLOP/s")
    assert 0.3 * bound < scalar <= 1.02 * bound
    assert 0.3 * bound < paired <= 2.04 * bound


def test_fp32_probe_rejects_bad_arguments(fd):
    v = ctypes.c_double()
    assert fd.lib().fdgs_measure_fp32_peak(2, ctypes.byref(v), None) == -1
    assert fd.lib().fdgs_measure_fp32_peak(0, None, None) == -1
