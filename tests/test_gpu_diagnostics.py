"""Diagnostics of the library on the GPU: the measured FP32 FMA ceiling."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_fp32_fma_peak_is_plausible():
    import torch
    assert torch.cuda.is_available()
    import paper_2609_27342_gb300 as pkg
    from paper_2609_27342_gb300 import build
    build.build()
    L = pkg.load()
    out = ctypes.c_double(0.0)
    assert L.bm_fp32_fma_peak(None, ctypes.byref(out)) == 0
    # 152 SMs x 128 lanes x 2 flop x clock: about 80 TFLOP/s at 2.07 GHz
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceiling = sms * 128 * 2 * 2.2e9 / 1e12
    assert 0.3 * ceiling < out.value < 1.05 * ceiling
