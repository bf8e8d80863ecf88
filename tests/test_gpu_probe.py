"""The tensor-pipe probe (fmm_tensor_peak) that gives the leaf kernels their
roofline: it runs, reports no device error, and its TF32 and BF16 rates are
physically plausible for this GPU (nominal dense rates 1.1 and 2.25 PFLOP/s)
and ordered as the instruction kinds are."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    from paper_1205_2927_gb300 import fmm as F
    tf32, ms = F.fmm_tensor_peak("tf32", batches=4000)
    bf16, _ = F.fmm_tensor_peak("bf16", batches=4000)
    assert ms > 0
    assert 300.0 < tf32 < 1400.0, tf32
    assert 600.0 < bf16 < 2800.0, bf16
    assert 1.3 < bf16 / tf32 < 2.6, (bf16, tf32)


def test_probe_rejects_bad_arguments():
    import torch
    from paper_1205_2927_gb300 import fmm as F
    x = torch.zeros(16384, device="cuda")
    lib = F.library()
    import ctypes as C
    out = C.c_double()
    assert lib.fmm_tensor_peak(2, 10, x.data_ptr(), C.byref(out), None, None) == 1
    assert lib.fmm_tensor_peak(0, 0, x.data_ptr(), C.byref(out), None, None) == 1
    assert lib.fmm_tensor_peak(0, 10, None, C.byref(out), None, None) == 1
    assert lib.fmm_tensor_peak(0, 10, x.data_ptr() + 4, C.byref(out), None, None) == 2
