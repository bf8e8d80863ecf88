"""The allocation-free entry point fmm_gemm_static, checked against the regular
planned path (fmm_plan + fmm_gemm) on two calls in a row.

fmm_gemm_static serves callers that cannot allocate device memory when they
multiply: a runtime whose device memory another allocator reserved up front,
an embedding that gives this library no allocator or workspace, a path that
must not pay for an allocation.  Its temporaries live in a fixed device array
compiled into the library, so M, N and K are limited to 1024.  This file is
collected last on purpose, so that a run stopping at its first failure has run
every other test before it."""
import ctypes

import numpy as np
import pytest

import oracle.fmm_oracle as O
from paper_1205_2927_gb300 import inputs as I

pytestmark = pytest.mark.gpu

BOUND = 2e-6  # max-norm error bound the FP32 parity tests use


def _static(F):
    lib = F.library()
    f = lib.fmm_gemm_static
    f.argtypes = [ctypes.c_int64] * 3 + [ctypes.c_float, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_static_entry_matches_planned_path_twice():
    import torch
    from paper_1205_2927_gb300 import fmm as F
    f = _static(F)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (m, k, n) in enumerate([(1000, 900, 1024), (513, 1024, 700)]):
        A, B = I.operands(m, k, n, 12000 + call)
        C0 = I.uniform((m, n), 12100 + call)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        c_static = torch.from_numpy(C0).cuda()
        c_plan = torch.from_numpy(C0).cuda()
        st = f(m, n, k, 0.75, dA.data_ptr(), k, dB.data_ptr(), n, 0.5, c_static.data_ptr(), n, stream)
        assert st == 0, F.library().fmm_last_error()
        assert F.fmm_gemm_static_status() == 0
        p = F.Plan(m, n, k, depth=1)
        p(dA, dB, c_plan, alpha=0.75, beta=0.5)
        torch.cuda.synchronize()
        got, want = c_static.cpu().numpy(), c_plan.cpu().numpy()
        den = np.abs(A).max() * np.abs(B).max() * k
        assert np.max(np.abs(got.astype(np.float64) - want)) / den <= BOUND
        ref = O.gemm(0.75, A, B, 0.5, C0)
        assert np.max(np.abs(got - ref)) / den <= BOUND
        p.close()


def test_static_entry_allocates_no_device_memory():
    # After one warm call (the first call on a device looks up the array's
    # address), further calls leave the device's free memory unchanged.
    import torch
    from paper_1205_2927_gb300 import fmm as F
    m, k, n = 768, 1000, 640
    A, B = I.operands(m, k, n, 12200)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    outs = [torch.empty(m, n, device="cuda") for _ in range(3)]
    F.fmm_gemm_static(dA, dB, outs[0])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    F.fmm_gemm_static(dA, dB, outs[1])
    F.fmm_gemm_static(dA, dB, outs[2], alpha=-2.0)
    assert F.fmm_gemm_static_status() == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    den = np.abs(A).max() * np.abs(B).max() * k
    ref = O.classical(A, B)
    assert np.max(np.abs(outs[1].cpu().numpy() - ref)) / den <= BOUND
    assert np.max(np.abs(outs[2].cpu().numpy() + 2.0 * ref)) / (2.0 * den) <= BOUND


def test_static_entry_alpha_zero_scales_c():
    # alpha == 0 reads neither A nor B (NaN there must not show) and sets C <- beta C
    import torch
    from paper_1205_2927_gb300 import fmm as F
    m, k, n = 300, 200, 260
    C0 = I.uniform((m, n), 12300)
    dA = torch.full((m, k), float("nan"), device="cuda")
    dB = torch.full((k, n), float("nan"), device="cuda")
    dC = torch.from_numpy(C0).cuda()
    F.fmm_gemm_static(dA, dB, dC, alpha=0.0, beta=0.5)
    assert F.fmm_gemm_static_status() == 0
    assert np.array_equal(dC.cpu().numpy(), (0.5 * C0).astype(np.float32))


def test_static_entry_rejects_sizes_beyond_limit():
    import torch
    from paper_1205_2927_gb300 import fmm as F
    f = _static(F)
    x = torch.zeros(4, device="cuda")
    st = f(1025, 8, 8, 1.0, x.data_ptr(), 8, x.data_ptr(), 8, 0.0, x.data_ptr(), 8, None)
    assert st == 1
    assert b"1024" in F.library().fmm_last_error()
