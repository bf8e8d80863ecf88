"""GPU parity of the host-resident path: operands in pinned host memory,
quadrants streamed in order of first use, the root level depth-first."""
import numpy as np
import pytest

import oracle.fmm_oracle as O
from paper_1205_2927_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1205_2927_gb300 import fmm
    return fmm


def run_host(F, A, B, C0=None, alpha=1.0, beta=0.0, **kw):
    import torch
    m, k = A.shape
    n = B.shape[1]
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = (torch.from_numpy(C0) if C0 is not None else torch.full((m, n), float("nan"))).pin_memory()
    p = F.Plan(m, n, k, host_operands=1, **kw)
    p(hA, hB, hC, alpha=alpha, beta=beta)
    torch.cuda.current_stream().synchronize()
    assert p.device_status() == 0
    p.close()
    return hC.numpy().copy()


@pytest.mark.parametrize("m,k,n,d", [(300, 200, 260, 2), (512, 512, 512, 1), (777, 333, 515, 0),
                                     (1024, 640, 768, 3), (130, 70, 90, 1)])
def test_host_resident_bit_exact(F, m, k, n, d):
    A = I.small_int((m, k), 11000 + m, r=2)
    B = I.small_int((k, n), 11100 + n, r=2)
    C = run_host(F, A, B, depth=d)
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
    assert np.array_equal(C, ref)


def test_host_resident_alpha_beta(F):
    m, k, n = 290, 150, 330
    A = I.small_int((m, k), 15, r=3)
    B = I.small_int((k, n), 16, r=3)
    C0 = I.small_int((m, n), 17, r=5)
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float64)
    for d in (0, 2):
        C = run_host(F, A, B, C0, alpha=2.0, beta=-1.0, depth=d)
        assert np.array_equal(C, (2.0 * ref - C0).astype(np.float32))


def test_host_resident_float_bound(F):
    n = 1024
    A, B = I.operands(n, n, n, I.seed_for(2, 9), "normal")
    C = run_host(F, A, B, depth=2)
    assert O.error_metric(C, O.classical(A, B), A, B) <= 2e-6


def test_pageable_host_memory_rejected(F):
    import torch
    A = torch.ones(64, 64)
    B = torch.ones(64, 64)
    C = torch.zeros(64, 64)
    p = F.Plan(64, 64, 64, host_operands=1, depth=1)
    with pytest.raises(F.FmmError) as ei:
        F.fmm_gemm(p.handle, 1.0, A.data_ptr(), B.data_ptr(), 0.0, C.data_ptr())
    assert ei.value.status == 1
    p.close()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3", "tf32"])
def test_host_resident_split_precision(F, prec):
    m, k, n = 640, 512, 768
    A = I.small_int((m, k), 14000, r=2)
    B = I.small_int((k, n), 14100, r=2)
    C = run_host(F, A, B, depth=2, precision=prec)
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
    assert np.array_equal(C, ref)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_host_resident_equals_device_resident(F, d):
    # the streamed root forms each C quadrant with the same U-chain operations as
    # the device-resident plan, and its child plan uses the same leaf tiles, so
    # the two results agree bit for bit on float data (alpha, beta included)
    import torch
    n = 1024
    A, B = I.operands(n, n, n, I.seed_for(2, 40 + d), "normal")
    C0 = I.uniform((n, n), 41 + d)
    host = run_host(F, A, B, C0, alpha=0.5, beta=-2.0, depth=d)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.from_numpy(C0).cuda()
    p = F.Plan(n, n, n, depth=d)
    p(dA, dB, dC, alpha=0.5, beta=-2.0)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    p.close()
    assert np.array_equal(host, dC.cpu().numpy())


@pytest.mark.parametrize("m,k,n,d", [(1000, 700, 900, 3), (700, 1030, 610, 2), (1100, 900, 1300, 4)])
def test_host_resident_ragged_sub_level_alpha_beta(F, m, k, n, d):
    # depth >= 2: the first and last root products stream sub-quadrants (A11 and
    # B11 in, C12 out); ragged sizes clip those sub-quadrant copies
    r = 1 if d == 4 else 2   # every partial sum stays an integer below 2^24
    A = I.small_int((m, k), 16000 + m, r=r)
    B = I.small_int((k, n), 16100 + n, r=r)
    C0 = I.small_int((m, n), 16200 + d, r=4)
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float64)
    C = run_host(F, A, B, C0, alpha=-1.0, beta=3.0, depth=d)
    assert np.array_equal(C, (-ref + 3.0 * C0).astype(np.float32))


@pytest.mark.parametrize("d", [2, 3])
def test_host_resident_ragged_equals_device_resident(F, d):
    # float data on ragged rectangular sizes: the padded device plan and the
    # streamed plan (sub-level first and last products) agree bit for bit
    import torch
    m, k, n = 1000, 1100, 900
    A, B = I.operands(m, k, n, I.seed_for(2, 60 + d), "normal")
    C0 = I.uniform((m, n), 61 + d)
    host = run_host(F, A, B, C0, alpha=1.5, beta=0.25, depth=d)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.from_numpy(C0).cuda()
    p = F.Plan(m, n, k, depth=d)
    p(dA, dB, dC, alpha=1.5, beta=0.25)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    p.close()
    assert np.array_equal(host, dC.cpu().numpy())


@pytest.mark.parametrize("m,k,n,d", [(300, 200, 260, 2), (512, 512, 512, 1), (777, 333, 515, 0),
                                     (1000, 700, 900, 3), (130, 70, 90, 1)])
def test_host_copy_by_sm_equals_copy_engines(F, m, k, n, d):
    # the same plan with its host traffic moved by SM loads/stores on the
    # device mapping of the pinned memory instead of the copy engines: the
    # device computes the same, so the results agree bit for bit (ragged
    # quadrants, beta != 0 reads C in)
    A, B = I.operands(m, k, n, I.seed_for(2, 70 + d), "normal")
    C0 = I.uniform((m, n), 71 + d)
    eng = run_host(F, A, B, C0, alpha=0.5, beta=-2.0, depth=d, host_copy="engine")
    sm = run_host(F, A, B, C0, alpha=0.5, beta=-2.0, depth=d, host_copy="sm")
    assert np.array_equal(eng, sm)
    ref = 0.5 * O.classical(A, B) - 2.0 * C0
    den = float(np.abs(A).max()) * float(np.abs(B).max()) * k
    assert float(np.max(np.abs(sm - ref))) <= 2e-6 * den + 4.0 * float(np.abs(C0).max()) * 2.0 ** -23


def test_host_copy_by_sm_strided_views(F):
    # pinned views with row strides that are not multiples of 4 (the copy
    # kernel's element-wise form) and an offset start, exact on integers
    import torch
    m, k, n = 301, 203, 257
    A = I.small_int((m, k), 17001, r=2)
    B = I.small_int((k, n), 17002, r=2)
    hA_full = torch.zeros((m, k + 3)).pin_memory()
    hB_full = torch.zeros((k, n + 5)).pin_memory()
    hC_full = torch.full((m, n + 1), float("nan")).pin_memory()
    hA, hB, hC = hA_full[:, 1:k + 1], hB_full[:, 2:n + 2], hC_full[:, :n]
    hA.copy_(torch.from_numpy(A))
    hB.copy_(torch.from_numpy(B))
    for d in (0, 2):
        launches = {}
        for how in ("engine", "sm"):
            hC.fill_(float("nan"))
            p = F.Plan(m, n, k, lda=k + 3, ldb=n + 5, ldc=n + 1, depth=d, host_operands=1, host_copy=how)
            p(hA, hB, hC)
            torch.cuda.current_stream().synchronize()
            assert p.device_status() == 0
            launches[how] = p.profile_read()["launches"]
            p.close()
            ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
            assert np.array_equal(hC.numpy(), ref)
            assert np.all(np.isnan(hC_full[:, n:].numpy()))
        # the SM form runs one copy kernel per block moved (pinned memory has a
        # device mapping here), the engine form none
        assert launches["sm"] > launches["engine"], launches


def test_host_copy_mode_query(F):
    # device plans report none; forced modes report themselves; the library
    # default starts on the copy engines and may move to SM copies (only if a
    # call's transfers stalled), with the same results either way
    import torch
    n = 4096
    A, B = I.operands(n, n, n, I.seed_for(2, 80))
    hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
    outs = {}
    for how in ("default", "engine", "sm"):
        p = F.Plan(n, n, n, depth=1, host_operands=1, host_copy=how)
        first = p.host_copy()
        hC = torch.empty((n, n)).pin_memory()
        for _ in range(3):
            p(hA, hB, hC)
        torch.cuda.current_stream().synchronize()
        assert p.device_status() == 0
        if how == "default":
            assert first == "engine" and p.host_copy() in ("engine", "sm")
        else:
            assert first == how and p.host_copy() == how
        outs[how] = hC.numpy().copy()
        p.close()
    assert np.array_equal(outs["default"], outs["engine"]) and np.array_equal(outs["sm"], outs["engine"])
    d = F.Plan(256, 256, 256)
    assert d.host_copy() is None
    d.close()
