"""GPU parity of the C-ABI path against the CPU oracle.

Bit-exact where every partial sum is an exact integer below 2^24 (small-integer
operands); otherwise within the max-norm bound
||C - C64||_max / (||A||_max ||B||_max K) <= 2e-6 for the FP32 (3xTF32) path at
depth <= 3.  All calls go through fmm_plan / fmm_gemm.
"""
import numpy as np
import pytest

import oracle.fmm_oracle as O
from paper_1205_2927_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP32_BOUND = 2e-6
# split-precision bounds: the FP32 bound scaled by each split's per-term error
# bound against 3xTF32's 2^-19 (BF16x3 3 * 2^-16 -> 4.8e-5; TF32 2^-10 ->
# 1.0e-3; FP16x3's 3 * 2^-22 is below 3xTF32's: held to the FP32 bound)
SPLIT_BOUND = {"fp32": FP32_BOUND, "fp16x3": FP32_BOUND, "bf16x3": 4.8e-5, "tf32": 1.0e-3}


@pytest.fixture(scope="module")
def fmm():
    import torch  # noqa: F401
    from paper_1205_2927_gb300 import fmm as F
    return F


def run(fmm, A, B, C0=None, alpha=1.0, beta=0.0, **kw):
    import torch
    M, K = A.shape
    N = B.shape[1]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.from_numpy(np.ascontiguousarray(C0)).cuda() if C0 is not None else torch.empty((M, N), device="cuda")
    plan = fmm.Plan(M, N, K, **kw)
    plan(dA, dB, dC, alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    info = plan.info
    plan.close()
    return dC.cpu().numpy(), info


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
@pytest.mark.parametrize("m,k,n", [(128, 32, 256), (256, 256, 256), (200, 100, 300), (777, 333, 515), (1, 1, 1)])
@pytest.mark.parametrize("bn", [128, 256])
def test_classical_bit_exact_small_int(fmm, prec, m, k, n, bn):
    A = I.small_int((m, k), 1000 + m, r=3)
    B = I.small_int((k, n), 2000 + n, r=3)
    C, info = run(fmm, A, B, depth=0, precision=prec, leaf_tile=bn)
    assert info["depth"] == 0
    ref = O.classical(A.astype(np.int64), B.astype(np.int64))
    assert np.array_equal(C, ref.astype(np.float32))


@pytest.mark.parametrize("m,k,n", [(512, 512, 512), (300, 200, 260), (1024, 640, 768)])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_winograd_bit_exact_small_int(fmm, m, k, n, d):
    A = I.small_int((m, k), 3000 + m + d, r=2)
    B = I.small_int((k, n), 4000 + n + d, r=2)
    C, info = run(fmm, A, B, depth=d, precision="fp32")
    assert info["depth"] == d
    ref = O.classical(A.astype(np.int64), B.astype(np.int64))
    # the fp32 oracle recursion is exact here too: both equal the integer product
    assert np.array_equal(O.winograd(A, B, d, "pad"), ref.astype(np.float32))
    assert np.array_equal(C, ref.astype(np.float32))


@pytest.mark.parametrize("dist", ["uniform", "normal"])
@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_fp32_error_bound(fmm, dist, d):
    n = 1024
    A, B = I.operands(n, n, n, I.seed_for(1, d), dist)
    C, _ = run(fmm, A, B, depth=d, precision="fp32")
    err = O.error_metric(C, O.classical(A, B), A, B)
    assert err <= FP32_BOUND, err


def test_tf32_is_coarser_than_fp32(fmm):
    n = 1024
    A, B = I.operands(n, n, n, I.seed_for(1, 7))
    ref = O.classical(A, B)
    e32 = O.error_metric(run(fmm, A, B, depth=0, precision="fp32")[0], ref, A, B)
    etf = O.error_metric(run(fmm, A, B, depth=0, precision="tf32")[0], ref, A, B)
    assert e32 < etf / 20, (e32, etf)


def test_fp32_matches_three_product_split_model(fmm):
    # the 3xTF32 leaf equals hi*hi + hi*lo + lo*hi with hi = trunc_tf32(x) (what the
    # tensor core reads from the raw operand) and lo = rn_tf32(x - hi), up to fp32
    # accumulation error -- far tighter than the error bound; a dropped or
    # mis-split term is off by ~2^-11 relative
    m, k, n = 256, 512, 256
    A, B = I.operands(m, k, n, 77)
    C, _ = run(fmm, A, B, depth=0, precision="fp32")
    Ah, Al = O.split_tf32(A, "trunc", "rne")
    Bh, Bl = O.split_tf32(B, "trunc", "rne")
    model = O.split_product(Ah, Al, Bh, Bl)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    assert np.max(np.abs(C - model) / scale) <= 4 * k * 2.0 ** -24


def test_tf32_input_conversion_rule(fmm):
    # Probe of how the tensor core reads fp32 operands in kind::tf32: a = 1 + 0.75 ulp(tf32)
    # rounds to 1 + 2^-10 to nearest and to 1 under truncation.  The test records which.
    k = 32
    A = np.zeros((128, k), np.float32)
    A[:, 0] = np.float32(1 + 2 ** -11 + 2 ** -12)
    A[:, 1] = np.float32(1 + 2 ** -12)            # 0.25 ulp: 1 under both rules
    B = np.zeros((k, 128), np.float32)
    B[0, :] = 1.0
    B[1, 1:] = 1.0
    C, _ = run(fmm, A, B, depth=0, precision="tf32")
    got0 = float(C[0, 0])
    assert got0 in (1.0, 1.0 + 2 ** -10), got0
    print("tf32 conversion:", "truncate" if got0 == 1.0 else "round-to-nearest")
    assert float(C[0, 1]) == got0 + 1.0


def test_blas_semantics(fmm):
    m, k, n = 130, 70, 90
    A = I.small_int((m, k), 5, r=3)
    B = I.small_int((k, n), 6, r=3)
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float64)
    Cnan = np.full((m, n), np.nan, np.float32)
    for d in (0, 1, 2, 3):
        C, _ = run(fmm, A, B, Cnan, alpha=2.0, beta=0.0, depth=d)
        assert np.array_equal(C, (2.0 * ref).astype(np.float32))
        C0 = I.small_int((m, n), 7, r=5)
        C, _ = run(fmm, A, B, C0, alpha=1.0, beta=-3.0, depth=d)
        assert np.array_equal(C, (ref - 3.0 * C0).astype(np.float32))
        Anan = np.full((m, k), np.nan, np.float32)
        C, _ = run(fmm, Anan, B, C0, alpha=0.0, beta=0.5, depth=d)
        assert np.array_equal(C, 0.5 * C0)


def test_degenerate_sizes(fmm):
    import torch
    C0 = I.small_int((5, 7), 8)
    C, _ = run(fmm, np.zeros((5, 0), np.float32), np.zeros((0, 7), np.float32), C0, beta=2.0)
    assert np.array_equal(C, 2.0 * C0)
    p = fmm.Plan(0, 7, 3)
    p(torch.empty((0, 3), device="cuda"), torch.empty((3, 7), device="cuda"), torch.empty((0, 7), device="cuda"))
    p.close()


def test_strided_operands(fmm):
    import torch
    m, k, n = 192, 160, 200
    lda, ldb, ldc = 171, 203, 211   # not multiples of 4: unaligned rows
    A = I.small_int((m, lda), 9)
    B = I.small_int((k, ldb), 10)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.zeros((m, ldc), device="cuda")
    ref = O.classical(A[:, :k].astype(np.int64), B[:, :n].astype(np.int64)).astype(np.float32)
    for d in (0, 1, 2):
        p = fmm.Plan(m, n, k, lda, ldb, ldc, depth=d)
        p(dA, dB, dC)
        torch.cuda.synchronize()
        got = dC.cpu().numpy()
        assert np.array_equal(got[:, :n], ref)
        assert np.all(got[:, n:] == 0)
        p.close()


# --- odd sizes: peeling ------------------------------------------------------

@pytest.mark.parametrize("m,k,n,d", [(300, 200, 260, 2), (1000, 1000, 1000, 3), (517, 133, 389, 1), (20, 40, 60, 3)])
def test_peel_bit_exact_small_int(fmm, m, k, n, d):
    A = I.small_int((m, k), 5000 + m, r=2)
    B = I.small_int((k, n), 6000 + n, r=2)
    C, info = run(fmm, A, B, depth=d, odd="peel")
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
    assert np.array_equal(O.winograd(A, B, d, "peel"), ref)
    assert np.array_equal(C, ref)


@pytest.mark.parametrize("odd", ["pad", "peel"])
def test_odd_size_error_bound(fmm, odd):
    m = k = n = 1187  # odd at every level
    A, B = I.operands(m, k, n, I.seed_for(2, 3))
    C, _ = run(fmm, A, B, depth=3, odd=odd)
    assert O.error_metric(C, O.classical(A, B), A, B) <= FP32_BOUND


def test_peel_blas_semantics(fmm):
    m, k, n = 290, 150, 330
    A = I.small_int((m, k), 15, r=3)
    B = I.small_int((k, n), 16, r=3)
    C0 = I.small_int((m, n), 17, r=5)
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float64)
    C, _ = run(fmm, A, B, C0, alpha=2.0, beta=-1.0, depth=2, odd="peel")
    assert np.array_equal(C, (2.0 * ref - C0).astype(np.float32))


# --- residual check ------------------------------------------------------------

@pytest.mark.parametrize("fp64", [0, 1])
@pytest.mark.parametrize("m,k,n", [(700, 500, 600), (301, 203, 157)])
def test_freivalds_residual_matches_oracle_and_detects_error(fmm, fp64, m, k, n):
    # (301, 203, 157): rows of A and C not 16-byte aligned (one column at a
    # time) and column counts with a remainder of 4 in every pass
    import torch
    A = I.small_int((m, k), 21, r=3)
    B = I.small_int((k, n), 22, r=3)
    Cx = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
    Cx[123, 45 % n] += 1.0
    x = I.rademacher(n, 23)
    dA, dB, dC, dx = (torch.from_numpy(np.ascontiguousarray(t)).cuda() for t in (A, B, Cx, x))
    r = fmm.fmm_residual(dA, dB, dC, dx, fp64=bool(fp64))
    torch.cuda.synchronize()
    got = r.cpu().numpy()
    want = O.freivalds(A, B, Cx, x)
    assert np.array_equal(got, want)           # integer data: exact in both accumulations
    assert np.count_nonzero(got) == 1 and abs(got[123]) == 1.0


@pytest.mark.parametrize("fp64", [0, 1])
def test_freivalds_residual_strided_views(fmm, fp64):
    # row strides that are multiples of 4 with column counts that are not: the
    # 16-byte path for the first columns of every row, one at a time for the rest
    import torch
    m, k, n = 257, 130, 99
    A = I.small_int((m, k), 31, r=3)
    B = I.small_int((k, n), 32, r=3)
    Cx = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
    Cx[200, 98] -= 2.0
    x = I.rademacher(n, 33)

    def view(t, ld):
        buf = torch.zeros((t.shape[0], ld), dtype=torch.float32, device="cuda")
        buf[:, : t.shape[1]] = torch.from_numpy(t).cuda()
        return buf[:, : t.shape[1]]

    dA, dB, dC = view(A, 132), view(B, 100), view(Cx, 100)
    assert dA.stride(0) == 132 and dB.stride(0) == 100
    r = fmm.fmm_residual(dA, dB, dC, torch.from_numpy(x).cuda(), fp64=bool(fp64))
    torch.cuda.synchronize()
    got = r.cpu().numpy()
    assert np.array_equal(got, O.freivalds(A, B, Cx, x))
    assert np.count_nonzero(got) == 1 and abs(got[200]) == 2.0


# --- split-precision leaves (BF16x3, FP16x3) ----------------------------------

@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("m,k,n,d", [(256, 96, 384, 0), (300, 200, 260, 0), (512, 512, 512, 2), (300, 200, 260, 1)])
def test_split16_bit_exact_small_int(fmm, prec, m, k, n, d):
    A = I.small_int((m, k), 8000 + m + d, r=2)
    B = I.small_int((k, n), 8100 + n + d, r=2)
    C, _ = run(fmm, A, B, depth=d, precision=prec)
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
    assert np.array_equal(C, ref)


def _fp16_scale(x, bound=1.0):
    # largest power of two s with bound * max|x| * s <= 2^14
    m = float(np.max(np.abs(x))) * bound
    e = 14 - (np.frexp(m)[1])
    return 2.0 ** e


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
def test_split16_matches_three_product_model(fmm, prec):
    m, k, n = 256, 512, 256
    A, B = I.operands(m, k, n, 78, "normal")
    C, _ = run(fmm, A, B, depth=0, precision=prec)
    if prec == "bf16x3":
        Ah, Al = O.split_bf16(A)
        Bh, Bl = O.split_bf16(B)
        model = O.split_product(Ah, Al, Bh, Bl)
    else:
        sa, sb = _fp16_scale(A), _fp16_scale(B)
        Ah, Al = O.split_fp16(A, sa)
        Bh, Bl = O.split_fp16(B, sb)
        model = O.split_product(Ah, Al, Bh, Bl) / (sa * sb)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    assert np.max(np.abs(C - model) / scale) <= 4 * k * 2.0 ** -24
    # and the split model itself is within its own error of the exact product
    err = O.error_metric(C, O.classical(A, B), A, B)
    assert err <= SPLIT_BOUND[prec]


@pytest.mark.parametrize("prec,dist,d", [("bf16x3", "normal", 2), ("bf16x3", "uniform", 3),
                                         ("bf16x3", "loguniform", 3), ("fp16x3", "loguniform", 3),
                                         ("fp16x3", "uniform", 3), ("fp16x3", "loguniform", 4),
                                         ("tf32", "normal", 1), ("tf32", "uniform", 3)])
def test_split_precision_winograd_bounds(fmm, prec, dist, d):
    n = 1024
    A, B = I.operands(n, n, n, I.seed_for(3, d), dist)
    C, _ = run(fmm, A, B, depth=d, precision=prec)
    assert np.all(np.isfinite(C))
    err = O.error_metric(C, O.classical(A, B), A, B)
    assert err <= SPLIT_BOUND[prec], err


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
def test_split16_peel_and_strided(fmm, prec):
    m, k, n = 517, 333, 389
    A = I.small_int((m, k), 13000 + m, r=2)
    B = I.small_int((k, n), 13100 + n, r=2)
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
    C, _ = run(fmm, A, B, depth=2, precision=prec, odd="peel")
    assert np.array_equal(C, ref)
    C, _ = run(fmm, A, B, depth=3, precision=prec, leaf_tile=128)
    assert np.array_equal(C, ref)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "tf32"])
@pytest.mark.parametrize("m,k,n,d", [(1024, 1024, 1024, 4), (1100, 900, 1300, 4), (800, 1024, 640, 3)])
def test_deep_recursion_bit_exact(fmm, prec, m, k, n, d):
    # depth >= 3 runs the bottom two levels of additions as fused passes
    A = I.small_int((m, k), 15000 + m + d, r=1)
    B = I.small_int((k, n), 15100 + n + d, r=1)
    C, info = run(fmm, A, B, depth=d, precision=prec)
    assert info["depth"] == d
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
    assert np.array_equal(C, ref)


# --- leaves on CTA pairs (cta_group::2, 256 x 256 tiles) ----------------------

@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16x3", "tf32"])
@pytest.mark.parametrize("m,k,n,d", [(256, 64, 256, 0), (300, 200, 260, 0), (777, 333, 515, 0), (1100, 900, 1300, 2),
                                     (512, 512, 512, 3), (1, 1, 1, 0), (640, 480, 704, 1)])
def test_pair_leaves_bit_exact(fmm, prec, m, k, n, d):
    A = I.small_int((m, k), 16000 + m + d, r=2)
    B = I.small_int((k, n), 16100 + n + d, r=2)
    C, info = run(fmm, A, B, depth=d, precision=prec, leaf_tile=512)
    assert info["leaf_tile"] == 512
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
    assert np.array_equal(C, ref)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "tf32"])
@pytest.mark.parametrize("tile", [512, 256, 128])
@pytest.mark.parametrize("n", [560, 912, 1030])
def test_narrow_last_tile_column_bit_exact(fmm, prec, tile, n):
    # depth 1 with leaves of K = 1024 runs the dynamic tile order, under which
    # the last tile column of each leaf issues MMAs of the valid width rounded
    # up to 32 (leaf widths 280, 456, 516: remainders 24, 200 / 72 and 4)
    m, k = 600, 2048
    A = I.small_int((m, k), 17000 + n + tile, r=1)
    B = I.small_int((k, n), 17100 + n + tile, r=1)
    C, info = run(fmm, A, B, depth=1, precision=prec, leaf_tile=tile)
    assert (info["depth"], info["leaf_tile"]) == (1, tile)
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
    assert np.array_equal(C, ref)


def test_pair_leaves_float_and_blas(fmm):
    n = 1024
    A, B = I.operands(n, n, n, I.seed_for(1, 21), "normal")
    C0 = I.uniform((n, n), 17)
    for d in (0, 2):
        C, _ = run(fmm, A, B, C0, alpha=0.5, beta=-2.0, depth=d, leaf_tile=512)
        ref = O.gemm(0.5, A, B, -2.0, C0)
        assert np.max(np.abs(C - ref)) / (np.abs(A).max() * np.abs(B).max() * n) <= FP32_BOUND
        single, _ = run(fmm, A, B, C0, alpha=0.5, beta=-2.0, depth=d, leaf_tile=256)
        assert np.max(np.abs(C - single)) / (np.abs(A).max() * np.abs(B).max() * n) <= FP32_BOUND


# --- algorithmic bytes of the addition phases -----------------------------------

def test_phase_bytes_closed_forms(fmm):
    import torch
    n = 1024
    A = torch.rand(n, n, device="cuda")
    B = torch.rand(n, n, device="cuda")
    C = torch.empty(n, n, device="cuda")
    # depth 0 (FP32): the operands are read once; B is written as raw + lo
    # planes, while a 16-byte aligned A serves as its own raw plane and only its
    # lo plane is written
    p = fmm.Plan(n, n, n, depth=0)
    p(A, B, C)
    torch.cuda.synchronize()
    assert p.phase_bytes() == {"pre_bytes": n * n * (4 + 4) + n * n * (4 + 8), "post_bytes": 0}
    p.close()
    # an A that starts off the 16-byte grid is split into both planes
    Aoff = torch.empty(n * n + 1, device="cuda")[1:].view(n, n)
    Aoff.copy_(A)
    p = fmm.Plan(n, n, n, depth=0)
    p(Aoff, B, C)
    torch.cuda.synchronize()
    assert p.phase_bytes() == {"pre_bytes": 2 * n * n * (4 + 8), "post_bytes": 0}
    p.close()
    # depth 2: root in, 49 leaf operands per side out (raw + lo fp32 planes);
    # 49 leaf products in, C out (read too when beta != 0)
    h = n // 4
    for beta, c_passes in ((0.0, 1), (0.5, 2)):
        p = fmm.Plan(n, n, n, depth=2)
        p(A, B, C, beta=beta)
        torch.cuda.synchronize()
        assert p.phase_bytes() == {"pre_bytes": 2 * n * n * 4 + 2 * 49 * h * h * 8,
                                   "post_bytes": 49 * h * h * 4 + c_passes * n * n * 4}
        p.close()
    # depth 3: all three levels in one pass per side (B transposed through
    # shared memory on the way): root in, 343 leaf operands out
    h3 = n // 8
    p = fmm.Plan(n, n, n, depth=3)
    p(A, B, C)
    torch.cuda.synchronize()
    assert p.phase_bytes() == {"pre_bytes": 2 * n * n * 4 + 2 * 343 * h3 * h3 * 8,
                               "post_bytes": 343 * h3 * h3 * 4 + n * n * 4}
    p.close()
    # BF16X3 planes are 2 + 2 bytes per element
    p = fmm.Plan(n, n, n, depth=2, precision="bf16x3")
    p(A, B, C)
    torch.cuda.synchronize()
    assert p.phase_bytes()["pre_bytes"] == 2 * n * n * 4 + 2 * 49 * h * h * 4
    p.close()


# --- failure path of the bounded device waits -----------------------------------

def test_wait_timeout_is_reported_and_context_stays_usable(fmm):
    import time
    import torch
    n = 256
    A = I.small_int((n, n), 71, r=2)
    B = I.small_int((n, n), 72, r=2)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty((n, n), device="cuda")
    p = fmm.Plan(n, n, n, depth=1)
    t0 = time.perf_counter()
    p.wait_selftest(limit_ns=20_000_000)   # a barrier nothing signals, 20 ms limit
    assert p.device_status() == fmm.FMM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert p.device_status() == fmm.FMM_OK   # the read cleared the word
    p(dA, dB, dC)
    torch.cuda.synchronize()
    assert p.device_status() == fmm.FMM_OK
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
    assert np.array_equal(dC.cpu().numpy(), ref)
    p.close()


# --- classical recursion of Table 1 (RMUL): k-blocks accumulated in C -------------

@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3", "fp16x3"])
@pytest.mark.parametrize("m,k,n,d", [(300, 200, 260, 1), (512, 512, 512, 2), (777, 333, 515, 3), (130, 5, 90, 3),
                                     (64, 1, 64, 2)])
def test_rmul_bit_exact_small_int(fmm, prec, m, k, n, d):
    A = I.small_int((m, k), 18000 + m + d, r=2)
    B = I.small_int((k, n), 18100 + n + d, r=2)
    C, info = run(fmm, A, B, depth=d, precision=prec, algo="classical")
    assert (info["depth"], info["algo"]) == (d, 1)
    ref = O.classical(A.astype(np.int64), B.astype(np.int64))
    assert np.array_equal(O.rmul(A.astype(np.int64), B.astype(np.int64), d), ref)
    assert np.array_equal(C, ref.astype(np.float32))


def test_rmul_float_and_blas(fmm):
    n = 1024
    A, B = I.operands(n, n, n, I.seed_for(1, 23), "normal")
    C0 = I.uniform((n, n), 19)
    for d in (1, 3):
        C, _ = run(fmm, A, B, C0, alpha=0.5, beta=-2.0, depth=d, algo="classical")
        ref = O.gemm(0.5, A, B, -2.0, C0)
        assert np.max(np.abs(C - ref)) / (np.abs(A).max() * np.abs(B).max() * n) <= FP32_BOUND
    # beta is applied once, then the later k-blocks accumulate: a NaN-filled C with beta = 0 stays clean
    C, _ = run(fmm, A, B, np.full((n, n), np.nan, np.float32), beta=0.0, depth=2, algo="classical")
    assert np.all(np.isfinite(C))
    assert O.error_metric(C, O.classical(A, B), A, B) <= FP32_BOUND


@pytest.mark.parametrize("m,k,n,d,bn", [(2100, 900, 1337, 2, 512), (1300, 1100, 700, 1, 256), (1100, 333, 1500, 1, 512)])
def test_tile_peel_bit_exact_small_int(fmm, m, k, n, d, bn):
    # FMM_ODD_TILE: whole-tile core through the recursion, the rest as classical
    # border leaves; exact on small integers like every other mode
    A = I.small_int((m, k), 15000 + m + d, r=2)
    B = I.small_int((k, n), 15100 + n + d, r=2)
    C, info = run(fmm, A, B, depth=d, precision="fp32", leaf_tile=bn, odd="tile")
    assert info["depth"] == d and info["odd"] == 2
    ref = O.classical(A.astype(np.int64), B.astype(np.int64))
    assert np.array_equal(C, ref.astype(np.float32))


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16x3"])
def test_tile_peel_float_bound_and_blas(fmm, prec):
    m, k, n = 3000, 2600, 2800
    A, B = I.operands(m, k, n, 15200, "normal")
    C0 = I.uniform((m, n), 15201)
    C, _ = run(fmm, A, B, C0, alpha=-1.25, beta=0.5, depth=2, precision=prec, leaf_tile=512, odd="tile")
    err = O.error_metric(C, O.gemm(-1.25, A, B, 0.5, C0), A, B)
    assert err <= SPLIT_BOUND[prec], err


def test_auto_odd_mode_takes_tile_peel_when_remainders_are_small(fmm):
    m, k, n = 2100, 900, 2150      # depth 2 on pairs: granule 1024, remainders 52 and 102
    A = I.small_int((m, k), 15300, r=2)
    B = I.small_int((k, n), 15301, r=2)
    C, info = run(fmm, A, B, depth=2, precision="fp32", leaf_tile=512)
    assert info["odd"] == 2
    assert np.array_equal(C, O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32))
    C2, info2 = run(fmm, A, B, depth=2, precision="fp32", leaf_tile=512, odd="auto")
    assert info2["odd"] == 2 and np.array_equal(C2, C)
    _, info3 = run(fmm, A[:, :], B[:, :1500], depth=2, precision="fp32", leaf_tile=512)
    assert info3["odd"] == 0       # remainder 476 of 1024: padded
