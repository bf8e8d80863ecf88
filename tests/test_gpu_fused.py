"""The last Winograd level fused into the CTA-pair leaf launch (fuse_last = 1).

The fused launch folds each node's seven products into its four output
quadrants in the U-chain's own order of fp32 additions, so its result must
equal the unfused plan's (products stored, then the post-addition pass) bit for
bit on any data; on small integers both equal the exact product.  Sizes span
several 256 x 256 pair tiles per leaf with ragged last tiles."""
import numpy as np
import pytest

import oracle.fmm_oracle as O
from paper_1205_2927_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP32_BOUND = 2e-6


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
    ws = plan.workspace_bytes
    plan.close()
    return dC.cpu().numpy(), ws


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16x3"])
@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("m,k,n", [(1500, 1300, 1700), (2048, 2048, 2048), (2100, 900, 1337)])
def test_fused_equals_unfused_bitwise(fmm, prec, d, m, k, n):
    A, B = I.operands(m, k, n, 7100 + d + m % 97)
    C0 = I.uniform((m, n), 7200 + n % 89)
    kw = dict(depth=d, precision=prec, leaf_tile=512)
    fused, ws_f = run(fmm, A, B, C0, alpha=0.75, beta=0.5, fuse_last=1, **kw)
    plain, ws_p = run(fmm, A, B, C0, alpha=0.75, beta=0.5, fuse_last=-1, **kw)
    assert np.array_equal(fused, plain)
    if prec == "fp32":
        err = O.error_metric(fused, O.gemm(0.75, A, B, 0.5, C0), A, B)
        assert err <= FP32_BOUND, err


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("m,k,n", [(1024, 640, 768), (1300, 1100, 900)])
def test_fused_bit_exact_small_int(fmm, d, m, k, n):
    A = I.small_int((m, k), 7300 + m + d, r=2)
    B = I.small_int((k, n), 7400 + n + d, r=2)
    C, _ = run(fmm, A, B, depth=d, precision="fp32", leaf_tile=512, fuse_last=1)
    ref = O.classical(A.astype(np.int64), B.astype(np.int64))
    assert np.array_equal(C, ref.astype(np.float32))


def test_fused_peel_equals_unfused(fmm):
    m, k, n = 1187, 1001, 1303
    A, B = I.operands(m, k, n, 7500)
    kw = dict(depth=2, precision="fp32", leaf_tile=512, odd="peel")
    fused, _ = run(fmm, A, B, fuse_last=1, **kw)
    plain, _ = run(fmm, A, B, fuse_last=-1, **kw)
    assert np.array_equal(fused, plain)


def test_fused_error_bound_and_smaller_workspace(fmm):
    n = 2048
    A, B = I.operands(n, n, n, I.seed_for(1, 11))
    C, ws_f = run(fmm, A, B, depth=3, precision="fp32", leaf_tile=512, fuse_last=1)
    _, ws_p = run(fmm, A, B, depth=3, precision="fp32", leaf_tile=512, fuse_last=-1)
    assert O.error_metric(C, O.classical(A, B), A, B) <= FP32_BOUND
    assert ws_f < ws_p + 64 * 1024 * 1024 + 1


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("m,k,n", [(4096, 4096, 4096), (4200, 4100, 4300)])
def test_fused_depth4_equals_unfused_bitwise(fmm, prec, m, k, n):
    # depth 4: the leaf launch writes the 343 level-3 node outputs, the
    # three-level post pass folds them into C
    A, B = I.operands(m, k, n, 7600 + m % 89)
    kw = dict(depth=4, precision=prec, leaf_tile=512, odd="pad")
    fused, _ = run(fmm, A, B, fuse_last=1, **kw)
    plain, _ = run(fmm, A, B, fuse_last=-1, **kw)
    assert np.array_equal(fused, plain)
    bound = 2e-6 if prec == "fp32" else 4.8e-5
    assert O.error_metric(fused, O.classical(A, B), A, B) <= bound
