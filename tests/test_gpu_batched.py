"""GPU parity of the batched path (one persistent leaf launch over many uneven
problems), including CUDA-graph capture and replay."""
import numpy as np
import pytest

import oracle.fmm_oracle as O
from paper_1205_2927_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1205_2927_gb300 import fmm
    return fmm


def _problems(count, seed, lo=16, hi=700, mult=1):
    shapes = I.batched_shapes(count, seed, lo=lo, hi=hi, multiple=mult)
    probs = []
    for i, (m, k, n) in enumerate(shapes):
        A = I.small_int((m, k), seed + 7 * i, r=2)
        B = I.small_int((k, n), seed + 7 * i + 3, r=2)
        probs.append((A, B))
    return probs


def _upload(probs):
    import torch
    As = [torch.from_numpy(A).cuda() for A, _ in probs]
    Bs = [torch.from_numpy(B).cuda() for _, B in probs]
    Cs = [torch.full((A.shape[0], B.shape[1]), float("nan"), device="cuda") for A, B in probs]
    return As, Bs, Cs


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16x3", "tf32"])
@pytest.mark.parametrize("cutoff,bn", [(4096, 256), (64, 256), (64, 128), (4096, 512), (64, 512)])
def test_batched_bit_exact_small_int(F, cutoff, bn, prec):
    import torch
    probs = _problems(48, 9100, lo=16, hi=700, mult=1)
    As, Bs, Cs = _upload(probs)
    bp = F.BatchedPlan(As, Bs, Cs, cutoff=cutoff, leaf_tile=bn, precision=prec)
    info = bp.info()
    if cutoff == 64:
        assert max(info["depths"]) >= 1  # some problems recurse
    bp.run()
    torch.cuda.synchronize()
    for (A, B), Cd in zip(probs, Cs):
        ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
        assert np.array_equal(Cd.cpu().numpy(), ref)
    bp.close()


@pytest.mark.parametrize("bn", [0, 512])
def test_batched_alpha_beta_and_float_bound(F, bn):
    # bn 512: leaf tiles of 256 x 256 on CTA pairs (the depth-0 problems and the
    # leaves of the recursing ones in the same persistent launch)
    import torch
    shapes = I.batched_shapes(24, 9200, lo=64, hi=1024, multiple=4)
    probs = [I.operands(m, k, n, 9300 + i) for i, (m, k, n) in enumerate(shapes)]
    As = [torch.from_numpy(A).cuda() for A, _ in probs]
    Bs = [torch.from_numpy(B).cuda() for _, B in probs]
    C0 = [I.uniform((A.shape[0], B.shape[1]), 9400 + i) for i, (A, B) in enumerate(probs)]
    Cs = [torch.from_numpy(c).cuda() for c in C0]
    bp = F.BatchedPlan(As, Bs, Cs, alpha=0.5, beta=2.0, cutoff=256, leaf_tile=bn)
    bp.run()
    torch.cuda.synchronize()
    for (A, B), c0, Cd in zip(probs, C0, Cs):
        ref = O.gemm(0.5, A, B, 2.0, c0)
        err = np.max(np.abs(Cd.cpu().numpy() - ref)) / (np.abs(A).max() * np.abs(B).max() * A.shape[1])
        assert err <= 2e-6


@pytest.mark.parametrize("bn", [256, 512])
def test_batched_fp16x3_scales_per_problem(F, bn):
    # operands of very different magnitudes in one launch: each problem gets its
    # own power-of-two scales (a shared scale would push the small problems'
    # lo halves below fp16's range); the recursing problems included
    import torch
    shapes = I.batched_shapes(24, 9600, lo=64, hi=900, multiple=4)
    probs, As, Bs, Cs = [], [], [], []
    for i, (m, k, n) in enumerate(shapes):
        s = 4.0 ** ((i % 7) - 3)               # magnitudes from 2^-6 to 2^6
        A, B = I.operands(m, k, n, 9700 + i, "normal")
        A = (A * s).astype(np.float32)
        B = (B / s).astype(np.float32)
        probs.append((A, B))
        As.append(torch.from_numpy(A).cuda())
        Bs.append(torch.from_numpy(B).cuda())
        Cs.append(torch.full((m, n), float("nan"), device="cuda"))
    bp = F.BatchedPlan(As, Bs, Cs, cutoff=128, leaf_tile=bn, precision="fp16x3")
    assert max(bp.info()["depths"]) >= 1
    bp.run()
    torch.cuda.synchronize()
    for (A, B), Cd in zip(probs, Cs):
        ref = O.classical(A, B)
        err = np.max(np.abs(Cd.cpu().numpy() - ref)) / (np.abs(A).max() * np.abs(B).max() * A.shape[1])
        assert err <= 2e-6, err
    bp.close()


def test_batched_graph_capture_replay(F):
    import torch
    probs = _problems(32, 9500, lo=32, hi=512, mult=4)
    As, Bs, Cs = _upload(probs)
    bp = F.BatchedPlan(As, Bs, Cs, cutoff=128)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bp.run(s)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for C in Cs:
        C.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bp.run(torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    for (A, B), Cd in zip(probs, Cs):
        ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
        assert np.array_equal(Cd.cpu().numpy(), ref)
    # replay again after changing inputs in place: the graph reads the new values
    for A in As:
        A.mul_(-1)
    g.replay()
    torch.cuda.synchronize()
    for (A, B), Cd in zip(probs, Cs):
        ref = O.classical(-A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
        assert np.array_equal(Cd.cpu().numpy(), ref)


def test_one_shot_gemm_batched_and_unsupported_forms(F):
    # fmm_gemm_batched: plan + run + release in one call, through the binding
    import torch
    probs = _problems(20, 9500, lo=16, hi=600, mult=1)
    As, Bs, Cs = _upload(probs)
    ws = F.fmm_gemm_batched(As, Bs, Cs, cutoff=128)
    torch.cuda.synchronize()
    del ws
    for (A, B), Cd in zip(probs, Cs):
        ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
        assert np.array_equal(Cd.cpu().numpy(), ref)
    # forms the batched path rejects before any device work
    for kw in ({"odd": "peel"}, {"algo": "classical"}):
        with pytest.raises(F.FmmError) as e:
            F.fmm_gemm_batched(As, Bs, Cs, **kw)
        assert e.value.status == 6
