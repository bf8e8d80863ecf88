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


def _max_depth(m, k, n):
    # the library's limit for a batched problem: depth <= 4, leaves >= 64 wide
    d = 4
    while d > 0 and (min(m, k, n) >> d) < 64:
        d -= 1
    return d


def _replay_ms(torch, bp, reps=5):
    bp.run()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        s.record()
        bp.run()
        e.record()
        torch.cuda.synchronize()
        ts.append(s.elapsed_time(e))
    return sorted(ts)[len(ts) // 2]


def test_batched_exhaustive_planner_per_class(F):
    # the library's own tuner: one depth per size class, whole-batch timings;
    # the plan it keeps is no slower than the fixed rule's, and exact on integers
    import torch
    probs = _problems(64, 9700, lo=128, hi=2048, mult=4)
    As, Bs, Cs = _upload(probs)
    fixed = F.BatchedPlan(As, Bs, Cs, planner="fixed")
    t_fixed = _replay_ms(torch, fixed)
    fixed.close()
    bp = F.BatchedPlan(As, Bs, Cs, planner="exhaustive")
    info = bp.info()
    by_class = {}
    for i, (A, B) in enumerate(probs):
        c = info["classes"][i]
        assert 0 <= c < info["nclasses"]
        m, k = A.shape
        n = B.shape[1]
        d = info["depths"][i]
        # members of a class share its depth, except where a member's own limit caps it
        by_class.setdefault(c, set()).add(d if d < _max_depth(m, k, n) else -1)
    assert all(len({x for x in v if x >= 0}) <= 1 for v in by_class.values())
    for c in Cs:
        c.fill_(float("nan"))
    t_ex = _replay_ms(torch, bp)
    for (A, B), Cd in zip(probs, Cs):
        ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
        assert np.array_equal(Cd.cpu().numpy(), ref)
    assert t_ex <= 1.10 * t_fixed, (t_ex, t_fixed)
    bp.close()


def _depth_preferring_model(F):
    # a hand-set cost model: predicted log(ms) = 5 - depth + 0.5 * (tile / 128),
    # features unstandardised, so the MLP planner must take every class to its
    # deepest level and the 256-wide tile
    p = np.zeros(F.NPARAM, dtype=np.float32)
    W1 = p[0:384].reshape(64, 6)
    W2 = p[448:448 + 4096].reshape(64, 64)
    W3 = p[448 + 4096 + 64:448 + 4096 + 64 + 64]
    W1[0, 3] = 1.0          # h1_0 = relu(depth)
    W1[1, 4] = 1.0          # h1_1 = relu(tile / 128)
    W2[0, 0] = 1.0
    W2[1, 1] = 1.0
    W3[0] = -1.0
    W3[1] = 0.5
    p[-1] = 5.0
    return p, np.zeros(6, np.float32), np.ones(6, np.float32)


def test_batched_mlp_planner_follows_the_model(F):
    # the hand-set model proposes every class at its deepest level on the 256
    # tile; the planner times that proposal against the fixed rule's plan as
    # whole batches and keeps the faster, so the plan is one of the two, exact
    # on integers and no slower than the fixed rule's (within timing noise)
    import torch
    probs = _problems(40, 9800, lo=128, hi=1500, mult=4)
    As, Bs, Cs = _upload(probs)
    fixed = F.BatchedPlan(As, Bs, Cs, planner="fixed")
    fixed_info = fixed.info()
    t_fixed = _replay_ms(torch, fixed)
    fixed.close()
    params, mean, std = _depth_preferring_model(F)
    F.fmm_set_cost_model(params, mean, std)
    try:
        bp = F.BatchedPlan(As, Bs, Cs, planner="mlp")
    finally:
        F.fmm_set_cost_model(None)
    info = bp.info()
    deepest = [_max_depth(A.shape[0], A.shape[1], B.shape[1]) for A, B in probs]
    if info["leaf_tile"] == 256:
        assert info["depths"] == deepest                      # the model's proposal was faster
    else:
        assert info["leaf_tile"] == fixed_info["leaf_tile"]   # the fixed rule's plan was faster
        assert info["depths"] == fixed_info["depths"]
    assert any(d != f for d, f in zip(deepest, fixed_info["depths"]))   # the two candidates differ
    for c in Cs:
        c.fill_(float("nan"))
    t_mlp = _replay_ms(torch, bp)
    for (A, B), Cd in zip(probs, Cs):
        ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
        assert np.array_equal(Cd.cpu().numpy(), ref)
    assert t_mlp <= 1.10 * t_fixed, (t_mlp, t_fixed)
    bp.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_batched_aligned_and_unaligned_a(F, prec):
    # depth-0 problems read an aligned A in place (FP32: only its lo plane is
    # written); an A that starts off a 16-byte boundary or has an odd row stride
    # goes through its own planes; both exact on integers
    import torch
    shapes = [(300, 257, 190), (128, 640, 512), (77, 129, 301), (512, 512, 512)]
    probs, As, Bs, Cs = [], [], [], []
    for i, (m, k, n) in enumerate(shapes):
        B = I.small_int((k, n), 9950 + i, r=2)
        if i % 2 == 0:   # a view one element in: 4-byte aligned only, row stride k + 3
            A = I.small_int((m, k + 3), 9900 + i, r=2)
            dA = torch.from_numpy(A).cuda()[:, 1:k + 1]
            A = A[:, 1:k + 1]
        else:            # contiguous, 16-byte aligned rows (k is a multiple of 4)
            A = I.small_int((m, k), 9900 + i, r=2)
            dA = torch.from_numpy(A).cuda()
        probs.append((A, B))
        As.append(dA)
        Bs.append(torch.from_numpy(B).cuda())
        Cs.append(torch.full((m, n), float("nan"), device="cuda"))
    bp = F.BatchedPlan(As, Bs, Cs, precision=prec, cutoff=8192)
    assert all(d == 0 for d in bp.info()["depths"])
    bp.run()
    torch.cuda.synchronize()
    for (A, B), Cd in zip(probs, Cs):
        ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
        assert np.array_equal(Cd.cpu().numpy(), ref)
    bp.close()
