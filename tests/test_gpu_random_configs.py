"""GPU parity over seeded random plan configurations: shape, depth, precision,
odd-size mode, last-level fusion, leaf tile, alpha/beta and operand residence
drawn together, on small-integer data, where every configuration must equal
the int64 product of the definition (c_ij = sum_k a_ik b_kj, Sec. 3.3) bit for
bit.

Exactness: with entries in [-r, r] a level's sums S, T grow at most 4x, so a
leaf product of depth d is bounded by (K / 2^d) r^2 16^d and the post-additions
multiply that by at most 4^d; the draw keeps that bound below 2^24 (fp32's
exact-integer range), and the split precisions hold |S|, |T| <= r 4^d exactly
in their hi parts (bf16: 256, tf32: 2048, fp16 after power-of-two scaling).
alpha, beta and C are powers of two and small integers, so alpha AB + beta C
is exact too.  Configurations the library refuses (FMM_ERR_UNSUPPORTED) are
counted, and most draws must run.
"""
import numpy as np
import pytest

import oracle.fmm_oracle as O
from paper_1205_2927_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N_CONFIGS = 200


def _draw(rng):
    d = int(rng.integers(0, 4))
    r = 2 if d <= 2 else 1
    kmax = 1500 if d <= 2 else 300
    # the exactness bound of the module docstring, with a margin
    while d > 0 and kmax * r * r * 8 ** d * 4 ** d >= 2 ** 23:
        kmax //= 2
    lo = max(1, 8 << d) if d > 0 else 1
    m = int(np.exp(rng.uniform(np.log(lo), np.log(1600))))
    n = int(np.exp(rng.uniform(np.log(lo), np.log(1600))))
    k = int(np.exp(rng.uniform(np.log(lo), np.log(max(lo + 1, kmax)))))
    cfg = dict(depth=d, precision=str(rng.choice(["fp32", "fp32", "bf16x3", "fp16x3", "tf32"])),
               odd=str(rng.choice(["pad", "peel", "tile", "auto"])), fuse_last=int(rng.choice([-1, 0, 1])),
               leaf_tile=int(rng.choice([0, 128, 256, 512])))
    host = bool(rng.random() < 0.2)
    if host:
        cfg["odd"] = str(rng.choice(["pad", "auto"]))
        cfg["host_operands"] = 1
        cfg["host_copy"] = str(rng.choice(["default", "engine", "sm"]))
    alpha = float(rng.choice([1.0, -1.0, 2.0, 0.5]))
    beta = float(rng.choice([0.0, 0.0, 1.0, -2.0]))
    return m, k, n, r, cfg, alpha, beta, host


def test_random_configurations_bit_exact():
    import torch
    from paper_1205_2927_gb300 import fmm as F
    rng = np.random.default_rng(I.seed_for(6, 0))
    ran, refused, seen = 0, 0, []
    for i in range(N_CONFIGS):
        m, k, n, r, cfg, alpha, beta, host = _draw(rng)
        A = I.small_int((m, k), I.seed_for(6, 1) + i, r=r)
        B = I.small_int((k, n), I.seed_for(6, 2) + i, r=r)
        C0 = I.small_int((m, n), I.seed_for(6, 3) + i, r=3)
        ref = (alpha * O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float64)
               + beta * C0.astype(np.float64)).astype(np.float32)
        try:
            p = F.Plan(m, n, k, **cfg)
        except F.FmmError as e:
            if e.status == F.FMM_ERR_UNSUPPORTED:
                refused += 1
                continue
            raise
        pad = (0, 0, 0)
        if host:
            tA, tB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
            tC = torch.from_numpy(C0.copy()).pin_memory()
        else:
            if rng.random() < 0.35:
                # operands as views of wider buffers: row strides that need not
                # be multiples of 4, NaN in the columns beyond each view
                p.close()
                pad = tuple(int(x) for x in rng.integers(1, 9, size=3))
                p = F.Plan(m, n, k, lda=k + pad[0], ldb=n + pad[1], ldc=n + pad[2], **cfg)
            fA = torch.full((m, k + pad[0]), float("nan"), device="cuda")
            fB = torch.full((k, n + pad[1]), float("nan"), device="cuda")
            fC = torch.full((m, n + pad[2]), float("nan"), device="cuda")
            tA, tB, tC = fA[:, :k], fB[:, :n], fC[:, :n]
            tA.copy_(torch.from_numpy(A))
            tB.copy_(torch.from_numpy(B))
            tC.copy_(torch.from_numpy(C0))
        p(tA, tB, tC, alpha=alpha, beta=beta)
        torch.cuda.synchronize()
        status = p.device_status()
        info = dict(p.info)
        p.close()
        got = tC.cpu().numpy()
        where = (m, k, n, pad, cfg, alpha, beta, info)
        assert status == 0, where
        assert np.array_equal(got, ref), (where, float(np.max(np.abs(got - ref))))
        if not host:
            assert torch.isnan(fC[:, n:]).all(), where    # nothing written beyond C
        ran += 1
        seen.append((cfg["depth"], cfg["precision"], info.get("odd"), info.get("fuse_last"), host))
    print(f"random configurations: {ran} run bit-exact, {refused} refused as unsupported")
    assert ran >= int(0.75 * N_CONFIGS), (ran, refused)
    # the draw reached the paths it is meant to cross
    assert {d for d, *_ in seen} >= {0, 1, 2, 3}
    assert {p for _, p, *_ in seen} >= {"fp32", "bf16x3", "fp16x3", "tf32"}
    assert any(h for *_, h in seen) and any(f for *_, f, _ in seen)


# per-term error bounds of the split forms against the FP32 bound (the same
# derivation as the full-size tests: BF16x3 3 * 2^-16, TF32 2^-10 per term)
SPLIT_BOUND = {"fp32": 2e-6, "fp16x3": 2e-6, "bf16x3": 4.8e-5, "tf32": 1.0e-3}


def test_random_configurations_float_bound():
    # float operands make every lo plane non-zero (integer data leaves lo = 0 in
    # every split), so this draw checks the lo paths the exact test cannot
    import torch
    from paper_1205_2927_gb300 import fmm as F
    rng = np.random.default_rng(I.seed_for(6, 10))
    worst = {}
    for i in range(40):
        m, k, n, _, cfg, _, _, host = _draw(rng)
        k = max(k, int(rng.integers(64, 1600)))   # floats need no exactness bound on K
        A, B = I.operands(m, k, n, I.seed_for(6, 11) + i, str(rng.choice(["normal", "loguniform"])))
        p = F.Plan(m, n, k, **cfg)
        if host:
            tA, tB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
            tC = torch.full((m, n), float("nan")).pin_memory()
        else:
            tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
            tC = torch.full((m, n), float("nan"), device="cuda")
        p(tA, tB, tC)
        torch.cuda.synchronize()
        assert p.device_status() == 0
        p.close()
        err = O.error_metric(tC.cpu().numpy(), O.classical(A, B), A, B)
        prec = cfg["precision"]
        worst[prec] = max(worst.get(prec, 0.0), err)
        assert err <= SPLIT_BOUND[prec], (m, k, n, cfg, err)
    print("worst error per precision:", {p: f"{e:.2e}" for p, e in worst.items()})


def test_random_batched_sets_bit_exact():
    # batched sets of random size and shape mix (including K = 0 and alpha = 0
    # members), random precision, leaf tile and cut-off, per-problem alpha/beta
    import torch
    from paper_1205_2927_gb300 import fmm as F
    rng = np.random.default_rng(I.seed_for(6, 20))
    for t in range(8):
        count = int(rng.integers(1, 40))
        probs, al, be = [], [], []
        for i in range(count):
            m, n = (int(x) for x in rng.integers(1, 700, size=2))
            k = 0 if rng.random() < 0.05 else int(rng.integers(1, 700))
            A = I.small_int((m, k), I.seed_for(6, 21) + 100 * t + i, r=2)
            B = I.small_int((k, n), I.seed_for(6, 22) + 100 * t + i, r=2)
            C0 = I.small_int((m, n), I.seed_for(6, 23) + 100 * t + i, r=3)
            probs.append((A, B, C0))
            al.append(0.0 if rng.random() < 0.05 else float(rng.choice([1.0, -1.0, 2.0])))
            be.append(float(rng.choice([0.0, 1.0, -0.5])))
        prec = str(rng.choice(["fp32", "bf16x3", "fp16x3", "tf32"]))
        tile = int(rng.choice([128, 256, 512])) if prec == "tf32" else int(rng.choice([256, 512]))
        cutoff = int(rng.choice([128, 4096]))   # depth <= 2 below 700: intermediates stay exact
        As = [torch.from_numpy(A).cuda() for A, _, _ in probs]
        Bs = [torch.from_numpy(B).cuda() for _, B, _ in probs]
        Cs = [torch.from_numpy(C0.copy()).cuda() for _, _, C0 in probs]
        bp = F.BatchedPlan(As, Bs, Cs, alpha=al, beta=be, precision=prec, leaf_tile=tile, cutoff=cutoff)
        bp.run()
        torch.cuda.synchronize()
        for (A, B, C0), a, b, Cd in zip(probs, al, be, Cs):
            ref = (a * O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float64)
                   + b * C0.astype(np.float64)).astype(np.float32)
            assert np.array_equal(Cd.cpu().numpy(), ref), (t, A.shape, B.shape, prec, tile, cutoff, a, b)
        bp.close()
