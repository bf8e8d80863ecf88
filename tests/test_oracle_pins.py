"""Pins of the CPU oracle against facts that do not come from the oracle itself:
brute-force triple loops, closed forms, a symbolic identity, exact integer
arithmetic, invariants, and library routines for the special cases that reduce
to them.  Each mutation test plants a plausible mistake in a copy of an oracle
step and checks that a pin catches it."""
import fractions
import itertools
import math
import os

import numpy as np
import pytest

import oracle.fmm_oracle as O
from paper_1205_2927_gb300 import inputs as I


def brute_matmul(A, B):
    """Pure-Python triple loop (exact for Python ints and Fractions)."""
    m, k = len(A), len(A[0]) if len(A) else 0
    n = len(B[0]) if len(B) else 0
    return [[sum(A[i][p] * B[p][j] for p in range(k)) for j in range(n)] for i in range(m)]


# --- classical product -------------------------------------------------------

@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (3, 5, 2), (7, 4, 6), (9, 9, 9)])
def test_classical_matches_triple_loop_int(m, k, n):
    A = I.small_int((m, k), 11 + m, r=9).astype(np.int64)
    B = I.small_int((k, n), 12 + n, r=9).astype(np.int64)
    ref = brute_matmul(A.tolist(), B.tolist())
    assert O.classical(A, B).tolist() == ref


def test_classical_matches_triple_loop_float_exactly():
    # float entries converted to exact rationals: float64 result must be the
    # correctly rounded exact sum within a few ulps
    A = I.uniform((5, 7), 3)
    B = I.uniform((7, 4), 4)
    exact = brute_matmul([[fractions.Fraction(float(x)) for x in r] for r in A.tolist()],
                         [[fractions.Fraction(float(x)) for x in r] for r in B.tolist()])
    C = O.classical(A, B)
    for i in range(5):
        for j in range(4):
            assert abs(C[i, j] - float(exact[i][j])) <= 8 * 2.0 ** -52 * 7


def test_closed_forms():
    m, k, n = 13, 17, 11
    assert np.all(O.classical(np.ones((m, k)), np.ones((k, n))) == k)
    A = I.uniform((m, k), 5).astype(np.float64)
    assert np.array_equal(O.classical(A, np.eye(k)), A)
    d = np.arange(1, m + 1, dtype=np.float64)
    B = I.uniform((m, n), 6).astype(np.float64)
    assert np.array_equal(O.classical(np.diag(d), B), d[:, None] * B)


def test_gemm_blas_semantics():
    A = I.uniform((4, 3), 1)
    B = I.uniform((3, 5), 2)
    C = np.full((4, 5), np.nan, dtype=np.float32)
    out = O.gemm(1.5, A, B, 0.0, C)          # beta = 0: C never read
    assert np.all(np.isfinite(out))
    Anan = np.full((4, 3), np.nan, dtype=np.float32)
    C2 = I.uniform((4, 5), 3)
    out = O.gemm(0.0, Anan, B, 2.0, C2)      # alpha = 0: A, B never read
    assert np.array_equal(out, 2.0 * C2.astype(np.float64))
    out = O.gemm(1.0, np.zeros((4, 0)), np.zeros((0, 5)), 0.5, C2)  # k = 0
    assert np.array_equal(out, 0.5 * C2.astype(np.float64))


# --- Eq. 1 -------------------------------------------------------------------

@pytest.mark.parametrize("m,n", [(1, 1), (2, 3), (5, 4), (7, 7), (6, 9)])
def test_quadrant_shapes_eq1(m, n):
    D = np.arange(m * n).reshape(m, n)
    D0, D1, D2, D3 = O.quadrants(D)
    assert D0.shape == (math.ceil(m / 2), math.ceil(n / 2))
    assert D3.shape == (m // 2, n // 2)
    assert D1.shape == (math.ceil(m / 2), n // 2)
    assert D2.shape == (m // 2, math.ceil(n / 2))
    top = np.concatenate([D0, D1], axis=1)
    bot = np.concatenate([D2, D3], axis=1)
    assert np.array_equal(np.concatenate([top, bot], axis=0), D)


def test_odd_border_counts_golden():
    # tests/golden/eq1_odd_border_counts.txt: the quadrant shapes of Eq. 1 and
    # the paper's count of C0's border elements (2N - 1) for odd n = 2N - 1
    path = os.path.join(os.path.dirname(__file__), "golden", "eq1_odd_border_counts.txt")
    rows = [list(map(int, l.split())) for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 5
    for n, r0, c0, r3, c3, extra in rows:
        D0, _, _, D3 = O.quadrants(np.zeros((n, n)))
        assert D0.shape == (r0, c0) and D3.shape == (r3, c3)
        assert D0.size - D3.size == extra == n


# --- Table 1 -------------------------------------------------------------------

@pytest.mark.parametrize("m,k,n,d", [(8, 8, 8, 1), (9, 7, 5, 2), (16, 3, 12, 3), (1, 5, 1, 2)])
def test_rmul_exact_int(m, k, n, d):
    A = I.small_int((m, k), 20 + m).astype(np.int64)
    B = I.small_int((k, n), 21 + n).astype(np.int64)
    assert np.array_equal(O.rmul(A, B, d), O.classical(A, B))


# --- Winograd step: symbolic identity ----------------------------------------

def test_winograd_step_symbolic_identity():
    sympy = pytest.importorskip("sympy")
    # blocks are non-commuting symbols, so the identity holds for matrix blocks
    a = sympy.symbols("a11 a12 a21 a22", commutative=False)
    b = sympy.symbols("b11 b12 b21 b22", commutative=False)
    A11, A12, A21, A22 = a
    B11, B12, B21, B22 = b
    S1 = A21 + A22; S2 = S1 - A11; S3 = A11 - A21; S4 = A12 - S2
    T1 = B12 - B11; T2 = B22 - T1; T3 = B22 - B12; T4 = T2 - B21
    P = [A11 * B11, A12 * B21, S4 * B22, A22 * T4, S1 * T1, S2 * T2, S3 * T3]
    P1, P2, P3, P4, P5, P6, P7 = [sympy.expand(p) for p in P]
    U2 = P1 + P6; U3 = U2 + P7
    got = [P1 + P2, U2 + P5 + P3, U3 - P4, U3 + P5]
    want = [A11 * B11 + A12 * B21, A11 * B12 + A12 * B22,
            A21 * B11 + A22 * B21, A21 * B12 + A22 * B22]
    for g, w in zip(got, want):
        assert sympy.expand(g - w) == 0
    # and the oracle's step, run on 2x2 blocks of 1x1 integers, agrees
    A = np.array([[3, -1], [2, 5]], dtype=np.int64)
    B = np.array([[-2, 4], [7, 1]], dtype=np.int64)
    assert np.array_equal(O.winograd_step(A, B, O.classical), A @ B)


# --- Winograd recursion: brute force on all small shapes ---------------------

def _shapes_upto(limit, step):
    vals = sorted(set(list(range(1, 9)) + list(range(9, limit + 1, step)) + [limit]))
    return vals


@pytest.mark.parametrize("odd", ["pad", "peel"])
def test_winograd_equals_classical_exactly_small(odd):
    dims = _shapes_upto(64, 7)
    rng = np.random.default_rng(7)
    count = 0
    for m, k, n in itertools.product(dims, dims, dims):
        if rng.random() > 0.08 and max(m, k, n) > 8:
            continue
        A = rng.integers(-5, 6, size=(m, k)).astype(np.int64)
        B = rng.integers(-5, 6, size=(k, n)).astype(np.int64)
        ref = A @ B
        dmax = max(0, int(math.floor(math.log2(max(1, min(m, k, n))))))
        for d in range(0, dmax + 1):
            got = O.winograd(A, B, d, odd)
            assert np.array_equal(got, ref), (m, k, n, d, odd)
            count += 1
    assert count > 200


def test_winograd_all_cube_shapes_to_16():
    for m, k, n in itertools.product(range(1, 17), repeat=3):
        A = I.small_int((m, k), m * 1000 + k * 10 + n).astype(np.int64)
        B = I.small_int((k, n), m + k * 100 + n * 10000).astype(np.int64)
        ref = A @ B
        for d in (1, 2, 4):
            assert np.array_equal(O.winograd(A, B, d, "pad"), ref)
            assert np.array_equal(O.winograd(A, B, d, "peel"), ref)


def test_winograd_float32_integer_data_bit_exact():
    # all partial sums are integers below 2^24, so fp32 Winograd is exact
    A = I.small_int((96, 80), 31, r=3)
    B = I.small_int((80, 72), 32, r=3)
    ref = O.classical(A.astype(np.int64), B.astype(np.int64)).astype(np.float32)
    for d in range(4):
        for odd in ("pad", "peel"):
            assert np.array_equal(O.winograd(A, B, d, odd), ref)


def test_pad_mode_equals_explicit_zero_padding_bitwise():
    A = I.uniform((37, 29), 41)
    B = I.uniform((29, 23), 42)
    got = O.winograd(A, B, 1, "pad")
    Ap = np.zeros((38, 30), np.float32); Ap[:37, :29] = A
    Bp = np.zeros((30, 24), np.float32); Bp[:29, :23] = B
    want = O.winograd_step(Ap, Bp, lambda X, Y: X @ Y)[:37, :23]
    assert np.array_equal(got, want)


def test_block_permutation_commutes_bitwise():
    # permuting rows identically inside each of the 2^d row blocks commutes with
    # every pre- and post-addition, so the fp32 result is permuted exactly
    d, blk = 2, 16
    m = blk * 2 ** d
    A = I.uniform((m, 64), 51)
    B = I.uniform((64, 48), 52)
    perm_blk = np.random.default_rng(3).permutation(blk)
    perm = np.concatenate([b * blk + perm_blk for b in range(2 ** d)])
    C = O.winograd(A, B, d, "pad")
    Cp = O.winograd(A[perm], B, d, "pad")
    assert np.array_equal(Cp, C[perm])


def test_depth0_is_classical():
    A = I.uniform((33, 20), 61)
    B = I.uniform((20, 17), 62)
    assert np.array_equal(O.winograd(A, B, 0), A @ B)


def test_float32_error_within_metric_bound():
    # float accuracy of the fp32 recursion against the fp64 definition
    n = 256
    A, B = I.operands(n, n, n, 71)
    C64 = O.classical(A, B)
    errs = [O.error_metric(O.winograd(A, B, d, "pad"), C64, A, B) for d in range(4)]
    assert all(e < 2e-6 for e in errs), errs
    assert errs[0] < 1e-7


# --- planted mistakes are caught ---------------------------------------------

def _mutated_step(kind):
    def step(A, B, rec):
        A11, A12, A21, A22 = O.quadrants(A)
        B11, B12, B21, B22 = O.quadrants(B)
        S1 = A21 + A22; S2 = S1 - A11; S3 = A11 - A21; S4 = A12 - S2
        T1 = B12 - B11; T2 = B22 - T1; T3 = B22 - B12; T4 = T2 - B21
        if kind == "sign":
            S3 = A21 - A11
        if kind == "transposed":
            T1 = B21 - B11
        P1 = rec(A11, B11); P2 = rec(A12, B21); P3 = rec(S4, B22); P4 = rec(A22, T4)
        P5 = rec(S1, T1); P6 = rec(S2, T2); P7 = rec(S3, T3)
        U1 = P1 + P2; U2 = P1 + P6; U3 = U2 + P7; U4 = U2 + P5
        U5 = U4 + P3 if kind != "dropped" else U4
        U6 = U3 - P4; U7 = U3 + P5
        return np.block([[U1, U5], [U6, U7]])
    return step


@pytest.mark.parametrize("kind", ["sign", "transposed", "dropped"])
def test_planted_mistake_is_caught(kind):
    A = I.small_int((8, 8), 81).astype(np.int64)
    B = I.small_int((8, 8), 82).astype(np.int64)
    got = _mutated_step(kind)(A, B, lambda X, Y: X @ Y)
    assert not np.array_equal(got, A @ B)


# --- residual check and error measure ----------------------------------------

def test_freivalds_zero_and_detects_planted_error():
    A = I.small_int((40, 30), 91).astype(np.float64)
    B = I.small_int((30, 20), 92).astype(np.float64)
    C = A @ B
    for s in range(5):
        x = I.rademacher(20, 93 + s)
        assert np.all(O.freivalds(A, B, C, x) == 0)
    Cbad = C.copy()
    Cbad[17, 3] += 1.0
    for s in range(5):  # a single wrong entry changes r[17] by +-1 for every x
        x = I.rademacher(20, 99 + s)
        r = O.freivalds(A, B, Cbad, x)
        assert abs(r[17]) == 1.0 and np.count_nonzero(r) == 1


def test_error_metric_value():
    A = np.array([[2.0, -1.0]])
    B = np.array([[0.5], [4.0]])
    C64 = A @ B
    C = C64 + 0.01
    assert O.error_metric(C, C64, A, B) == pytest.approx(0.01 / (2.0 * 4.0 * 2))


# --- operand splits ----------------------------------------------------------

def _round_bits_reference(x, keep):
    """Round-to-nearest-even onto `keep` explicit mantissa bits by exact rational
    arithmetic (independent of the bit-twiddling implementation)."""
    if x == 0.0:
        return 0.0
    m, e = math.frexp(abs(x))          # |x| = m * 2^e, 0.5 <= m < 1
    q = fractions.Fraction(abs(x)) / fractions.Fraction(2) ** (e - 1 - keep)
    f = math.floor(q)
    r = q - f
    if r > fractions.Fraction(1, 2) or (r == fractions.Fraction(1, 2) and f % 2 == 1):
        f += 1
    return math.copysign(float(fractions.Fraction(f) * fractions.Fraction(2) ** (e - 1 - keep)), x)


def test_round_mantissa_matches_exact_rounding():
    xs = np.concatenate([I.log_uniform((400,), 5), I.normal((400,), 6),
                         np.array([1 + 2 ** -11, 1 + 3 * 2 ** -11, 1 + 2 ** -12 + 2 ** -13,
                                   -(1 + 2 ** -11), 1.5 + 2 ** -8], dtype=np.float32)])
    for keep in (10, 7):
        got = O.round_mantissa(xs, keep, "rne")
        for x, g in zip(xs.tolist(), got.tolist()):
            assert g == _round_bits_reference(x, keep), (x, keep)
    tr = O.round_mantissa(np.array([1 + 2 ** -11 + 2 ** -12], np.float32), 10, "trunc")
    assert tr[0] == 1.0


def test_bf16_split_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    x = I.normal((1000,), 8)
    hi, lo = O.split_bf16(x)
    t_hi = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    assert np.array_equal(hi, t_hi)
    t_lo = torch.from_numpy((x - t_hi).astype(np.float32)).to(torch.bfloat16).float().numpy()
    assert np.array_equal(lo, t_lo)


def test_tf32_split_reconstructs():
    x = np.concatenate([I.normal((2000,), 9), I.log_uniform((2000,), 10)])
    bounds = {("rne", "rne"): 2.0 ** -21, ("trunc", "trunc"): 2.0 ** -20, ("trunc", "rne"): 2.0 ** -21}
    for (mode, lo_mode), bound in bounds.items():
        hi, lo = O.split_tf32(x, mode, lo_mode)
        assert np.array_equal(O.round_mantissa(hi, 10, "trunc"), hi)
        assert np.array_equal(O.round_mantissa(lo, 10, "trunc"), lo)
        err = np.abs(hi.astype(np.float64) + lo - x) / np.abs(x)
        assert err.max() <= bound, (mode, lo_mode)


def test_split_product_error_bound():
    A = I.uniform((64, 128), 11)
    B = I.uniform((128, 32), 12)
    ref = O.classical(A, B)
    Ah, Al = O.split_tf32(A)
    Bh, Bl = O.split_tf32(B)
    e = np.max(np.abs(O.split_product(Ah, Al, Bh, Bl) - ref))
    assert e <= 128 * 4 * 2.0 ** -22
    # dropping a cross term is caught
    bad = Ah.astype(np.float64) @ Bh + Al.astype(np.float64) @ Bh
    assert np.max(np.abs(bad - ref)) > 10 * e


# --- cost-model network --------------------------------------------------------

def test_mlp_grad_matches_finite_differences():
    rng = np.random.default_rng(5)
    theta = rng.standard_normal(O.MLP_NPARAM) * 0.3
    X = rng.standard_normal((16, 6))
    t = rng.standard_normal(16)
    loss, g = O.mlp_grad(theta, X, t)
    assert loss == pytest.approx(O.mlp_loss(theta, X, t))
    idx = rng.choice(O.MLP_NPARAM, size=60, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (O.mlp_loss(tp, X, t) - O.mlp_loss(tm, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd)


def test_adam_step_matches_scalar_loop_and_decreases_loss():
    rng = np.random.default_rng(6)
    theta = rng.standard_normal(O.MLP_NPARAM) * 0.3
    m = np.zeros_like(theta); v = np.zeros_like(theta)
    X = rng.standard_normal((64, 6)); t = X[:, 0] - 0.5 * X[:, 2]
    loss0, g = O.mlp_grad(theta, X, t)
    th1, m1, v1 = O.adam_step(theta, m, v, g, 1, 1e-3)
    for i in range(0, O.MLP_NPARAM, 97):
        mi = 0.1 * g[i]; vi = 0.001 * g[i] * g[i]
        ref = theta[i] - 1e-3 * (mi / 0.1) / (math.sqrt(vi / 0.001) + 1e-8)
        assert th1[i] == pytest.approx(ref, rel=1e-12, abs=1e-15)
    th, mm, vv = theta, m, v
    for s in range(1, 201):
        _, g = O.mlp_grad(th, X, t)
        th, mm, vv = O.adam_step(th, mm, vv, g, s, 3e-3)
    assert O.mlp_loss(th, X, t) < 0.5 * loss0


# --- sampled rows ----------------------------------------------------------------

def test_classical_rows_equals_full_rows_on_integers():
    A = I.small_int((23, 17), 401, r=7)
    B = I.small_int((17, 29), 402, r=7)
    rows = [0, 22, 5, 5, 11, 1]          # any order, repeats allowed
    full = brute_matmul(A.astype(np.int64).tolist(), B.astype(np.int64).tolist())
    got = O.classical_rows(A, B, rows)
    assert got.dtype == np.float64
    assert got.tolist() == [[float(v) for v in full[r]] for r in rows]
    # a transposed right operand (a plausible indexing mistake) does not pass
    Bsq = I.small_int((17, 17), 403, r=7)
    bad = np.matmul(A[rows].astype(np.float64), Bsq.T.astype(np.float64))
    want = brute_matmul(A.astype(np.int64).tolist(), Bsq.astype(np.int64).tolist())
    assert O.classical_rows(A, Bsq, rows).tolist() == [[float(v) for v in want[r]] for r in rows]
    assert bad.tolist() != [[float(v) for v in want[r]] for r in rows]


# --- IEEE half split ---------------------------------------------------------------

_F = fractions.Fraction


def _round_half_reference(v):
    """Round a rational v to IEEE binary16 with ties to even, by exact rational
    arithmetic: 10 fraction bits for |v| >= 2^-14, the fixed subnormal quantum
    2^-24 below it, +-inf past the largest finite value 65504."""
    if v == 0:
        return 0.0
    a = abs(v)
    e = math.floor(math.log2(a))
    while _F(2) ** e > a:          # exact floor(log2(a)) for a rational
        e -= 1
    while _F(2) ** (e + 1) <= a:
        e += 1
    q = _F(2) ** (max(e, -14) - 10)
    f = math.floor(a / q)
    r = a / q - f
    if r > _F(1, 2) or (r == _F(1, 2) and f % 2 == 1):
        f += 1
    out = f * q
    if out > 65504:
        return math.copysign(math.inf, v)
    return math.copysign(float(out), v)


def _split_half_reference(x, scale):
    xs = _F(float(np.float32(x))) * _F(scale)          # the scale is a power of two: exact
    hi = _round_half_reference(xs)
    lo = _round_half_reference(xs - _F(hi))              # x*s - hi is exact in fp32 and here
    return hi, lo


def _fp16_cases(scale=1.0):
    """Normals, subnormals, ties and the largest finite half, kept within range
    after scaling (the split's precondition)."""
    tiny = np.array([2.0 ** -24, 3 * 2.0 ** -25, 2.0 ** -25, 2.0 ** -26, 2.0 ** -14 - 2.0 ** -24,
                     2.0 ** -14, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -11 + 2.0 ** -20,
                     2047.5, 2048.5, 65504.0, -(1.0 + 2.0 ** -11), 0.0], dtype=np.float32)
    xs = np.concatenate([tiny, -tiny, I.normal((300,), 404), I.log_uniform((300,), 405),
                           I.log_uniform((200,), 406, -7.5, -4.0)]).astype(np.float32)
    return xs[np.abs(xs.astype(np.float64)) * scale <= 65504.0]


@pytest.mark.parametrize("scale", [1.0, 2.0 ** 5, 2.0 ** -3])
def test_split_fp16_matches_exact_rounding(scale):
    xs = _fp16_cases(scale)
    hi, lo = O.split_fp16(xs, scale)
    for x, h, l in zip(xs.tolist(), hi.tolist(), lo.tolist()):
        rh, rl = _split_half_reference(x, scale)
        assert (h, l) == (rh, rl), (x, scale, h, l, rh, rl)


def test_split_fp16_planted_mistakes_are_caught():
    xs = _fp16_cases(2.0 ** 5)
    ref = [_split_half_reference(x, 2.0 ** 5) for x in xs.tolist()]

    def truncating(x, scale):            # round toward zero instead of to nearest
        v = np.asarray(x, np.float32) * np.float32(scale)
        hi = np.array([math.copysign(float(_F(abs(float(t))) // _F(2) ** (max(math.frexp(abs(t))[1] - 1, -14) - 10)
                                           * _F(2) ** (max(math.frexp(abs(t))[1] - 1, -14) - 10)), t)
                       if t != 0 else 0.0 for t in v.tolist()], dtype=np.float32)
        lo = (v - hi).astype(np.float16).astype(np.float32)
        return hi, lo

    def double_scale(x, scale):          # the scale applied twice
        return O.split_fp16(np.asarray(x, np.float32) * np.float32(scale), scale)

    for bad in (truncating, double_scale):
        with np.errstate(over="ignore"):      # the doubled scale overflows half on purpose
            hi, lo = bad(xs, 2.0 ** 5)
        assert [(h, l) for h, l in zip(hi.tolist(), lo.tolist())] != ref


# --- cost-model network forward ------------------------------------------------------

def _hand_network():
    """A network whose output has a closed form: W1 copies the six features into
    hidden units 0..5 (the rest get bias -1), W2 mixes three of them with an
    asymmetric matrix (the rest get bias -1), W3 weighs the results."""
    p = {name: np.zeros(shape) for name, shape in O.MLP_SHAPES}
    for h in range(6):
        p["W1"][h, h] = 1.0
    p["b1"][6:] = -1.0
    p["W2"][0, 1] = 2.0; p["b2"][0] = -1.0               # z2_0 = 2 h1 - 1
    p["W2"][1, 0] = 1.0; p["W2"][1, 2] = -0.5            # z2_1 = h0 - 0.5 h2
    p["W2"][2, 3] = 3.0; p["b2"][2] = 0.25               # z2_2 = 3 h3 + 0.25
    p["b2"][3:] = -1.0
    p["W3"][0, 0], p["W3"][0, 1], p["W3"][0, 2] = 1.0, -2.0, 0.5
    p["W3"][0, 3:] = 0.1
    p["b3"][0] = 0.3
    return np.concatenate([p[name].reshape(-1) for name, _ in O.MLP_SHAPES])


def _hand_output(x):
    r = lambda v: max(v, 0.0)
    h = [r(v) for v in x]
    return r(2 * h[1] - 1) - 2 * r(h[0] - 0.5 * h[2]) + 0.5 * r(3 * h[3] + 0.25) + 0.3


def _hand_inputs():
    return np.array([[0.0] * 6, [1.0, 2.0, 0.5, -1.0, 3.0, -2.0], [-1.0, -2.0, -3.0, 0.5, 0.0, 1.0],
                     [2.0, 0.25, 3.0, 1.0, -1.0, 0.0], [0.7, 0.6, -0.4, -0.1, 5.0, 5.0]])


def test_mlp_forward_closed_form():
    theta = _hand_network()
    X = _hand_inputs()
    y, _ = O.mlp_forward(theta, X)
    assert y.tolist() == pytest.approx([_hand_output(x) for x in X.tolist()], abs=1e-15)


def test_mlp_forward_planted_mistakes_are_caught():
    theta = _hand_network()
    X = _hand_inputs()
    want = np.array([_hand_output(x) for x in X.tolist()])
    p = O.mlp_unpack(theta)

    def no_second_relu(X):
        h1 = np.maximum(X @ p["W1"].T + p["b1"], 0.0)
        h2 = h1 @ p["W2"].T + p["b2"]
        return (h2 @ p["W3"].T + p["b3"])[:, 0]

    def w2_transposed(X):
        h1 = np.maximum(X @ p["W1"].T + p["b1"], 0.0)
        h2 = np.maximum(h1 @ p["W2"] + p["b2"], 0.0)
        return (h2 @ p["W3"].T + p["b3"])[:, 0]

    for bad in (no_second_relu, w2_transposed):
        assert np.max(np.abs(bad(X) - want)) > 0.1


def test_mlp_loss_closed_form():
    theta = _hand_network()
    X = _hand_inputs()
    t = np.array([0.5, -1.0, 2.0, 0.0, 1.25])
    y = np.array([_hand_output(x) for x in X.tolist()])
    assert O.mlp_loss(theta, X, t) == pytest.approx(0.5 * float(np.mean((y - t) ** 2)), abs=1e-14)
