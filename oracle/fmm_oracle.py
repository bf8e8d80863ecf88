"""CPU oracle of the fast matrix multiply.  TEST INFRASTRUCTURE ONLY.

This module is the plain, slow, obviously correct statement of what the GPU
library computes.  It shares no code with the CUDA path and imports nothing
from it.  Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` may import it; the product path
never does.

What it states, each with the passage of D'Alberto, "A Heterogeneous
Accelerated Matrix Multiplication: OpenCL + APU + GPU + Fast Matrix Multiply"
(arXiv 1205.2927) it follows:

* ``classical``/``gemm``: the definition c_ij = sum_k a_ik b_kj (Sec. 3.3, the
  row-by-column formula) with BLAS semantics C <- alpha*A*B + beta*C (Sec. 3.2,
  the SGEMM leaf; beta = 0 never reads C, alpha = 0 never reads A or B).
* ``quadrants``: the four-quadrant division of any m x n matrix (Eq. 1): the
  top-left block is ceil(m/2) x ceil(n/2), the bottom-right floor(m/2) x floor(n/2).
* ``rmul``: the balanced classical recursion C = AB / C += AB of Table 1.
* ``winograd``: the fast recursive algorithm based on Winograd's variant of
  Strassen's method, which the paper names as the next step (Sec. 4.3, last
  paragraph; Winograd's MM on the CPU in Sec. 4.1).  The paper does not print
  the formulas; the textbook variant (7 products, 8 pre-additions, 7
  post-additions) is used, in the S/T/P/U notation, with odd sizes handled by
  the zero padding implied by Eq. 1 ("pad") or by dynamic peeling ("peel").
* ``freivalds``/``error_metric``: the residual check and the max-norm error
  measure that results are held to (the paper itself reports no error analysis,
  Sec. 1, last paragraph).
* ``split_*``/``split_product``: the hi/lo operand splits of the split-precision
  leaves (three products, fp32 accumulation).
* ``mlp_*``: the 6-64-64-1 cost model, forward, loss, backward and Adam step,
  in float64.

Parity status: every function here is pinned by the CPU tests in
``tests/test_oracle_pins.py`` (brute force, closed forms, symbolic identity,
invariants); none is "parity unpinned".
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Classical product (the definition) and BLAS-style GEMM semantics
# ---------------------------------------------------------------------------


def classical(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """C = A B by the definition c_ij = sum_k a_ik b_kj (Sec. 3.3).

    float inputs are promoted to float64; integer inputs stay int64 (exact as
    long as no partial sum overflows).  The library matmul is used as the step
    that evaluates the sums.
    """
    if np.issubdtype(A.dtype, np.integer) and np.issubdtype(B.dtype, np.integer):
        return np.matmul(A.astype(np.int64), B.astype(np.int64))
    return np.matmul(A.astype(np.float64), B.astype(np.float64))


def classical_rows(A: np.ndarray, B: np.ndarray, rows) -> np.ndarray:
    """Rows `rows` of A B in float64 (the sampled form used at large sizes)."""
    rows = np.asarray(rows)
    return np.matmul(A[rows].astype(np.float64), B.astype(np.float64))


def gemm(alpha, A, B, beta, C=None):
    """C <- alpha * A B + beta * C in float64 (SGEMM semantics, Sec. 3.2).

    beta == 0: C is not read (so NaN in C does not propagate).
    alpha == 0 or an empty inner dimension: A and B are not read, C <- beta*C.
    """
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    if beta == 0 or C is None:
        out = np.zeros((m, n), dtype=np.float64)
    else:
        out = float(beta) * C.astype(np.float64)
    if alpha != 0 and k > 0 and m > 0 and n > 0:
        out = out + float(alpha) * classical(A, B)
    return out


# ---------------------------------------------------------------------------
# Eq. 1: quadrant division
# ---------------------------------------------------------------------------


def quadrants(D: np.ndarray):
    """(D0, D1, D2, D3) of Eq. 1 in row-major order 0 = top-left, 1 = top-right,
    2 = bottom-left, 3 = bottom-right.  D0 is ceil(m/2) x ceil(n/2) and D3 is
    floor(m/2) x floor(n/2)."""
    m, n = D.shape
    mh, nh = (m + 1) // 2, (n + 1) // 2
    return D[:mh, :nh], D[:mh, nh:], D[mh:, :nh], D[mh:, nh:]


def _zero_pad(X: np.ndarray, rows: int, cols: int) -> np.ndarray:
    if X.shape == (rows, cols):
        return X
    out = np.zeros((rows, cols), dtype=X.dtype)
    out[: X.shape[0], : X.shape[1]] = X
    return out


# ---------------------------------------------------------------------------
# Table 1: balanced classical recursion RMUL (C = AB and C += AB)
# ---------------------------------------------------------------------------


def rmul(A: np.ndarray, B: np.ndarray, depth: int, leaf=None) -> np.ndarray:
    """Classical 8-product quadrant recursion of Table 1 (left column: C = AB;
    the += products follow the right column).  Shape-oblivious: quadrants per
    Eq. 1; the inner split of A's columns matches the split of B's rows."""
    leaf = leaf or (lambda X, Y: np.matmul(X, Y))
    m, k = A.shape
    n = B.shape[1]
    if depth == 0 or min(m, k, n) < 2:
        return leaf(A, B)
    A0, A1, A2, A3 = quadrants(A)
    B0, B1, B2, B3 = quadrants(B)
    C = np.empty((m, n), dtype=np.result_type(A.dtype, B.dtype))
    mh, nh = (m + 1) // 2, (n + 1) // 2
    # C0 = A0 B0; C1 = A0 B1; C2 = A2 B0; C3 = A2 B1
    C[:mh, :nh] = rmul(A0, B0, depth - 1, leaf)
    C[:mh, nh:] = rmul(A0, B1, depth - 1, leaf)
    C[mh:, :nh] = rmul(A2, B0, depth - 1, leaf)
    C[mh:, nh:] = rmul(A2, B1, depth - 1, leaf)
    # C0 += A1 B2; C1 += A1 B3; C2 += A3 B2; C3 += A3 B3
    C[:mh, :nh] += rmul(A1, B2, depth - 1, leaf)
    C[:mh, nh:] += rmul(A1, B3, depth - 1, leaf)
    C[mh:, :nh] += rmul(A3, B2, depth - 1, leaf)
    C[mh:, nh:] += rmul(A3, B3, depth - 1, leaf)
    return C


# ---------------------------------------------------------------------------
# Winograd's variant of Strassen's recursion
# ---------------------------------------------------------------------------


def _leaf_default(X, Y):
    return np.matmul(X, Y)


def winograd_step(A, B, rec):
    """One level of Winograd's variant on operands whose dimensions are even.

    Pre-additions (8):  S1 = A21 + A22, S2 = S1 - A11, S3 = A11 - A21, S4 = A12 - S2,
                        T1 = B12 - B11, T2 = B22 - T1, T3 = B22 - B12, T4 = T2 - B21.
    Products (7):       P1 = A11 B11, P2 = A12 B21, P3 = S4 B22, P4 = A22 T4,
                        P5 = S1 T1, P6 = S2 T2, P7 = S3 T3.
    Post-additions (7): U1 = P1 + P2, U2 = P1 + P6, U3 = U2 + P7, U4 = U2 + P5,
                        U5 = U4 + P3, U6 = U3 - P4, U7 = U3 + P5;
                        C11 = U1, C12 = U5, C21 = U6, C22 = U7.
    """
    A11, A12, A21, A22 = quadrants(A)
    B11, B12, B21, B22 = quadrants(B)
    S1 = A21 + A22
    S2 = S1 - A11
    S3 = A11 - A21
    S4 = A12 - S2
    T1 = B12 - B11
    T2 = B22 - T1
    T3 = B22 - B12
    T4 = T2 - B21
    P1 = rec(A11, B11)
    P2 = rec(A12, B21)
    P3 = rec(S4, B22)
    P4 = rec(A22, T4)
    P5 = rec(S1, T1)
    P6 = rec(S2, T2)
    P7 = rec(S3, T3)
    U1 = P1 + P2
    U2 = P1 + P6
    U3 = U2 + P7
    U4 = U2 + P5
    U5 = U4 + P3
    U6 = U3 - P4
    U7 = U3 + P5
    top = np.concatenate([U1, U5], axis=1)
    bottom = np.concatenate([U6, U7], axis=1)
    return np.concatenate([top, bottom], axis=0)


def winograd(A: np.ndarray, B: np.ndarray, depth: int, odd: str = "pad",
             leaf=None, cutoff: int = 1) -> np.ndarray:
    """C = A B by `depth` levels of Winograd's recursion over classical leaves.

    The arithmetic happens in the dtype of the operands (int64 -> exact,
    float32 -> every addition rounded to fp32, float64).  Recursion stops at
    depth 0 or when a dimension is below 2*cutoff.

    odd == "pad":  quadrants per Eq. 1; the bottom/right quadrants are
                   completed with an implicit zero row/column to the top-left
                   size, and the padding is dropped from the result.
    odd == "peel": the even core (m', k', n' rounded down to even) goes through
                   the Winograd step; then (dynamic peeling)
                   k odd:  C[:m', :n'] += a[:m', k-1] b[k-1, :n']   (rank 1)
                   m odd:  C[m-1, :]   = a[m-1, :] B                 (row)
                   n odd:  C[:m', n-1] = A[:m', :] b[:, n-1]         (column)
    """
    leaf = leaf or _leaf_default
    m, k = A.shape
    k2, n = B.shape
    assert k == k2, "inner dimensions differ"
    if depth == 0 or min(m, k, n) < 2 * max(1, cutoff):
        return leaf(A, B)

    def rec(X, Y):
        return winograd(X, Y, depth - 1, odd, leaf, cutoff)

    if odd == "pad":
        mh, kh, nh = (m + 1) // 2, (k + 1) // 2, (n + 1) // 2
        Ap = _zero_pad(A, 2 * mh, 2 * kh)
        Bp = _zero_pad(B, 2 * kh, 2 * nh)
        return winograd_step(Ap, Bp, rec)[:m, :n]
    if odd == "peel":
        m2, k2, n2 = m - m % 2, k - k % 2, n - n % 2
        C = np.empty((m, n), dtype=np.result_type(A.dtype, B.dtype))
        C[:m2, :n2] = winograd_step(A[:m2, :k2], B[:k2, :n2], rec)
        if k % 2:
            C[:m2, :n2] += np.outer(A[:m2, k - 1], B[k - 1, :n2])
        if m % 2:
            C[m - 1, :] = A[m - 1, :] @ B
        if n % 2:
            C[:m2, n - 1] = A[:m2, :] @ B[:, n - 1]
        return C
    raise ValueError(f"unknown odd-size mode {odd!r}")


# ---------------------------------------------------------------------------
# Error measure and residual check
# ---------------------------------------------------------------------------


def error_metric(C, C64, A, B) -> float:
    """||C - C64||_max / (||A||_max * ||B||_max * k), k the inner dimension."""
    k = A.shape[1]
    den = float(np.max(np.abs(A))) * float(np.max(np.abs(B))) * max(k, 1)
    if den == 0.0:
        return float(np.max(np.abs(C.astype(np.float64) - C64))) if C.size else 0.0
    return float(np.max(np.abs(C.astype(np.float64) - C64))) / den


def freivalds(A, B, C, x) -> np.ndarray:
    """Residual r = C x - A (B x) in float64 for a probe vector x (+-1 entries)."""
    x = x.astype(np.float64)
    return C.astype(np.float64) @ x - A.astype(np.float64) @ (B.astype(np.float64) @ x)


# ---------------------------------------------------------------------------
# Split-precision operand splits (hi + lo, three products, fp32 accumulation)
# ---------------------------------------------------------------------------


def _f32_bits(x):
    return np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)


def round_mantissa(x: np.ndarray, keep_bits: int, mode: str = "rne") -> np.ndarray:
    """Round float32 values to `keep_bits` explicit mantissa bits (of 23).

    mode "trunc": clear the dropped bits (round toward zero).
    mode "rne":   round to nearest, ties to even, on the bit pattern.
    Finite inputs only.  TF32 keeps 10 bits, bfloat16 keeps 7.
    """
    drop = 23 - keep_bits
    u = _f32_bits(x).astype(np.uint64)
    mask = np.uint64((0xFFFFFFFF >> drop) << drop)
    if mode == "trunc":
        r = u & mask
    elif mode == "rne":
        half = np.uint64(1 << (drop - 1)) - np.uint64(1)
        lsb = (u >> np.uint64(drop)) & np.uint64(1)
        r = (u + half + lsb) & mask
    else:
        raise ValueError(mode)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)


def split_tf32(x: np.ndarray, mode: str = "rne", lo_mode: str | None = None):
    """x = hi + lo (+ residual): hi = tf32(x) rounded by `mode`, lo = tf32(x - hi)
    rounded by `lo_mode` (default: `mode`); x - hi is exact in fp32.

    ("trunc", "rne") is the split whose hi is what a tensor core that truncates
    fp32 operands to TF32 reads from the raw value."""
    x = np.asarray(x, dtype=np.float32)
    hi = round_mantissa(x, 10, mode)
    lo = round_mantissa((x - hi).astype(np.float32), 10, lo_mode or mode)
    return hi, lo


def split_bf16(x: np.ndarray):
    """x = hi + lo (+ residual) with hi, lo bfloat16 values (round to nearest even)."""
    x = np.asarray(x, dtype=np.float32)
    hi = round_mantissa(x, 7, "rne")
    lo = round_mantissa((x - hi).astype(np.float32), 7, "rne")
    return hi, lo


def split_fp16(x: np.ndarray, scale: float):
    """x*scale = hi + lo (+ residual) with hi, lo IEEE half values (round to nearest
    even, subnormals kept); `scale` is a power of two chosen to keep x*scale in range."""
    xs = np.asarray(x, dtype=np.float32) * np.float32(scale)
    hi = xs.astype(np.float16)
    lo = (xs - hi.astype(np.float32)).astype(np.float16)
    return hi.astype(np.float32), lo.astype(np.float32)


def split_product(Ahi, Alo, Bhi, Blo) -> np.ndarray:
    """Ahi Bhi + Ahi Blo + Alo Bhi in float64: the three-product form of a split
    leaf, with the (lo, lo) term dropped and exact (float64) accumulation."""
    f = lambda X: X.astype(np.float64)
    return f(Ahi) @ f(Bhi) + f(Ahi) @ f(Blo) + f(Alo) @ f(Bhi)


# ---------------------------------------------------------------------------
# Cost-model network: 6 -> 64 -> 64 -> 1, ReLU, float64
# ---------------------------------------------------------------------------

MLP_IN, MLP_HID = 6, 64
MLP_SHAPES = [("W1", (MLP_HID, MLP_IN)), ("b1", (MLP_HID,)),
              ("W2", (MLP_HID, MLP_HID)), ("b2", (MLP_HID,)),
              ("W3", (1, MLP_HID)), ("b3", (1,))]
MLP_NPARAM = sum(int(np.prod(s)) for _, s in MLP_SHAPES)


def mlp_unpack(theta: np.ndarray) -> dict:
    """Parameter dict from the flat vector (W1, b1, W2, b2, W3, b3 in that order,
    weights row-major [out, in])."""
    out, off = {}, 0
    for name, shp in MLP_SHAPES:
        size = int(np.prod(shp))
        out[name] = theta[off:off + size].reshape(shp).astype(np.float64)
        off += size
    return out


def mlp_forward(theta, X):
    """y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for each row x of X; returns
    (y, cache)."""
    p = mlp_unpack(np.asarray(theta, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = (h2 @ p["W3"].T + p["b3"])[:, 0]
    return y, (X, z1, h1, z2, h2, p)


def mlp_loss(theta, X, t) -> float:
    """0.5 * mean((y - t)^2)."""
    y, _ = mlp_forward(theta, X)
    return 0.5 * float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def mlp_grad(theta, X, t):
    """(loss, d loss / d theta) by reverse-mode differentiation of mlp_loss."""
    y, (X, z1, h1, z2, h2, p) = mlp_forward(theta, X)
    t = np.asarray(t, dtype=np.float64)
    B = X.shape[0]
    dy = (y - t) / B
    loss = 0.5 * float(np.mean((y - t) ** 2))
    g = {}
    g["W3"] = dy[None, :] @ h2
    g["b3"] = np.array([dy.sum()])
    dh2 = dy[:, None] @ p["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    flat = np.concatenate([g[name].reshape(-1) for name, _ in MLP_SHAPES])
    return loss, flat


def adam_step(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) with bias correction; `step` counts from 1."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v
