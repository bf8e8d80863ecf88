"""Seeded synthetic operand generators shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the fast matrix multiply: it only draws the
operand matrices.  Both the CUDA path and the CPU oracle receive the very same
host arrays from here, so neither side ever produces the other's inputs.

The paper measures on synthetic square single-precision matrices only (Sec. 4,
GFLOPS = 2N^3/t); the distributions below are the ones the workloads name:
uniform[-1, 1], standard normal, log-uniform magnitude sign * 10^U(-3, 3), and
small integers (every partial sum then stays exact in fp32, which is what the
bit-exact tests rely on).

Seeds follow one convention: seed = 20260000 + 100 * workload + case.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20260000


def seed_for(workload: int, case: int = 0) -> int:
    """Seed of case `case` of workload `workload` (1-based workload numbers)."""
    return SEED_BASE + 100 * int(workload) + int(case)


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """i.i.d. uniform[lo, hi) float32 matrix (C-contiguous, row-major)."""
    return _rng(seed).uniform(lo, hi, size=shape).astype(np.float32)


def normal(shape, seed: int) -> np.ndarray:
    """i.i.d. N(0, 1) float32 matrix."""
    return _rng(seed).standard_normal(size=shape, dtype=np.float64).astype(np.float32)


def log_uniform(shape, seed: int, lo_exp: float = -3.0, hi_exp: float = 3.0) -> np.ndarray:
    """sign * 10^U(lo_exp, hi_exp): magnitudes spread over six decades, random sign."""
    g = _rng(seed)
    mag = 10.0 ** g.uniform(lo_exp, hi_exp, size=shape)
    sign = np.where(g.integers(0, 2, size=shape) == 0, -1.0, 1.0)
    return (sign * mag).astype(np.float32)


def small_int(shape, seed: int, r: int = 4) -> np.ndarray:
    """Integers uniform in [-r, r] stored as float32 (exact)."""
    return _rng(seed).integers(-r, r + 1, size=shape).astype(np.float32)


def rademacher(n: int, seed: int) -> np.ndarray:
    """Random +-1 float32 vector (the probe vector of a Freivalds check)."""
    return np.where(_rng(seed).integers(0, 2, size=n) == 0, -1.0, 1.0).astype(np.float32)


DISTRIBUTIONS = {
    "uniform": uniform,
    "normal": normal,
    "loguniform": log_uniform,
    "smallint": small_int,
}


def operands(m: int, k: int, n: int, seed: int, dist: str = "uniform"):
    """A (m x k) and B (k x n) drawn from `dist`, A from `seed`, B from `seed + 50`."""
    f = DISTRIBUTIONS[dist]
    return f((m, k), seed), f((k, n), seed + 50)


def batched_shapes(count: int, seed: int, lo: int = 128, hi: int = 4096, multiple: int = 4):
    """`count` (M, K, N) triples, each dimension log-uniform in [lo, hi] and rounded to
    a multiple of `multiple` (kept within [lo, hi])."""
    g = _rng(seed)
    raw = np.exp(g.uniform(np.log(lo), np.log(hi), size=(count, 3)))
    dims = np.clip(np.round(raw / multiple) * multiple, lo, hi).astype(np.int64)
    return [tuple(int(x) for x in row) for row in dims]
