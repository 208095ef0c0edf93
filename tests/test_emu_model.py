"""Exact integer model of the FP64-accurate products from bf16 slices (the
error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012, with eight 7-bit
slices), on the CPU: it checks the design constants the tensor-core kernels
rely on, independently of them.

  * A value x below the line scale 2^E is written as X = |x| 2^(56-E) (exact
    when x is within four binades of the scale, else rounded) with balanced
    base-2^7 digits d_1 in [0, 128] and d_2..d_8 in [-64, 63]; each slice
    d_p 2^(-7(p-1)) is exact in bf16 (8 significant bits).
  * For K <= 512 (the kernels' exact accumulation) the level sums of the
    slice products with p + q - 2 <= 4 stay below 2^24, i.e. exact in an
    FP32 accumulator.
  * Keeping the 36 products with p + q <= 9 (levels 5..7 in one FP32
    accumulator) gives |C - AB| <= (9K + 64) 2^-56 2^(E_m + F_n) per entry.
The model rounds the shared FP32 accumulator once at the end, whereas the
tensor cores round at every accumulation step; that case is measured by the
GPU tests (against long-double products), this model pins the rest of the
arithmetic exactly (Python integers and fractions).
"""
from __future__ import annotations

from fractions import Fraction
import math

import numpy as np
import pytest

H = 64 * sum(1 << (56 - 7 * p) for p in range(2, 9))


def _scale_exp(v: np.ndarray) -> int:
    """E with max |v| < 2^E: one more than the largest entry's exponent."""
    m = float(np.abs(v).max())
    return 0 if m == 0.0 else math.frexp(m)[1]


def _digits(x: float, E: int) -> list[int]:
    """Balanced digits of |x| 2^(56-E), the sign of x on every digit."""
    if x == 0.0:
        return [0] * 8
    mant, ex = math.frexp(abs(x))            # |x| = mant 2^ex, mant in [0.5, 1)
    M = int(mant * (1 << 53))                 # 53-bit integer significand
    sh = (ex - 53) - E + 56                   # |x| 2^(56-E) = M 2^sh
    if sh >= 0:
        X = M << sh
    elif sh > -54:
        X = (M + (1 << (-sh - 1))) >> -sh     # nearest, ties up
    else:
        X = 0
    assert X < (1 << 56)
    Y = X + H
    d = [Y >> 49] + [((Y >> (56 - 7 * p)) & 127) - 64 for p in range(2, 9)]
    assert sum(dp << (56 - 7 * p) for p, dp in enumerate(d, 1)) == X
    return [-v for v in d] if x < 0 else d


def _emulated(A: np.ndarray, B: np.ndarray):
    """C = A B the way the kernels form it: exact level sums, levels 5..7 in
    one FP32 accumulator, combined in units of 2^-35 of the level-0 unit."""
    M, K = A.shape
    N = B.shape[1]
    Es = [_scale_exp(A[i]) for i in range(M)]
    Fs = [_scale_exp(B[:, j]) for j in range(N)]
    da = [[_digits(A[i, k], Es[i]) for k in range(K)] for i in range(M)]
    db = [[_digits(B[k, j], Fs[j]) for k in range(K)] for j in range(N)]
    C = np.zeros((M, N))
    levels_max = [0] * 8
    for i in range(M):
        for j in range(N):
            L = [0] * 8
            for k in range(K):
                a, b = da[i][k], db[j][k]
                for p in range(1, 9):
                    for q in range(1, 10 - p):
                        L[p + q - 2] += a[p - 1] * b[q - 1]
            for l in range(8):
                levels_max[l] = max(levels_max[l], abs(L[l]))
            # the shared accumulator: FP32 sum of levels 5..7 (weights 2^-35 .. 2^-49),
            # here evaluated exactly and rounded once to FP32, then to units of 2^-35
            shared = np.float32(sum(Fraction(L[l], 1 << (7 * l)) for l in range(5, 8)))
            S = sum(L[l] << (7 * (5 - l)) for l in range(5)) + int(round(float(shared) * (1 << 35)))
            C[i, j] = math.ldexp(S, Es[i] + Fs[j] - 49)
    return C, Es, Fs, levels_max


def _exact(A, B, i, j):
    return sum(Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(A.shape[1]))


def test_digits_reconstruct_and_stay_in_range():
    r = np.random.default_rng(11)
    for x in list(r.standard_normal(300) * 10.0 ** r.uniform(-30, 30, 300)) + [0.0, -1.0, 2.0 ** -1074]:
        E = math.frexp(abs(x))[1] + int(r.integers(0, 3)) if x != 0.0 else 0
        d = _digits(x, E)
        assert 0 <= abs(d[0]) <= 128 and all(abs(v) <= 64 for v in d[1:])
        # each slice d_p is an integer of at most 8 significant bits: exact in bf16
        assert all(abs(v) < 256 for v in d)


def test_level_sums_stay_exact_in_fp32_for_k_512():
    """Worst-case digits (|d_1| = 128, |d_p| = 64): the level sums of
    levels 0..4 over K = 512 terms (the kernels' exact accumulation) stay
    below 2^24."""
    K = 512
    mx = [128] + [64] * 7
    for l in range(5):
        worst = K * sum(mx[p - 1] * mx[q - 1] for p in range(1, 9) for q in range(1, 10 - p) if p + q - 2 == l)
        assert worst < (1 << 24), (l, worst)
    # the largest K that keeps every level exact: 585 (level 4 dominates), so
    # the long products drain their accumulators every 512 values
    per_term = max(sum(mx[p - 1] * mx[q - 1] for p in range(1, 9) for q in range(1, 10 - p) if p + q - 2 == l)
                   for l in range(5))
    assert per_term == 2 * 128 * 64 + 3 * 64 * 64
    assert ((1 << 24) - 1) // per_term == 585


@pytest.mark.parametrize("K,seed,graded", [(16, 1, False), (64, 2, True), (256, 3, False), (256, 4, True)])
def test_error_bound(K, seed, graded):
    r = np.random.default_rng(seed)
    M, N = 3, 3
    A = r.standard_normal((M, K))
    B = r.standard_normal((K, N))
    if graded:   # entries of each line spread over many binades
        A *= 2.0 ** r.integers(-40, 1, size=(M, K))
        B *= 2.0 ** r.integers(-40, 1, size=(K, N))
    C, Es, Fs, lv = _emulated(A, B)
    assert max(lv[:5]) < (1 << 24)
    for i in range(M):
        for j in range(N):
            err = abs(Fraction(C[i, j]) - _exact(A, B, i, j))
            bound = Fraction(9 * K + 64) * Fraction(2) ** (Es[i] + Fs[j] - 56)
            assert err <= bound, (i, j, float(err / bound))


@pytest.mark.parametrize("K", [128, 512])
def test_adversarial_lines_of_equal_magnitude(K):
    """Every entry just below the scale (the largest digits in every slot):
    still within the bound, and over one exact accumulation of K = 512 the
    level sums stay exact."""
    v = np.full(K, 1.0 - 2.0 ** -53)
    A = (v * np.where(np.arange(K) % 2 == 0, 1.0, -1.0))[None, :]
    B = v[:, None]
    C, Es, Fs, lv = _emulated(A, B)
    err = abs(Fraction(C[0, 0]) - _exact(A, B, 0, 0))
    assert err <= Fraction(9 * K + 64) * Fraction(2) ** (Es[0] + Fs[0] - 56)
    assert max(lv[:5]) < (1 << 24)
