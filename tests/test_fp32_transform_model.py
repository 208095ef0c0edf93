"""CPU model of a pivot transform accumulated in FP32 (the low-precision
sweeps of the mixed form).

The pivot solve chooses its rotations in FP64 (one inner sweep of the
round-robin order over k indices, k - 1 rounds); the transform V that feeds
the split-precision products is accumulated in FP32: s and tau rounded to
FP32 once per rotation, each entry pair (x, y) of a row updated in
Rutishauser's form by two FP32 fused multiply-adds
    x' = fl(x - s fl(y + tau x)),  y' = fl(y + s fl(x - tau y)).
The parity tests bound the result entry-wise by |V32 - V| <= 6 k u32
(a round's update of a pair of norm <= 1 errs by at most 6 u32, and later
rotations carry it without growth).  Here the rotations come from a plain
FP64 sweep in numpy, the FP32 fma is modelled exactly (an FP32 product is
exact in FP64 and the FP64 sum is rounded once to FP32; double rounding
occurs only for sums that need more than 53 bits, far below the bound), and
the bound is checked against the same sweep's FP64 transform.
"""
from __future__ import annotations

import numpy as np
import pytest

U32 = 2.0 ** -24


def round_robin_pairs(k: int, rd: int):
    nr = k - 1
    def at(pos):
        return 0 if pos == 0 else 1 + (pos - 1 + rd) % nr
    out = []
    for e in range(k // 2):
        a, b = at(e), at(k - 1 - e)
        out.append((min(a, b), max(a, b)))
    return out


def textbook(app, aqq, apq):
    zeta = (aqq - app) / (2.0 * apq)
    t = (1.0 if zeta >= 0 else -1.0) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
    c = 1.0 / np.sqrt(1.0 + t * t)
    s = t * c
    return c, s, s / (1.0 + c)


def fma32(a, b, c):
    """fl32(a * b + c) for FP32 a, b, c (arrays): the product is exact in FP64."""
    return (np.float64(a) * np.asarray(b, dtype=np.float64) + np.asarray(c, dtype=np.float64)).astype(np.float32)


def one_sweep(A: np.ndarray):
    """One round-robin sweep of scalar Jacobi on the symmetric A (FP64),
    returning V accumulated in FP64 and in FP32 (the kernel's form)."""
    k = A.shape[0]
    A = A.copy()
    V64 = np.eye(k)
    V32 = np.eye(k, dtype=np.float32)
    for rd in range(k - 1):
        rots = []
        for p, q in round_robin_pairs(k, rd):
            if A[p, q] != 0.0:
                rots.append((p, q) + textbook(A[p, p], A[q, q], A[p, q]))
        for p, q, c, s, tau in rots:   # disjoint pairs: the order within a round is immaterial
            ap, aq = A[:, p].copy(), A[:, q].copy()          # A <- A J
            A[:, p], A[:, q] = c * ap - s * aq, s * ap + c * aq
            ap, aq = A[p, :].copy(), A[q, :].copy()          # A <- J^T A
            A[p, :], A[q, :] = c * ap - s * aq, s * ap + c * aq
            A[p, q] = A[q, p] = 0.0
            xp, xq = V64[:, p].copy(), V64[:, q].copy()
            V64[:, p] = xp - s * (xq + tau * xp)
            V64[:, q] = xq + s * (xp - tau * xq)
            s32, t32 = np.float32(s), np.float32(tau)
            x, y = V32[:, p].copy(), V32[:, q].copy()
            V32[:, p] = fma32(-s32, fma32(t32, x, y), x)
            V32[:, q] = fma32(s32, fma32(-t32, y, x), y)
    return V64, V32


@pytest.mark.parametrize("k,seed", [(32, 1), (64, 2), (128, 3)])
def test_fp32_accumulated_transform_within_the_bound(k, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((k, k))
    A = (M + M.T) / 2 + np.diag(np.linspace(1.0, 3.0, k))
    V64, V32 = one_sweep(A)
    err = np.abs(V32.astype(np.float64) - V64).max()
    # the bound the parity tests use, and a floor so that the check is not vacuous
    assert err <= 6 * k * U32, err / (k * U32)
    assert err >= U32 / 4
    # V stays orthogonal to FP32 accuracy
    assert np.abs(V32.astype(np.float64).T @ V32 - np.eye(k)).max() <= 12 * k * U32
