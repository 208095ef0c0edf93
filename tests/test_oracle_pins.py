"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names the passage of the paper (or the mathematical fact) it pins.
A plausible mistake in the oracle -- a dropped term, a wrong sign, a
transposed V, a wrong index in the ordering -- fails at least one of them:

* closed form of the 2x2 symmetric eigenproblem; off^2 drops by exactly
  2 a_pq^2 per rotation (Sec. 1);
* diagonal input -> no rotation, Q = I bit-exactly;
* matrices built with a known spectrum; trace / Frobenius invariance;
  the block form of the off^2 identity over one parallel step (Algorithm 2);
* exact characteristic-polynomial roots (rational arithmetic + Sturm
  bisection) for n <= 4;
* LAPACK (numpy) as an independent accuracy witness; mpmath in 40 digits for
  the relative accuracy on a graded DHD matrix;
* the paper's printed ordering list, label matrix and transformation
  patterns (Sec. 3, eqs. (disjoint), (group_one_transformation),
  (alt_transformations), (parallel_list); Algorithm 3);
* Gram block as a sum over row tiles (Sec. 6, eq. after (SVD_subproblem));
* tight clusters: the invariant (singular) subspaces' projectors against the
  constructed ones within the Davis-Kahan / Wedin perturbation bound.
"""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np
import pytest

import jacobi_inputs as gen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53


def _offsq(A):
    A = np.asarray(A)
    return float(np.sum(A * A) - np.sum(np.diag(A) ** 2))


# ------------------------------------------------------------------ 2x2 / one rotation
def test_rotation_matches_2x2_closed_form():
    r = np.random.default_rng(11)
    for _ in range(2000):
        a, b, c = r.standard_normal(3) * 10.0 ** r.uniform(-3, 3, 3)
        cs, sn, t = oracle.rotation(a, c, b)
        J = np.array([[cs, sn], [-sn, cs]])
        M = np.array([[a, b], [b, c]])
        D = J.T @ M @ J
        scale = np.abs(M).max()
        assert abs(D[0, 1]) <= 8 * U * scale
        # closed-form eigenvalues (a+c)/2 -+ sqrt(((a-c)/2)^2 + b^2)
        mid, rad = 0.5 * (a + c), np.hypot(0.5 * (a - c), b)
        lo, hi = mid - rad, mid + rad
        got = sorted([a - t * b, c + t * b])
        assert abs(got[0] - lo) <= 8 * U * scale and abs(got[1] - hi) <= 8 * U * scale
        assert abs(cs * cs + sn * sn - 1.0) <= 4 * U
        assert abs(t) <= 1.0  # |angle| <= pi/4 (inner rotation)


def test_rotation_large_zeta_branch():
    cs, sn, t = oracle.rotation(0.0, 1e300, 1e-10)
    assert cs == 1.0 and abs(t - 0.5 / (1e300 / 2e-10)) <= 1e-16 * abs(t)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_single_rotation_drops_off2_by_2apq2(seed):
    r = np.random.default_rng(seed)
    n = 9
    A = gen.sym_gaussian(n, 100 + seed)
    p, q = sorted(r.choice(n, 2, replace=False))
    apq = A[p, q]
    A2, Q2, applied = oracle.rotate(A, np.eye(n), p, q)
    assert applied and A2[p, q] == 0.0 and A2[q, p] == 0.0
    assert abs(_offsq(A2) - (_offsq(A) - 2 * apq * apq)) <= 1e-13 * _offsq(A)
    # similarity: Q A2 Q^T == A, Q orthogonal
    assert np.abs(Q2 @ A2 @ Q2.T - A).max() <= 1e-14 * np.abs(A).max() * n
    assert np.abs(Q2.T @ Q2 - np.eye(n)).max() <= 4 * U * n
    assert np.allclose(np.linalg.eigvalsh(A2), np.linalg.eigvalsh(A), atol=1e-13, rtol=0)


def test_zero_entry_is_not_rotated():
    A = np.diag([1.0, 2.0, 3.0])
    A2, Q2, applied = oracle.rotate(A, np.eye(3), 0, 2)
    assert not applied and np.array_equal(A2, A) and np.array_equal(Q2, np.eye(3))


# ------------------------------------------------------------------ stop statistics
def test_off_norm_exact_on_integer_matrices():
    """Xi(A)^2 = sum_{i != j} a_ij^2 (Sec. 2.1, eq. (Omega_A)) in exact integer
    arithmetic: small integer entries make every square and partial sum exact
    in binary64, so the oracle's value is the correctly rounded square root
    of the exact integer, and Xi(A)^2 + sum a_ii^2 = ||A||_F^2 exactly."""
    r = np.random.default_rng(71)
    for n in (1, 2, 5, 17):
        M = r.integers(-1000, 1001, (n, n))
        exact_off = sum(int(M[i, j]) ** 2 for i in range(n) for j in range(n) if i != j)
        exact_all = sum(int(v) ** 2 for v in M.ravel())
        assert oracle.off_norm(M.astype(float)) == np.sqrt(float(exact_off))
        assert exact_off + sum(int(M[i, i]) ** 2 for i in range(n)) == exact_all
        # invariant under a symmetric permutation (the same set of entries)
        p = r.permutation(n)
        assert oracle.off_norm(M[np.ix_(p, p)].astype(float)) == np.sqrt(float(exact_off))


def test_relative_measure_closed_forms_and_scaling():
    """max_{i != j} |a_ij| / sqrt(|a_ii a_jj|): the 2 x 2 closed form, the
    zero-diagonal rule, and invariance under a two-sided diagonal scaling
    D A D (the property the relative stop test is for; powers of two keep
    the scaled entries exact)."""
    assert oracle.rel_off(np.array([[4.0, 3.0], [3.0, 9.0]])) == 0.5
    assert oracle.rel_off(np.array([[4.0, -6.0], [-6.0, 1.0]])) == 3.0
    assert oracle.rel_off(np.diag([1.0, 2.0, 3.0])) == 0.0
    Z = np.array([[0.0, 1e-9], [1e-9, 1.0]])
    assert np.isinf(oracle.rel_off(Z))
    assert oracle.rel_off(np.array([[0.0, 0.0], [0.0, 1.0]])) == 0.0
    r = np.random.default_rng(72)
    n = 12
    A = gen.sym_gaussian(n, 73) + np.diag(r.uniform(1.0, 2.0, n))
    d = 2.0 ** r.integers(-30, 30, n)
    B = d[:, None] * A * d[None, :]
    assert abs(oracle.rel_off(B) - oracle.rel_off(A)) <= 8 * U * oracle.rel_off(A)
    # the maximum is attained at the entry with the largest normalised size
    i, j = 3, 8
    A2 = np.diag(np.full(n, 4.0))
    A2[i, j] = A2[j, i] = 2.0
    A2[1, 2] = A2[2, 1] = 1.0
    assert oracle.rel_off(A2) == 0.5


# ------------------------------------------------------------------ special inputs
@pytest.mark.parametrize("scalar", [False, True])
def test_diagonal_input_no_rotation(scalar):
    d = np.array([-3.0, -1.0, 0.0, 0.5, 2.0, 7.0, 7.5, 9.0, 11.0, 12.0])
    A = np.diag(d)
    w, Q, Af, st, status = oracle.syev(A, b=2, scalar=scalar)
    assert status == 0 and st.rotations == 0 and st.sweeps == 0
    assert np.array_equal(w, d) and np.array_equal(Q, np.eye(len(d)))


def test_sorted_output_permutes_q():
    d = np.array([3.0, -1.0, 2.0, 0.0])
    w, Q, *_ = oracle.syev(np.diag(d), b=1)
    assert np.array_equal(w, np.sort(d))
    P = np.eye(4)[:, np.argsort(d, kind="stable")]
    assert np.array_equal(Q, P)


# ------------------------------------------------------------------ known spectrum
@pytest.mark.parametrize("b,ordering,kind", [
    (8, oracle.ORDER_ROUND_ROBIN, "uniform"),
    (5, oracle.ORDER_ROUND_ROBIN, "uniform"),     # ragged: 64 = 12*5 + 4
    (8, oracle.ORDER_ANTI_DIAGONAL, "uniform"),
    (8, oracle.ORDER_ROUND_ROBIN, "graded"),
    (64, oracle.ORDER_ROUND_ROBIN, "uniform"),    # n <= b: a single padded pair
])
def test_known_spectrum_blocked(b, ordering, kind):
    n = 64
    A, lam = gen.sym_known(n, kind, seed=21)
    w, Q, Af, st, status = oracle.syev(A, b=b, ordering=ordering)
    nrm2 = np.abs(lam).max()
    assert status == 0
    assert np.abs(w - np.sort(lam)).max() <= 1e-13 * nrm2
    assert np.linalg.norm(A @ Q - Q * w[None, :]) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13 * n


def _clustered(n, seed, width=1e-12, m=5):
    """A = Q diag(lam) Q^T with m eigenvalues within `width` of 1 and the rest
    in [-1, 0.5] (gap 0.5 to the cluster); returns A, lam, the cluster's basis."""
    r = gen.rng(seed)
    Q = gen.haar_q(n, n, r)
    lam = np.concatenate([1.0 + width * np.arange(m), r.uniform(-1.0, 0.5, n - m)])
    A = (Q * lam[None, :]) @ Q.T
    return np.asfortranarray(0.5 * (A + A.T)), lam, Q[:, :m]


@pytest.mark.parametrize("scalar,b", [(False, 4), (True, 1)])
def test_clustered_eigenvalues_invariant_subspace(scalar, b):
    """Within a tight cluster the eigenvectors are not unique but the
    invariant subspace is: its projector matches the constructed one within
    the perturbation bound u ||A|| / gap (Davis-Kahan sin-theta), and every
    eigenvalue matches within 1e-13 ||A||_2."""
    n, m = 40, 5
    A, lam, Qc = _clustered(n, 31, m=m)
    w, Q, Af, st, status = oracle.syev(A, b=b, scalar=scalar)
    assert status == 0
    assert np.abs(w - np.sort(lam)).max() <= 1e-13
    P = Q[:, -m:] @ Q[:, -m:].T
    assert np.linalg.norm(P - Qc @ Qc.T, 2) <= 1e-12
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13 * n


def test_known_spectrum_scalar():
    n = 48
    A, lam = gen.sym_known(n, "uniform", seed=22)
    w, Q, Af, st, status = oracle.syev(A, scalar=True)
    assert status == 0
    assert np.abs(w - np.sort(lam)).max() <= 1e-13
    assert np.linalg.norm(A @ Q - Q * w[None, :]) <= 1e-12 * np.linalg.norm(A)


def test_trace_and_frobenius_invariance_through_steps():
    n, b = 40, 4
    A = gen.sym_gaussian(n, 31)
    N = oracle.padded_blocks(n, b)
    tab = oracle.ordering(oracle.ORDER_ROUND_ROBIN, N)
    Q = np.eye(n)
    tr0, fr0 = np.trace(A), np.linalg.norm(A)
    Ak = A.copy()
    for s in range(len(tab)):
        Ak, Q, _ = oracle.syev_step(Ak, Q, b, tab[s])
        assert abs(np.trace(Ak) - tr0) <= 1e-13 * fr0
        assert abs(np.linalg.norm(Ak) - fr0) <= 1e-13 * fr0
    assert np.abs(Q @ Ak @ Q.T - A).max() <= 1e-13 * fr0


def test_block_off2_identity_over_one_step():
    """off^2(A') = off^2(A) - sum_p (off^2(Ahat_p) - off^2(Dhat_p)) (Algorithm 2:
    every non-pivot block is multiplied by orthogonal factors only, and the
    pivot blocks are replaced by Dhat)."""
    n, b = 48, 6
    A = gen.sym_gaussian(n, 32)
    N = oracle.padded_blocks(n, b)
    step = oracle.ordering(oracle.ORDER_ROUND_ROBIN, N)[3]
    drop = 0.0
    for (I, J) in step:
        idx = np.r_[I * b:(I + 1) * b, J * b:(J + 1) * b]
        Ah = A[np.ix_(idx, idx)]
        D, V, rot, sw = oracle.pivot_solve(Ah)
        drop += _offsq(Ah) - _offsq(D)
    A2, _, _ = oracle.syev_step(A, None, b, step, inner_max=30)
    assert abs(_offsq(A2) - (_offsq(A) - drop)) <= 1e-12 * np.sum(A * A)


@pytest.mark.parametrize("order", [0, 1])
def test_step_pivot_blocks_hold_dhat_and_match_explicit_product(order):
    """The update formulas of Algorithm 2 applied to the pivot itself give
    Vhat^T Ahat Vhat = Dhat, and the step writes Dhat there; with pivot_order 1
    the eigenpairs are first permuted (Qhat <- Qhat P) so diag(Dhat) descends."""
    n, b = 32, 4
    A = gen.sym_gaussian(n, 33)
    N = oracle.padded_blocks(n, b)
    step = oracle.ordering(oracle.ORDER_ROUND_ROBIN, N)[0]
    A2, _, _ = oracle.syev_step(A, None, b, step, inner_max=30, pivot_order=order)
    W = np.eye(n)
    for (I, J) in step:
        idx = np.r_[I * b:(I + 1) * b, J * b:(J + 1) * b]
        Ah = A[np.ix_(idx, idx)]
        D, V, rot, sw = oracle.pivot_solve(Ah)
        if order == 1:
            perm = np.argsort(-np.diag(D), kind="stable")
            D, V = D[np.ix_(perm, perm)], V[:, perm]
            assert np.all(np.diff(np.diag(A2[np.ix_(idx, idx)])) <= 0)
        assert np.abs(V.T @ Ah @ V - D).max() <= 1e-14 * np.abs(Ah).max() * 2 * b
        assert np.array_equal(A2[np.ix_(idx, idx)], D)
        W[np.ix_(idx, idx)] = V
    # the whole step is A' = W^T A W off the pivot blocks (W = direct sum of Vhat)
    ref = W.T @ A @ W
    assert np.abs(A2 - ref).max() <= 1e-13 * np.abs(A).max() * n


def test_pivot_solve_orthogonal_and_diagonal():
    Ah = gen.sym_gaussian(32, 34)
    D, V, rot, sw = oracle.pivot_solve(Ah)
    assert rot > 0 and sw >= 2
    assert np.abs(V.T @ V - np.eye(32)).max() <= 1e-14
    od = np.abs(D - np.diag(np.diag(D)))
    dd = np.sqrt(np.abs(np.diag(D)))
    assert (od <= 4 * U * np.outer(dd, dd) + 1e-300).all()
    assert np.allclose(np.sort(np.diag(D)), np.linalg.eigvalsh(Ah), atol=1e-13, rtol=0)


def test_pivot_solve_preserves_energy_without_bias():
    """||Dhat||_F = ||Ahat||_F (orthogonal similarity).  The diagonal is
    carried as hi + lo so that late rotations whose diagonal change is below
    half an ulp do not drop the energy of the zeroed entry: the mean change over
    many pivots stays within rounding noise instead of a systematic -4u."""
    ch = []
    for sd in range(16):
        Ah = gen.sym_gaussian(128, 700 + sd)
        D, V, rot, sw = oracle.pivot_solve(Ah)
        e0 = np.sum(Ah * Ah)
        ch.append((np.sum(D * D) - e0) / e0 / U)
    assert abs(np.mean(ch)) <= 1.0, np.mean(ch)


def test_pivot_eigenvectors_keep_unit_length():
    """Columns of Vhat stay unit length on average: the rotation update in
    Rutishauser's form does not let the small angles of late sweeps lengthen
    them (the plain c x - s y form drifts by about +180 u at k = 128)."""
    d = []
    for sd in range(6):
        D, V, rot, sw = oracle.pivot_solve(gen.sym_gaussian(128, 500 + sd))
        d.append(np.diag(V.T @ V) - 1.0)
    assert abs(np.mean(np.concatenate(d))) / U <= 2.0


def test_blocked_accuracy_matches_lapack_at_n512():
    """Backward-stable accuracy at a size where drifting rotations would
    show: eigenvalues within 2e-14 ||A||_2 of LAPACK (the plain form of the
    rotation update and a single-word diagonal give ~1.5e-13 here), and the
    accumulated Q orthogonal to 1e-15 n."""
    A, lam = gen.sym_known(512, "uniform", seed=2)
    w, Q, _, st, status = oracle.syev(A, b=16)
    wl = np.linalg.eigvalsh(A)
    assert status == 0
    assert np.abs(w - wl).max() <= 2e-14 * np.abs(wl).max()
    assert np.linalg.norm(Q.T @ Q - np.eye(512)) <= 1e-15 * 512


def test_inner_sweep_cap_gives_approximate_solve():
    Ah = gen.sym_gaussian(32, 35)
    D, V, rot, sw = oracle.pivot_solve(Ah, max_sweeps=1)
    assert sw == 1 and _offsq(D) > 0 and _offsq(D) < _offsq(Ah)
    assert np.abs(V.T @ Ah @ V - D).max() <= 1e-13


# ------------------------------------------------------------------ brute force n <= 4
def _charpoly_exact(A):
    """Coefficients (highest first) of det(x I - A) in exact rationals, by
    Faddeev-LeVerrier: M_0 = 0, c_n = 1; M_k = A M_{k-1} + c_{n-k+1} I,
    c_{n-k} = -tr(A M_k)/k."""
    n = len(A)
    F = [[Fraction(float(A[i][j])) for j in range(n)] for i in range(n)]
    coeffs = [Fraction(1)]
    M = [[Fraction(0)] * n for _ in range(n)]
    c_prev = Fraction(1)
    for k in range(1, n + 1):
        AM = [[sum(F[i][l] * M[l][j] for l in range(n)) for j in range(n)] for i in range(n)]
        M = [[AM[i][j] + (c_prev if i == j else 0) for j in range(n)] for i in range(n)]
        AMk = [[sum(F[i][l] * M[l][j] for l in range(n)) for j in range(n)] for i in range(n)]
        c = -sum(AMk[i][i] for i in range(n)) / k
        coeffs.append(c)
        c_prev = c
    return coeffs


def _peval(p, x):
    v = Fraction(0)
    for c in p:
        v = v * x + c
    return v


def _prem(a, b):
    a = list(a)
    while len(a) >= len(b) and any(a):
        f = a[0] / b[0]
        for i in range(len(b)):
            a[i] -= f * b[i]
        a.pop(0)
    while a and a[0] == 0:
        a.pop(0)
    return a


def _sturm_roots(p, lo, hi, iters=80):
    deriv = [c * (len(p) - 1 - i) for i, c in enumerate(p[:-1])]
    chain = [p, deriv]
    while len(chain[-1]) > 1:
        r = _prem(chain[-2], chain[-1])
        if not r:
            break
        chain.append([-c for c in r])

    def count(x):  # sign changes of the chain at x
        s = [_peval(q, x) for q in chain]
        s = [v for v in s if v != 0]
        return sum(1 for a, b in zip(s, s[1:]) if (a > 0) != (b > 0))

    n = len(p) - 1
    roots = []
    for kth in range(n):  # kth smallest root: count(lo) - count(x) = #roots in (lo, x]
        a, b = Fraction(lo), Fraction(hi)
        c_lo = count(a)
        for _ in range(iters):
            mid = (a + b) / 2
            if c_lo - count(mid) > kth:
                b = mid
            else:
                a = mid
            a = Fraction(float(a)) if _ % 8 == 7 else a
        roots.append(float((a + b) / 2))
    return roots


@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("seed", [40, 41, 42])
def test_brute_force_charpoly_roots(n, seed):
    A = gen.sym_gaussian(n, seed)
    p = _charpoly_exact(A)
    R = float(np.abs(A).sum(axis=1).max()) + 1.0
    roots = _sturm_roots(p, -R, R)
    for scalar in (False, True):
        w, Q, *_ = oracle.syev(A, b=1, scalar=scalar)
        assert np.abs(w - np.array(roots)).max() <= 1e-14 * max(1.0, np.abs(roots).max())


# ------------------------------------------------------------------ LAPACK witness
@pytest.mark.parametrize("n,b", [(100, 8), (77, 10)])
def test_lapack_witness(n, b):
    A = gen.sym_gaussian(n, 50 + n)
    w, Q, Af, st, status = oracle.syev(A, b=b)
    wl = np.linalg.eigvalsh(A)
    nrm2 = np.abs(wl).max()
    assert status == 0 and st.sweeps >= 3
    assert np.abs(w - wl).max() <= 1e-13 * nrm2
    assert np.linalg.norm(A @ Q - Q * w[None, :]) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13 * n
    assert st.off_final <= 1e-14 * st.norm_fro or st.stalled


def test_blocked_and_scalar_agree_and_sweep_history_decreases():
    A = gen.sym_gaussian(60, 61)
    w1, *_ , st1, _ = oracle.syev(A, b=6)
    w2, *_ , st2, _ = oracle.syev(A, scalar=True)
    assert np.abs(w1 - w2).max() <= 1e-13 * np.abs(w1).max()
    h = st1.off_hist
    assert all(h[i + 1] < h[i] for i in range(len(h) - 1))


def test_pivot_order_sorting_keeps_the_answer_and_saves_sweeps():
    """The permutation after each pivot solve changes the iterates, not the
    eigenvalues; on a graded spectrum it shortens the iteration."""
    A, lam = gen.sym_known(96, "graded", seed=63)
    w0, Q0, _, st0, s0 = oracle.syev(A, b=8, pivot_order=0)
    w1, Q1, _, st1, s1 = oracle.syev(A, b=8, pivot_order=1)
    assert s0 == 0 and s1 == 0
    assert np.abs(w0 - w1).max() <= 1e-13 * np.abs(lam).max()
    assert st1.sweeps < st0.sweeps


def test_max_sweeps_reports_nonconvergence():
    A = gen.sym_gaussian(40, 62)
    w, Q, Af, st, status = oracle.syev(A, b=4, max_sweeps=1)
    assert status == 1 and st.sweeps == 1


# ------------------------------------------------------------------ padding
def test_padding_is_exact():
    """b that does not divide n: zero rows/columns stay exactly zero, so the
    ragged run equals the run on the explicitly zero-padded matrix (without
    the pivot permutation, which treats explicit zeros as real rows)."""
    n, b = 10, 4
    A = gen.sym_gaussian(n, 70)
    Ap = np.zeros((12, 12), order="F")
    Ap[:n, :n] = A
    w, Q, Af, st, s1 = oracle.syev(A, b=b, pivot_order=0)
    wp, Qp, Afp, stp, s2 = oracle.syev(Ap, b=b, pivot_order=0)
    assert st.rotations == stp.rotations and st.sweeps == stp.sweeps
    # the padded run has two extra exact zero eigenvalues; removing them gives w
    z = np.where(wp == 0.0)[0]
    assert len(z) >= 2
    keep = np.ones(12, bool)
    keep[z[:2]] = False
    assert np.array_equal(wp[keep], w)
    assert np.all(Afp[n:, :] == 0.0) and np.all(Afp[:, n:] == 0.0)
    # with the permutation the padding positions stay fixed: same eigenvalues
    w1, Q1, *_ = oracle.syev(A, b=b, pivot_order=1)
    assert np.abs(w1 - np.linalg.eigvalsh(A)).max() <= 1e-13 * np.abs(w1).max()
    assert np.linalg.norm(A @ Q1 - Q1 * w1[None, :]) <= 1e-12 * np.linalg.norm(A)


def test_padding_inside_a_step():
    n, b = 12, 4
    A = np.zeros((n, n), order="F")
    A[:10, :10] = gen.sym_gaussian(10, 71)
    tab = oracle.ordering(oracle.ORDER_ANTI_DIAGONAL, 3)
    Ak = A
    for step in tab:
        Ak, _, _ = oracle.syev_step(Ak, None, b, step, pivot_order=0)
        assert np.all(Ak[10:, :] == 0.0) and np.all(Ak[:, 10:] == 0.0)


# ------------------------------------------------------------------ graded spectra
def test_graded_dhd_relative_accuracy_vs_mpmath():
    mpmath = pytest.importorskip("mpmath")
    n = 24
    A, d, H = gen.graded_dhd(n, seed=4)
    mpmath.mp.dps = 40
    ev = mpmath.eigsy(mpmath.matrix(A.tolist()), eigvals_only=True)
    exact = np.sort(np.array([float(x) for x in ev]))
    w, Q, Af, st, status = oracle.syev(A, b=4, conv=oracle.CONV_REL, tol=4 * U)
    assert status == 0
    assert exact.min() > 0 and exact.max() / exact.min() > 1e10
    assert np.abs(w - exact).max() / 1.0 <= 1e-12 * exact.max()
    assert (np.abs(w - exact) / exact).max() <= 1e-12


# ------------------------------------------------------------------ orderings
def _read_groups():
    out = []
    for line in open(os.path.join(GOLD, "anti_diagonal_N8_list.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        out.append({tuple(int(x) - 1 for x in tok.split(",")) for tok in line.split()})
    return out


def test_algorithm3_matches_printed_list():
    printed = _read_groups()
    tab = oracle.ordering(oracle.ORDER_ANTI_DIAGONAL, 8)
    assert len(tab) == 8 and len(printed) == 8
    assert {frozenset(g) for g in tab} == {frozenset(g) for g in printed}
    # our group K holds the pairs with (I+J) mod 8 == K (1-based); the printed
    # list is ordered by label l = 1..8 with K = (2 - l) mod 8
    for ell, g in enumerate(printed, start=1):
        assert set(tab[(2 - ell) % 8]) == g


def test_algorithm3_matches_printed_label_matrix():
    tab = oracle.ordering(oracle.ORDER_ANTI_DIAGONAL, 8)
    label = {}
    for K, g in enumerate(tab):
        for (I, J) in g:
            label[(I, J)] = (2 - K) % 8 or 8
    rows = [l.split() for l in open(os.path.join(GOLD, "anti_diagonal_N8_labels.txt"))
            if l.strip() and not l.startswith("#")]
    for I, row in enumerate(rows):
        for k, tok in enumerate(row):
            assert label[(I, I + 1 + k)] == int(tok)


@pytest.mark.parametrize("fname,ell", [("group_one_pattern.txt", 1), ("group_two_pattern.txt", 2)])
def test_transformation_patterns(fname, ell):
    tab = oracle.ordering(oracle.ORDER_ANTI_DIAGONAL, 8)
    group = sorted(tab[(2 - ell) % 8], key=lambda p: -p[0])  # numbered in printed order
    owner = {}
    for t, (I, J) in enumerate(group, start=1):
        owner[I] = t
        owner[J] = t
    rows = [l.split() for l in open(os.path.join(GOLD, fname))
            if l.strip() and not l.startswith("#")]
    for I, row in enumerate(rows):
        for k, tok in enumerate(row):
            J = I + k
            L, R = owner.get(I), owner.get(J)
            if L is not None and L == R:
                want = f"{L}*"
            else:
                want = f"{L if L else '_'}{R if R else '_'}"
            assert tok == want, (I, J, tok, want)


@pytest.mark.parametrize("N", list(range(2, 41, 2)))
def test_round_robin_covers_every_pair_once(N):
    tab = oracle.ordering(oracle.ORDER_ROUND_ROBIN, N)
    assert len(tab) == N - 1
    seen = set()
    for g in tab:
        assert len(g) == N // 2
        used = [x for p in g for x in p]
        assert len(set(used)) == len(used)  # disjoint
        for (I, J) in g:
            assert 0 <= I < J < N
            seen.add((I, J))
    assert len(seen) == N * (N - 1) // 2


@pytest.mark.parametrize("N", list(range(2, 30)))
def test_anti_diagonal_covers_every_pair_once(N):
    tab = oracle.ordering(oracle.ORDER_ANTI_DIAGONAL, N)
    assert len(tab) == N
    allp = [p for g in tab for p in g]
    assert len(allp) == len(set(allp)) == N * (N - 1) // 2
    for K, g in enumerate(tab):
        used = [x for p in g for x in p]
        assert len(set(used)) == len(used)
        assert all((I + 1 + J + 1) % N == K for (I, J) in g)
        assert len(g) in (N // 2, N // 2 - 1, (N - 1) // 2)


# ------------------------------------------------------------------ one-sided SVD
def test_hestenes_rotation_orthogonalises_two_columns():
    G = gen.tall_gaussian(50, 2, 80, dtype=np.float64)
    U, s, V, st, status = oracle.gesvd(G, b=1, scalar=True, max_sweeps=1)
    Gr = U * s[None, :]
    assert abs(Gr[:, 0] @ Gr[:, 1]) <= 1e-15 * s[0] * s[1] * 50
    sl = np.linalg.svd(G, compute_uv=False)
    assert np.abs(s - sl).max() <= 1e-14 * sl[0]


@pytest.mark.parametrize("scalar,b", [(False, 4), (False, 6), (True, 1)])
def test_known_singular_values(scalar, b):
    m, n = 200, 40
    G, sig = gen.svd_known(m, n, seed=81, decades=6.0)
    U, s, V, st, status = oracle.gesvd(G, b=b, scalar=scalar)
    assert status == 0
    assert np.abs(s - sig).max() <= 1e-13 * sig[0]
    big = sig >= 1e-3 * sig[0]
    assert (np.abs(s - sig)[big] / sig[big]).max() <= 1e-12
    assert np.linalg.norm(U.T @ U - np.eye(n)) <= 1e-12 * n
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-13 * n
    assert np.linalg.norm(G @ V - U * s[None, :]) <= 1e-13 * np.linalg.norm(G)


@pytest.mark.parametrize("qr", [False, True])
def test_clustered_singular_values_subspaces(qr):
    """Four singular values within 1e-12 of each other (gap 0.5 to the
    rest): the right and left singular subspaces of the cluster (their
    projectors) match the constructed ones within u ||G|| / gap, direct and
    QR-preconditioned."""
    m, n, c = 160, 30, 4
    r = gen.rng(83)
    Uc = gen.haar_q(m, n, r)
    Vc = gen.haar_q(n, n, r)
    sig = np.concatenate([1.0 + 1e-12 * np.arange(c)[::-1], r.uniform(0.01, 0.5, n - c)])
    G = np.asfortranarray((Uc * sig[None, :]) @ Vc.T)
    U, s, V, st, status = (oracle.gesvd_qr if qr else oracle.gesvd)(G, b=5)
    assert status == 0
    assert np.abs(s - np.sort(sig)[::-1]).max() <= 1e-13
    PV = V[:, :c] @ V[:, :c].T
    PU = U[:, :c] @ U[:, :c].T
    assert np.linalg.norm(PV - Vc[:, :c] @ Vc[:, :c].T, 2) <= 1e-12
    assert np.linalg.norm(PU - Uc[:, :c] @ Uc[:, :c].T, 2) <= 1e-12


@pytest.mark.parametrize("transpose,m,n,b", [(True, 200, 40, 4), (False, 200, 40, 4), (True, 60, 60, 6),
                                             (True, 150, 33, 5)])
def test_qr_preconditioned_svd_known_singular_values(transpose, m, n, b):
    """G = QR, the one-sided method on R^T (or R), U = Q times the left
    singular vectors of R: the constructed sigma, orthonormal U and V, and
    G V = U Sigma."""
    G, sig = gen.svd_known(m, n, seed=85, decades=6.0)
    U, s, V, st, status = oracle.gesvd_qr(G, b=b, transpose=transpose)
    assert status == 0
    assert np.abs(s - sig).max() <= 1e-13 * sig[0]
    big = sig >= 1e-3 * sig[0]
    assert (np.abs(s - sig)[big] / sig[big]).max() <= 1e-12
    assert np.linalg.norm(U.T @ U - np.eye(n)) <= 1e-12 * n
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-12 * n
    assert np.linalg.norm(G @ V - U * s[None, :]) <= 1e-13 * np.linalg.norm(G)
    s_direct = oracle.gesvd(G, b=b)[1]
    assert np.abs(s - s_direct).max() <= 1e-13 * sig[0]


def test_qr_preconditioned_svd_on_graded_columns_keeps_lapack_values():
    # columns scaled over 8 decades: the factor R inherits the grading
    m, n = 120, 24
    G = gen.tall_gaussian(m, n, 86, dtype=np.float64) * (10.0 ** -np.linspace(0, 8, n))[None, :]
    U, s, V, st, status = oracle.gesvd_qr(G, b=4)
    sl = np.linalg.svd(G, compute_uv=False)
    assert status == 0 and np.abs(s - sl).max() <= 1e-13 * sl[0]
    assert np.linalg.norm(G @ V - U * s[None, :]) <= 1e-13 * np.linalg.norm(G)


def test_svd_lapack_witness_and_zero_column():
    m, n = 90, 30
    G = gen.tall_gaussian(m, n, 82, dtype=np.float64)
    G[:, 7] = 0.0
    U, s, V, st, status = oracle.gesvd(G, b=4)
    sl = np.linalg.svd(G, compute_uv=False)
    assert status == 0
    assert np.abs(s - sl).max() <= 1e-13 * sl[0]
    assert s[-1] == 0.0 and np.all(U[:, -1] == 0.0)
    assert np.all(np.isfinite(U))


def test_gram_is_sum_over_row_tiles():
    m, b = 300, 5
    G = gen.tall_gaussian(m, 20, 83, dtype=np.float64)
    full = oracle.gram_pair(G, b, 1, 3)
    idx = np.r_[1 * b:2 * b, 3 * b:4 * b]
    assert np.abs(full - G[:, idx].T @ G[:, idx]).max() <= 1e-13 * m
    parts = sum(oracle.gram_pair(G[r:r + 64], b, 1, 3) for r in range(0, m, 64))
    assert np.abs(parts - full).max() <= 1e-13 * m


def test_svd_step_returns_pre_rotation_measure():
    m, b = 60, 3
    G = gen.tall_gaussian(m, 12, 84, dtype=np.float64)
    tab = oracle.ordering(oracle.ORDER_ROUND_ROBIN, 4)
    G2, V2, r = oracle.gesvd_step(G, np.eye(12), b, tab[0], tol_rel=1e-15)
    want = 0.0
    for (I, J) in tab[0]:
        idx = np.r_[I * b:(I + 1) * b, J * b:(J + 1) * b]
        Ah = G[:, idx].T @ G[:, idx]
        d = np.sqrt(np.diag(Ah))
        R = np.abs(Ah) / np.outer(d, d)
        np.fill_diagonal(R, 0)
        want = max(want, R.max())
    assert abs(r - want) <= 1e-13
    assert np.abs(G2 @ V2.T - G).max() <= 1e-13 * np.abs(G).max() * 12


# ------------------------------------------------------------------ bf16 split
def test_bf16_split_definition():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(90)
    x = (r.standard_normal(20000) * 10.0 ** r.uniform(-5, 5, 20000)).astype(np.float32)
    hi, lo = oracle.split_bf16(x)
    hi_t = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(hi, hi_t)  # round-to-nearest-even, as torch's cast
    assert np.array_equal(lo, torch.from_numpy(x - hi).to(torch.bfloat16).float().numpy())
    assert np.all(hi.view(np.uint32) & 0xFFFF == 0)
    rel = np.abs((hi.astype(np.float64) + lo) - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -16
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8], np.float32)
    h, _ = oracle.split_bf16(ties)
    assert h[0] == 1.0 and h[1] == np.float32(1 + 2 ** -6)


# ------------------------------------------------------------------ pivoting step (QRCP, Sec. 2.1)
@pytest.mark.parametrize("r,c,seed", [(8, 16, 1), (5, 12, 2), (16, 32, 3), (7, 7, 4)])
def test_qrcp_order_matches_lapack(r, c, seed):
    """The QRCP rule against LAPACK's pivoted QR (scipy, dgeqp3) on generic
    matrices: the same leading columns in the same order."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    X = np.random.default_rng(seed).standard_normal((r, c))
    mine = oracle.qrcp_perm(X)
    _, _, piv = scipy_linalg.qr(X, pivoting=True, mode="economic")
    assert list(mine[:min(r, c)]) == list(piv[:min(r, c)])
    assert sorted(mine) == list(range(c))


def test_qrcp_pivoting_step_keeps_the_step_a_similarity():
    """pivot_order = 2 permutes each pivot's eigenpairs only: the step is
    still an orthogonal similarity (spectrum, Frobenius norm, Q orthogonal),
    the leading b x b block of every Vhat P is well conditioned, and the
    full solve meets the FP64 gates."""
    n, b = 48, 6
    A, lam = gen.sym_known(n, "uniform", seed=91)
    tab = oracle.ordering(oracle.ORDER_ROUND_ROBIN, n // b)
    A2, Q2, rot = oracle.syev_step(A, np.eye(n), b, tab[0], pivot_order=2)
    assert rot > 0
    assert np.abs(np.linalg.eigvalsh(A2) - np.sort(lam)).max() <= 1e-14 * n
    assert np.linalg.norm(Q2.T @ Q2 - np.eye(n)) <= 1e-14 * n
    assert abs(np.linalg.norm(A2) - np.linalg.norm(A)) <= 1e-14 * np.linalg.norm(A)
    w, Q, Af, st, status = oracle.syev(A, b=b, pivot_order=2)
    assert status == 0
    assert np.abs(w - np.sort(lam)).max() <= 1e-13
    assert np.linalg.norm(A @ Q - Q * w[None, :]) <= 1e-12 * np.linalg.norm(A)


def test_qrcp_pivoting_one_sided():
    G, sig = gen.svd_known(150, 30, seed=92, decades=6.0)
    U, s, V, st, status = oracle.gesvd(G, b=5, pivot_order=2)
    assert status == 0 and np.abs(s - sig).max() <= 1e-13 * sig[0]
    assert np.linalg.norm(G @ V - U * s[None, :]) <= 1e-13 * np.linalg.norm(G)


def test_qrcp_selects_a_well_conditioned_leading_block():
    """The point of the pivoting step: the leading rows of Vhat have
    orthonormal rows, and the b columns QRCP moves to the front form a block
    much better conditioned than the unpermuted leading block of a pivot
    whose eigenvectors are scrambled."""
    b = 8
    r = np.random.default_rng(93)
    Qh = np.linalg.qr(r.standard_normal((2 * b, 2 * b)))[0]
    Ah = Qh @ np.diag(np.linspace(-1, 1, 2 * b)) @ Qh.T
    _, V, _, _ = oracle.pivot_solve(Ah)
    perm = oracle.qrcp_perm(V[:b, :])
    s_sel = np.linalg.svd(V[:b, perm[:b]], compute_uv=False)[-1]
    s_first = np.linalg.svd(V[:b, :b], compute_uv=False)[-1]
    assert s_sel >= s_first and s_sel > 0.1
