"""GPU parity of the stop statistic (off-norm and relative measure) against
the CPU oracle.

The two-sided method stops when Xi(A) = sqrt(sum_{i != j} a_ij^2) <=
tol ||A||_F (Sec. 2.1, eq. (Omega_A); Algorithm 1's stop test), or, under
the relative criterion, when max_{i != j} |a_ij| / sqrt(|a_ii a_jj|) <= tol.
The library computes both with one fixed-order reduction kernel.  These tests
put its values next to the oracle's:

* on arbitrary matrices through jacobi_off_norm (every shape class: tiny,
  ragged, lda > n, zero, diagonal, zero diagonal entries);
* on the matrix one step leaves (jacobi_syev_step vs oracle.syev_step);
* after every sweep of a full solve: the statistic the library reports for
  sweep s (jacobi_stats.off_hist / rel_hist) against the oracle's off-norm of
  the iterate the library returns when it stops after s sweeps, and against
  the oracle's own per-sweep history (the two trajectories differ by the
  iterates' difference, which is measured).

Tolerance of a sum of N = n^2 non-negative rounded squares: each order's
relative error is below gamma_d = d u / (1 - d u) for a summation depth d
(recursive summation in the oracle: d = n^2 + 1; the library: per-thread
sums of at most ceil(n/G) ceil(n/256) terms, a tree of 8 levels over the 256
threads of a CTA, then the G CTA partials in order, G = min(n, 608)).  So
|off_gpu - off_or| <= (gamma_{d_gpu} + gamma_{d_or}) / 2 * off + 2u off
(the square root halves a relative error and adds one rounding).  The
relative measure is a maximum of quotients, each within 4 u on either side.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import jacobi_inputs as gen
import oracle

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def jg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_28952_gb300 as m
    m.lib()
    return m


def _dev(x, ld=None):
    import torch

    import paper_2608_28952_gb300 as m
    x = np.asarray(x, dtype=np.float64)
    if ld is None:
        return m.colmajor(x, device="cuda", dtype=torch.float64)
    buf = m.colmajor_empty(ld, x.shape[1], torch.float64, "cuda").fill_(float("nan"))
    buf[: x.shape[0]].copy_(torch.from_numpy(x))
    return buf[: x.shape[0]]


def sum_tol(n: int) -> float:
    """Relative bound on the difference of the two off-norm evaluations."""
    G = max(1, min(n, 608))
    d_gpu = math.ceil(n / G) * math.ceil(n / 256) + 8 + G + 1
    d_or = n * n + 1
    gam = lambda d: d * U / (1.0 - d * U)
    return 0.5 * (gam(d_gpu) + gam(d_or)) + 2 * U


REL_TOL = 8 * U


def _check_entry(jg, A, ld=None):
    n = A.shape[0]
    rc, off, fro, rel = jg.jacobi_off_norm(_dev(A, ld), want_rel=True)
    assert rc == 0
    off_or, rel_or = oracle.off_norm(A), oracle.rel_off(A)
    fro_or = math.sqrt(off_or ** 2 + float(np.sum(np.diag(A) ** 2)))
    tol = sum_tol(n)
    assert abs(off - off_or) <= tol * off_or, (off, off_or)
    assert abs(fro - fro_or) <= (tol + 4 * U) * fro_or, (fro, fro_or)
    if math.isinf(rel_or):
        assert math.isinf(rel)
    else:
        assert abs(rel - rel_or) <= REL_TOL * rel_or, (rel, rel_or)
    rc, off2, fro2, rel2 = jg.jacobi_off_norm(_dev(A, ld), want_rel=False)
    assert rc == 0 and off2 == off and fro2 == fro and rel2 == 0.0
    return off, rel


@pytest.mark.parametrize("n,ld", [(1, None), (2, 5), (3, None), (37, 40), (256, None),
                                  (609, 611), (1000, None)])
def test_off_norm_matches_oracle_on_random_matrices(jg, n, ld):
    """Gaussian symmetric and non-symmetric matrices, graded rows, lda > n
    (the rows past n hold NaN and must not be read)."""
    r = gen.rng(5100, n)
    _check_entry(jg, gen.sym_gaussian(n, 5100 + n), ld)
    _check_entry(jg, r.standard_normal((n, n)) * 10.0 ** r.uniform(-8, 8, (n, 1)), ld)


def test_off_norm_special_matrices(jg):
    n = 64
    assert _check_entry(jg, np.zeros((n, n)))[0] == 0.0
    d = np.diag(np.linspace(-3.0, 5.0, n))
    off, rel = _check_entry(jg, d)
    assert off == 0.0 and rel == 0.0
    # a zero diagonal entry under a non-zero off-diagonal entry: +inf
    A = np.diag(np.linspace(1.0, 2.0, n))
    A[5, 5] = 0.0
    A[5, 9] = A[9, 5] = 1e-3
    off, rel = _check_entry(jg, A)
    assert math.isinf(rel) and abs(off - math.sqrt(2) * 1e-3) <= 4 * U * off
    # the 2 x 2 closed form: off = sqrt(2)|b|, rel = |b| / sqrt(|a c|)
    rc, off, fro, rel = jg.jacobi_off_norm(_dev(np.array([[4.0, 3.0], [3.0, 9.0]])))
    assert rc == 0 and abs(off - 3.0 * math.sqrt(2.0)) <= 2 * U * off and rel == 0.5


def test_off_norm_after_one_step(jg):
    """The statistic of the matrix one step leaves, library vs oracle, on
    the same step's output (element-wise parity of the step itself is in
    test_gpu_evd): the library's value on its own output against the
    oracle's value on the oracle's output, within the step difference."""
    np_, b = 384, 32
    A0 = gen.sym_gaussian(np_, 5200)
    tab = oracle.ordering(0, np_ // b)
    for s in (0, 3):
        A_or, _, _ = oracle.syev_step(A0, None, b, tab[s])
        Ad = _dev(A0)
        assert jg.jacobi_syev_step(Ad, None, s, jg.params(b=b)) == 0
        rc, off, _, rel = jg.jacobi_off_norm(Ad)
        Ag = Ad.cpu().numpy()
        assert rc == 0
        off_or = oracle.off_norm(A_or)
        assert abs(off - oracle.off_norm(Ag)) <= sum_tol(np_) * off
        diff = oracle.off_norm(Ag - A_or) + np.linalg.norm(np.diag(Ag - A_or))
        assert abs(off - off_or) <= diff + 2 * sum_tol(np_) * off_or, (off, off_or, diff)
        assert abs(rel - oracle.rel_off(Ag)) <= REL_TOL * rel


def _per_sweep(jg, A, b, conv, tol, sweeps):
    """For s = 1..sweeps: the library's reported statistic after sweep s
    (from one solve capped at `sweeps`) and the iterate it returns when it
    stops after s sweeps."""
    w, Q, D, st = jg.syev(A, b=b, conv=conv, tol=tol, max_sweeps=sweeps)
    hist = list(st.off_hist), list(st.rel_hist)
    its = []
    for s in range(1, sweeps + 1):
        w, Q, D, st_s = jg.syev(A, b=b, conv=conv, tol=tol, max_sweeps=s)
        assert st_s.sweeps == s
        assert st_s.off_hist == hist[0][:s]          # the solve is deterministic
        assert st_s.off_final == hist[0][s - 1]
        its.append(D.cpu().numpy())
    return hist, its


@pytest.mark.parametrize("case", ["c1", "ragged", "dhd_rel"])
def test_stop_statistic_every_sweep(jg, case):
    """Every sweep's reported statistic equals the oracle's off-norm (and
    relative measure) of the iterate the library returns after that sweep;
    the oracle's own history agrees within the measured iterate difference
    (Xi is a seminorm: |Xi(X) - Xi(Y)| <= Xi(X - Y) <= ||X - Y||_F)."""
    if case == "c1":
        A, _ = gen.sym_known(256, "uniform", seed=gen.SEEDS["c1"])
        b, conv, tol = 16, 0, 1e-14
    elif case == "ragged":
        A = gen.sym_gaussian(203, 5300)
        b, conv, tol = 24, 0, 1e-14
    else:
        A, _, _ = gen.graded_dhd(160, seed=gen.SEEDS["c2dhd"])
        b, conv, tol = 16, 1, 4 * U
    n = A.shape[0]
    _, _, _, st_or, s_or = oracle.syev(A, b=b, conv=conv, tol=tol)
    w, Q, D_fin, st = jg.syev(A, b=b, conv=conv, tol=tol)
    D_fin = D_fin.cpu().numpy()
    assert s_or == 0 and st.status == 0 and abs(st.sweeps - st_or.sweeps) <= 1
    S = min(st.sweeps, st_or.sweeps)
    (off_h, rel_h), its = _per_sweep(jg, A, b, conv, tol, S)
    tol_sum = sum_tol(n)
    for s in range(S):
        D = its[s]
        assert abs(off_h[s] - oracle.off_norm(D)) <= tol_sum * off_h[s] + 1e-300, s
        if conv == 1:
            assert abs(rel_h[s] - oracle.rel_off(D)) <= REL_TOL * rel_h[s], s
        else:
            assert rel_h[s] == 0.0
        # the oracle's trajectory: its iterate after s + 1 sweeps, ordered
        # like the library's output (ascending diagonal, stable)
        _, _, A_or, st_s, _ = oracle.syev(A, b=b, conv=conv, tol=tol, max_sweeps=s + 1)
        perm = np.argsort(np.diag(A_or), kind="stable")
        A_or = A_or[np.ix_(perm, perm)]
        assert abs(st_s.off_hist[s] - st_or.off_hist[s]) <= tol_sum * st_or.off_hist[s]
        gap = np.linalg.norm(D - A_or)
        assert abs(off_h[s] - st_or.off_hist[s]) <= gap + 2 * tol_sum * st_or.off_hist[s], (
            s, off_h[s], st_or.off_hist[s], gap)
    # the final statistic passes the stop test and is the oracle's value on
    # the returned iterate
    assert abs(st.off_final - oracle.off_norm(D_fin)) <= tol_sum * st.off_final + 1e-300
    if conv == 0:
        assert st.off_final <= tol * st.norm_fro or st.stalled
    else:
        assert st.rel_final <= tol or st.stalled
        assert abs(st.rel_final - oracle.rel_off(D_fin)) <= REL_TOL * st.rel_final


def test_trajectory_of_a_well_conditioned_solve(jg):
    """Pivots with well separated eigenvalues (A = diag(1..2n) + 0.05 G):
    every step is well conditioned, and one step of the library and of the
    oracle agree within 1e-13 of the largest entry per entry (the step-parity
    tolerance of test_gpu_evd).  A step is an orthogonal similarity, so the
    differences add up: after t steps the iterates differ by at most
    t * n * 1e-13 max|A| in the Frobenius norm, and so do the per-sweep
    off-norms (plus the two summation errors)."""
    n, b = 256, 32
    d = np.linspace(1.0, 2.0 * n, n)
    A = np.asfortranarray(np.diag(d) + 0.05 * gen.sym_gaussian(n, 5400))
    _, _, _, st_or, s_or = oracle.syev(A, b=b)
    w, Q, D, st = jg.syev(A, b=b)
    assert s_or == 0 and st.status == 0 and st.sweeps == st_or.sweeps
    steps_per_sweep = n // b - 1
    amax = np.abs(A).max()
    for s in range(st.sweeps):
        a, o = st.off_hist[s], st_or.off_hist[s]
        bound = (s + 1) * steps_per_sweep * n * 1e-13 * amax + 2 * sum_tol(n) * o
        assert abs(a - o) <= bound, (s, a, o, bound)
    assert st.off_hist[0] > 1e3 * (steps_per_sweep * n * 1e-13 * amax)   # the first sweep is a real test
