"""GPU parity of the two-sided blocked Jacobi EVD against the CPU oracle.

Element-wise parity of single steps (Algorithm 2: pivot solves + block-row /
block-column updates), then full solves compared on what is unique
(eigenvalues; eigenvectors through residual and orthogonality, since they are
not unique).  Tolerances: |lambda - lambda_oracle| <= 1e-13 ||A||_2,
||AQ - QD||_F <= 1e-12 ||A||_F, ||Q^T Q - I||_F <= 1e-13 n.
"""
from __future__ import annotations

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


def _dev(x):
    import paper_2608_28952_gb300 as m
    import torch
    return m.colmajor(x, device="cuda", dtype=torch.float64)


def _np(t):
    return t.detach().cpu().numpy()


def check(A, w, Q, w_ref, eig=1e-13, res=1e-12, orth=1e-13):
    n = A.shape[0]
    nrm2 = max(np.abs(w_ref).max(), 1e-300)
    assert np.abs(w - w_ref).max() <= eig * nrm2, np.abs(w - w_ref).max() / nrm2
    if Q is not None:
        r = np.linalg.norm(A @ Q - Q * w[None, :])
        assert r <= res * max(np.linalg.norm(A), 1e-300), r / np.linalg.norm(A)
        o = np.linalg.norm(Q.T @ Q - np.eye(n))
        assert o <= orth * n, o / n


# ------------------------------------------------------------------ single steps
STEP_CASES = [
    (64, 8, 0, [0, 3, 6]),
    (96, 16, 0, [0, 4]),          # k = 32
    (256, 64, 0, [0, 1]),         # k = 128, shared-memory pivot at its limit
    (512, 128, 0, [0]),           # k = 256, pivot in global scratch
    (40, 5, 0, [0, 2]),           # odd b, ragged tiles
    (80, 8, 1, [0, 1, 5]),        # Algorithm 3 with frozen blocks
    (4, 1, 0, [0, 2]),            # b = 1: 2 x 2 pivots
]


def _step_pair(jg, A0, b, ordering, s):
    np_ = A0.shape[0]
    tab = oracle.ordering(ordering, np_ // b)
    A_or, Q_or, _ = oracle.syev_step(A0, np.eye(np_), b, tab[s])
    Ad, Qd = _dev(A0), _dev(np.eye(np_))
    assert jg.jacobi_syev_step(Ad, Qd, s, jg.params(b=b, ordering=ordering)) == 0
    Ag, Qg = _np(Ad), _np(Qd)
    assert np.array_equal(Ag, Ag.T)  # mirrored writes keep exact symmetry
    return Ag, Qg, A_or, Q_or, tab[s]


@pytest.mark.parametrize("np_,b,ordering,steps", STEP_CASES)
def test_step_parity_well_separated(jg, np_, b, ordering, steps):
    """Pivots with well separated eigenvalues (A = diag(1..2np) + 0.05 G):
    the step is well conditioned, so GPU and oracle agree to rounding."""
    d = np.linspace(1.0, 2.0 * np_, np_)
    A0 = np.asfortranarray(np.diag(d) + 0.05 * gen.sym_gaussian(np_, 900 + np_ + b))
    for s in steps:
        Ag, Qg, A_or, Q_or, _ = _step_pair(jg, A0, b, ordering, s)
        scale = np.abs(A0).max()
        assert np.abs(Ag - A_or).max() <= 1e-13 * scale, np.abs(Ag - A_or).max() / scale
        assert np.abs(Qg - Q_or).max() <= 1e-13, np.abs(Qg - Q_or).max()


def pivot_vector_tol(A0, b, pairs):
    """Bound on the difference of two correctly rounded eigenvector bases of
    the step's pivots: 32 k u ||Ahat|| / gap, gap = the smallest eigenvalue
    gap of a pivot (LAPACK on the pivot, independent of both sides)."""
    cond = 1.0
    for (I, J) in pairs:
        idx = np.r_[I * b:(I + 1) * b, J * b:(J + 1) * b]
        ev = np.linalg.eigvalsh(A0[np.ix_(idx, idx)])
        gap = max(np.diff(ev).min(), 1e-300) if len(ev) > 1 else 1.0
        cond = max(cond, np.abs(ev).max() / gap)
    return 32 * (2 * b) * U * cond


@pytest.mark.parametrize("np_,b,ordering,steps", STEP_CASES)
def test_step_parity_random(jg, np_, b, ordering, steps):
    """Gaussian pivots: eigenvectors of a pivot with close eigenvalues are
    determined only to u ||Ahat|| / gap, so the tolerance is that bound."""
    A0 = gen.sym_gaussian(np_, 1000 + np_ + b)
    for s in steps:
        Ag, Qg, A_or, Q_or, pairs = _step_pair(jg, A0, b, ordering, s)
        tol_v = pivot_vector_tol(A0, b, pairs)
        nrm2 = np.linalg.norm(A0, 2)
        assert np.abs(Qg - Q_or).max() <= max(1e-13, tol_v), (np.abs(Qg - Q_or).max(), tol_v)
        assert np.abs(Ag - A_or).max() <= max(1e-13, 4 * tol_v) * nrm2


@pytest.mark.parametrize("cl", ["1", "2", "4", "8"])
@pytest.mark.parametrize("np_,b", [(256, 32), (512, 128), (384, 64)])
def test_step_parity_cluster_sizes(jg, monkeypatch, cl, np_, b):
    """The pivot solves with 1 CTA per pair and with clusters of 2, 4, 8 CTAs
    (distributed pivot in shared memory) give the oracle's step."""
    monkeypatch.setenv("JACOBI_PIVOT_CLUSTER", cl)
    d = np.linspace(1.0, 2.0 * np_, np_)
    A0 = np.asfortranarray(np.diag(d) + 0.05 * gen.sym_gaussian(np_, 930 + np_ + b))
    for s in (0, 2):
        Ag, Qg, A_or, Q_or, _ = _step_pair(jg, A0, b, 0, s)
        assert np.abs(Ag - A_or).max() <= 1e-13 * np.abs(A0).max()
        assert np.abs(Qg - Q_or).max() <= 1e-13


@pytest.mark.parametrize("cl", ["1", "4"])
def test_full_solve_cluster_sizes(jg, monkeypatch, cl):
    monkeypatch.setenv("JACOBI_PIVOT_CLUSTER", cl)
    A, lam = gen.sym_known(512, "uniform", seed=1960)
    w, Q, _, st = jg.syev(A, b=64)
    assert st.status == 0
    check(A, _np(w), _np(Q), np.sort(lam))


def test_step_without_permutation(jg):
    """pivot_order = 0 (eigenpairs as solved, the paper's pseudocode)."""
    np_, b = 96, 16
    d = np.linspace(1.0, 2.0 * np_, np_)
    A0 = np.asfortranarray(np.diag(d) + 0.05 * gen.sym_gaussian(np_, 1900))
    tab = oracle.ordering(0, np_ // b)
    A_or, Q_or, _ = oracle.syev_step(A0, np.eye(np_), b, tab[2], pivot_order=0)
    Ad, Qd = _dev(A0), _dev(np.eye(np_))
    assert jg.jacobi_syev_step(Ad, Qd, 2, jg.params(b=b, pivot_order=0)) == 0
    assert np.abs(_np(Ad) - A_or).max() <= 1e-13 * np.abs(A0).max()
    assert np.abs(_np(Qd) - Q_or).max() <= 1e-13


# ------------------------------------------------------------------ full solves
def test_config1_n256_b16(jg):
    """n = 256, b = 16, lambda ~ U[-1,1], round-robin, off(A) <= 1e-14 ||A||_F."""
    A, lam = gen.sym_known(256, "uniform", seed=gen.SEEDS["c1"])
    w_or, Q_or, _, st_or, s_or = oracle.syev(A, b=16)
    w, Q, D, st = jg.syev(A, b=16)
    w, Q, D = _np(w), _np(Q), _np(D)
    assert st.status == 0 and s_or == 0
    check(A, w, Q, w_or)
    assert np.abs(w - np.sort(lam)).max() <= 1e-13 * np.abs(lam).max()
    assert abs(st.sweeps - st_or.sweeps) <= 1
    assert st.off_final <= 1e-14 * st.norm_fro or st.stalled
    # on exit (D, Q) is a consistent state: A = Q D Q^T, diag(D) = w
    assert np.array_equal(np.diag(D), w)
    assert np.abs(Q @ D @ Q.T - A).max() <= 1e-13 * np.abs(A).max() * 16


@pytest.mark.parametrize("n,b,ordering", [
    (200, 16, 0), (77, 8, 0), (130, 64, 0), (300, 128, 0), (50, 5, 0), (20, 1, 0),
    (100, 8, 1), (99, 7, 1), (33, 64, 0),
])
def test_ragged_and_orderings(jg, n, b, ordering):
    A = gen.sym_gaussian(n, 2000 + n)
    w_or, _, _, _, s_or = oracle.syev(A, b=b, ordering=ordering)
    w, Q, _, st = jg.syev(A, b=b, ordering=ordering)
    assert st.status == 0 and s_or == 0
    check(A, _np(w), _np(Q), w_or)


def test_full_solve_without_permutation(jg):
    A, lam = gen.sym_known(192, "uniform", seed=1950)
    w_or, *_ , s_or = oracle.syev(A, b=16, pivot_order=0)
    w, Q, _, st = jg.syev(A, b=16, pivot_order=0)
    assert st.status == 0 and s_or == 0
    check(A, _np(w), _np(Q), w_or)


def test_graded_spectrum_absolute_and_relative(jg):
    """lambda_i = +-10^(-12 i/(n-1)); gate absolute 1e-13 ||A||_2 everywhere and
    relative 1e-12 for |lambda| >= 1e-3 ||A||_2 (the stored entries do not fix
    smaller eigenvalues to relative accuracy)."""
    A, lam = gen.sym_known(256, "graded", seed=gen.SEEDS["c2g"])
    w_or, *_ = oracle.syev(A, b=16)
    w, Q, _, st = jg.syev(A, b=16)
    w, Q = _np(w), _np(Q)
    check(A, w, Q, w_or)
    big = np.abs(w_or) >= 1e-3 * np.abs(w_or).max()
    assert (np.abs(w - w_or)[big] / np.abs(w_or[big])).max() <= 1e-12


def test_graded_dhd_relative_criterion(jg):
    """A = D H D, kappa(H) <= 10: with the relative stop criterion every
    eigenvalue agrees with the oracle to 1e-12 relative."""
    A, d, H = gen.graded_dhd(128, seed=gen.SEEDS["c2dhd"])
    w_or, *_ = oracle.syev(A, b=16, conv=oracle.CONV_REL, tol=4 * U)
    w, Q, _, st = jg.syev(A, b=16, conv=jg.CONV_REL, tol=4 * U)
    w = _np(w)
    assert st.status == 0
    assert (np.abs(w - w_or) / np.abs(w_or)).max() <= 1e-12


# ------------------------------------------------------------------ edge cases
def test_clustered_eigenvalues_invariant_subspace(jg):
    """Five eigenvalues within 1e-12 of each other (gap 0.5 to the rest): the
    eigenvalues and the cluster's invariant subspace (its projector, which
    is unique where the vectors are not) against the constructed ones."""
    n, m = 200, 5
    r = gen.rng(3800)
    Qt = gen.haar_q(n, n, r)
    lam = np.concatenate([1.0 + 1e-12 * np.arange(m), r.uniform(-1.0, 0.5, n - m)])
    A = (Qt * lam[None, :]) @ Qt.T
    A = np.asfortranarray(0.5 * (A + A.T))
    w, Q, _, st = jg.syev(A, b=16)
    w, Q = _np(w), _np(Q)
    assert st.status == 0
    check(A, w, Q, np.sort(lam))
    P = Q[:, -m:] @ Q[:, -m:].T
    assert np.linalg.norm(P - Qt[:, :m] @ Qt[:, :m].T, 2) <= 1e-12


def test_diagonal_input_no_rotation(jg):
    d = np.linspace(-2, 3, 40)
    w, Q, D, st = jg.syev(np.diag(d), b=8)
    assert st.status == 0 and st.sweeps == 0 and st.rotations == 0
    assert np.array_equal(_np(w), d) and np.array_equal(_np(Q), np.eye(40))


def test_tiny_orders(jg):
    for n in (1, 2, 3):
        A = gen.sym_gaussian(n, 3000 + n)
        w, Q, _, st = jg.syev(A, b=1)
        check(A, _np(w), _np(Q), np.linalg.eigvalsh(A))
    w, Q, _, st = jg.syev(np.array([[5.0]]), b=4)
    assert _np(w)[0] == 5.0 and _np(Q)[0, 0] == 1.0


def test_zero_and_identity(jg):
    w, Q, _, st = jg.syev(np.zeros((24, 24)), b=4)
    assert st.status == 0 and np.all(_np(w) == 0)
    w, Q, _, st = jg.syev(np.eye(24) * 3.0, b=4)
    assert np.all(_np(w) == 3.0) and np.array_equal(_np(Q), np.eye(24))


def test_nonfinite_and_bad_arguments(jg):
    import torch
    A = gen.sym_gaussian(16, 3100)
    A[5, 2] = np.nan
    Ad = _dev(A)
    w = torch.empty(16, dtype=torch.float64, device="cuda")
    Q = jg.colmajor_empty(16, 16, torch.float64, "cuda")
    rc, _ = jg.jacobi_syev(Ad, w, Q, jg.params(b=4))
    assert rc == jg.ERR_NONFINITE
    A[5, 2] = 0.0
    A[2, 5] = np.inf  # upper triangle is not read
    rc, _ = jg.jacobi_syev(_dev(A), w, Q, jg.params(b=4))
    assert rc == 0
    assert jg.jacobi_syev(_dev(A), w, Q, jg.params(b=0))[0] == -7
    assert jg.jacobi_syev(_dev(A), w, Q, jg.params(b=129))[0] == jg.ERR_UNSUPPORTED
    assert jg.jacobi_syev(_dev(A), w, Q, jg.params(ordering=5))[0] == -7


def test_workspace_fault_injection_leaves_the_context_usable(jg, monkeypatch):
    """A workspace cap (JACOBI_WORKSPACE_LIMIT, host-side fault injection)
    makes the call return JACOBI_ERR_ALLOC before any launch, with the
    caller's buffers untouched; the next call without the cap succeeds."""
    import torch
    A, lam = gen.sym_known(64, "uniform", seed=3900)
    Ad = _dev(A)
    A0 = Ad.clone()
    w = torch.full((64,), 7.0, dtype=torch.float64, device="cuda")
    Q = jg.colmajor_empty(64, 64, torch.float64, "cuda")
    monkeypatch.setenv("JACOBI_WORKSPACE_LIMIT", "4096")
    rc, st = jg.jacobi_syev(Ad, w, Q, jg.params(b=16))
    assert rc == jg.ERR_ALLOC and st.status == rc
    assert torch.equal(Ad, A0) and bool((w == 7.0).all())
    monkeypatch.delenv("JACOBI_WORKSPACE_LIMIT")
    rc, st = jg.jacobi_syev(Ad, w, Q, jg.params(b=16))
    assert rc == 0
    check(A, _np(w), _np(Q), np.sort(lam))


def test_leading_dimension_and_no_vectors(jg):
    import torch
    n, ld = 50, 64
    A = gen.sym_gaussian(n, 3200)
    big = torch.zeros((n, ld), dtype=torch.float64, device="cuda").t()  # ld x n storage
    Ad = big[:n, :]
    Ad.copy_(torch.from_numpy(A))
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    rc, st = jg.jacobi_syev(Ad, w, None, jg.params(b=8, want_vectors=0))
    assert rc == 0
    check(A, _np(w), None, np.linalg.eigvalsh(A))
    assert torch.all(big[n:, :] == 0)  # rows past n untouched


def test_max_sweeps_reports_nonconvergence(jg):
    A = gen.sym_gaussian(64, 3300)
    w, Q, _, st = jg.syev(A, b=8, max_sweeps=1)
    assert st.status == 1 and st.sweeps == 1


def test_deterministic(jg):
    A = gen.sym_gaussian(160, 3400)
    w1, Q1, _, _ = jg.syev(A, b=16)
    w2, Q2, _, _ = jg.syev(A, b=16)
    assert np.array_equal(_np(w1), _np(w2)) and np.array_equal(_np(Q1), _np(Q2))


def test_warm_start_resume(jg):
    import torch
    A, lam = gen.sym_known(128, "uniform", seed=3500)
    w, Q, D, st = jg.syev(A, b=16, max_sweeps=2)
    assert st.status == 2
    w2 = torch.empty_like(w)
    rc, st2 = jg.jacobi_syev(D, w2, Q, jg.params(b=16, warm_start=1))
    assert rc == 0
    check(A, _np(w2), _np(Q), np.sort(lam))


def test_host_buffers_match_device(jg):
    import torch
    A = gen.sym_gaussian(96, 3600)
    w, Q, _, _ = jg.syev(A, b=16)
    Ah = jg.colmajor(A, dtype=torch.float64).pin_memory()
    wh = torch.empty(96, dtype=torch.float64).pin_memory()
    Qh = jg.colmajor_empty(96, 96, torch.float64, "cpu")
    rc, st = jg.jacobi_syev_h(Ah, wh, Qh, jg.params(b=16))
    assert rc == 0
    assert np.array_equal(wh.numpy(), _np(w)) and np.array_equal(Qh.numpy(), _np(Q))


def test_fp32_storage_is_the_fp64_solve_rounded_once(jg):
    """jacobi_syev_f32: the FP32 matrix widened exactly, solved by the FP64
    path, D, w and Q rounded once, i.e. bitwise the FP64 call on the widened
    matrix rounded to FP32 (the FP64 path is deterministic).  Padding rows
    of the leading dimensions hold NaN: they are neither read nor written."""
    import torch
    n = 150
    A, lam = gen.sym_known(n, "uniform", seed=3700)
    A32 = A.astype(np.float32)
    Ad = _dev(A32.astype(np.float64))
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    Q = jg.colmajor_empty(n, n, torch.float64, "cuda")
    rc, st = jg.jacobi_syev(Ad, w, Q, jg.params(b=16))
    assert rc == 0
    Ap = jg.colmajor_empty(n + 5, n, torch.float32, "cuda").fill_(float("nan"))
    Qp = jg.colmajor_empty(n + 3, n, torch.float32, "cuda").fill_(float("nan"))
    A32d, Q32 = Ap[:n], Qp[:n]
    A32d.copy_(torch.from_numpy(A32))
    w32 = torch.empty(n, dtype=torch.float32, device="cuda")
    rc32, st32 = jg.jacobi_syev_f32(A32d, w32, Q32, jg.params(b=16))
    assert rc32 == 0 and st32.status == 0 and st32.sweeps == st.sweeps
    assert torch.equal(w32, w.float()) and torch.equal(Q32, Q.float()) and torch.equal(A32d, Ad.float())
    assert torch.isnan(Ap[n:]).all() and torch.isnan(Qp[n:]).all()
    check(A32.astype(np.float64), _np(w32).astype(np.float64), _np(Q32).astype(np.float64),
          np.sort(lam), eig=1e-6, res=1e-5, orth=1e-6)
    # eigenvalues only
    w32b = torch.empty(n, dtype=torch.float32, device="cuda")
    B = jg.colmajor(A32, device="cuda", dtype=torch.float32)
    rc, _ = jg.jacobi_syev_f32(B, w32b, None, jg.params(b=16, want_vectors=0))
    assert rc == 0 and torch.allclose(w32b, w32, rtol=0, atol=1e-6)
    # a non-finite entry: the error code, the caller's buffers untouched
    A32[7, 3] = np.inf
    C32 = jg.colmajor(A32, device="cuda", dtype=torch.float32)
    C0 = C32.clone()
    w0 = torch.full((n,), 5.0, dtype=torch.float32, device="cuda")
    rc, st = jg.jacobi_syev_f32(C32, w0, Q32, jg.params(b=16))
    assert rc == jg.ERR_NONFINITE and st.status == rc
    assert torch.equal(C32.isinf(), C0.isinf()) and torch.equal(C32.nan_to_num(), C0.nan_to_num())
    assert (w0 == 5.0).all()
    with pytest.raises(TypeError):
        jg.jacobi_syev_f32(Ad, w, Q, jg.params(b=16))


# ------------------------------------------------------------------ full size (n = 4096, b = 64)
def test_full_size_n4096_b64(jg):
    """The benchmark workload: first step element-wise against the oracle at
    full size, then the converged solve against the constructed spectrum and
    the residual / orthogonality bounds."""
    n, b = 4096, 64
    A, lam = gen.sym_known(n, "uniform", seed=gen.SEEDS["c2u"])
    tab = oracle.ordering(oracle.ORDER_ROUND_ROBIN, n // b)
    A_or, _, _ = oracle.syev_step(A, None, b, tab[0])
    Ad = _dev(A)
    assert jg.jacobi_syev_step(Ad, None, 0, jg.params(b=b)) == 0
    tol_v = pivot_vector_tol(A, b, tab[0])
    assert np.abs(_np(Ad) - A_or).max() <= max(1e-13, 4 * tol_v) * np.abs(lam).max()
    del Ad
    w, Q, _, st = jg.syev(A, b=b)
    w, Q = _np(w), _np(Q)
    assert st.status == 0
    check(A, w, Q, np.sort(lam))


@pytest.mark.parametrize("np_,b,cl", [(256, 32, "2"), (512, 64, "4"), (1024, 128, "4"), (768, 64, "8")])
def test_pivot_schedules_agree_bit_for_bit(jg, monkeypatch, np_, b, cl):
    """The cluster pivot kernel's fused schedule (one barrier per round; each
    rotation chosen once per cluster by the thread that rotates the quad
    holding its pivot entry) and its split schedule (JACOBI_PIVOT_SCHEDULE=
    split) run the same operations on the same values: the steps, and a
    full solve with several inner sweeps, agree bit for bit."""
    import torch
    monkeypatch.setenv("JACOBI_PIVOT_CLUSTER", cl)
    A0 = gen.sym_gaussian(np_, 5500 + np_)
    out = {}
    for sched in ("split", "fused"):
        monkeypatch.setenv("JACOBI_PIVOT_SCHEDULE", sched)
        Ad, Qd = _dev(A0), _dev(np.eye(np_))
        for s in (0, 1):
            assert jg.jacobi_syev_step(Ad, Qd, s, jg.params(b=b, inner_max_sweeps=3)) == 0
        w, Q, D, st = jg.syev(A0, b=b, inner_max_sweeps=2)
        assert st.status == 0
        out[sched] = (_np(Ad), _np(Qd), _np(w), _np(Q), st.rotations, st.inner_sweeps)
    a, f = out["split"], out["fused"]
    for x, y in zip(a, f):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("np_,b,cl", [(512, 64, "1"), (512, 64, "4"), (1024, 128, "4"), (768, 64, "8")])
def test_fp32_transform_schedules_agree_bit_for_bit(jg, monkeypatch, np_, b, cl):
    """The low-precision step accumulates each pivot's V in FP32: the split
    and fused cluster schedules still agree bit for bit (cluster size 1 runs
    the one-CTA kernel; its accuracy, like the others', is held to the
    oracle's step by the mixed-form tests)."""
    import torch
    monkeypatch.setenv("JACOBI_PIVOT_CLUSTER", cl)
    A32 = np.asfortranarray(gen.sym_gaussian(np_, 5600 + np_).astype(np.float32))
    out = {}
    for sched in ("split", "fused"):
        monkeypatch.setenv("JACOBI_PIVOT_SCHEDULE", sched)
        Ad = jg.colmajor(A32, device="cuda", dtype=torch.float32)
        Qd = jg.colmajor(np.eye(np_, dtype=np.float32), device="cuda", dtype=torch.float32)
        for s in (0, 1):
            assert jg.jacobi_syev_step_lowp(Ad, Qd, s, jg.params(b=b, precision=2)) == 0
        out[sched] = (_np(Ad), _np(Qd))
    for x, y in zip(out["split"], out["fused"]):
        assert np.array_equal(x, y)
