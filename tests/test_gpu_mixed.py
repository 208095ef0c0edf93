"""GPU parity of the mixed-precision form.

One low-precision step (FP64 pivot solves on the promoted FP32 pivots, block
updates on the tensor cores from bf16 hi/lo splits) against the oracle's FP64
step on the same FP32 input, element-wise within the bound of the split
product: every product loses at most the lo*lo term (2^-18 relative per
operand pair), two products per A entry, FP32 accumulation over k terms:
(2^-15 + 4 k u32) (|V|^T |A| |V|).  In these sweeps the pivot accumulates V
in FP32 (the products take it rounded to FP32 anyway): each of its k - 1
rounds rotates a row's entry pair (x, y), of norm <= 1, with s and tau
rounded to FP32 and two FP32 fma roundings, an error of at most 6 u32
(later exact rotations carry it without growth), so |E| <= 6 k u32 entry-wise
inside each pair's k x k block (mask B) and A' gains
6 k u32 (B |A| |V| + |V|^T |A| B), Q' gains 6 k u32 |Q| B.

Full mixed solves are held to ten times the FP64 gates (eigenvalues,
residual, orthogonality), against the constructed spectrum and the oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

import jacobi_inputs as gen
import oracle

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
MIXED = 2
MIXED_F16 = 3
MIXED_TF32 = 4


@pytest.fixture(scope="module")
def jg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_28952_gb300 as m
    m.lib()
    return m


def _np(t):
    return t.detach().cpu().numpy()


def check(A, w, Q, w_ref, eig=1e-12, res=1e-11, orth=1e-12):
    n = A.shape[0]
    nrm2 = max(np.abs(w_ref).max(), 1e-300)
    assert np.abs(w - w_ref).max() <= eig * nrm2, np.abs(w - w_ref).max() / nrm2
    if Q is not None:
        r = np.linalg.norm(A @ Q - Q * w[None, :])
        assert r <= res * max(np.linalg.norm(A), 1e-300), r / np.linalg.norm(A)
        o = np.linalg.norm(Q.T @ Q - np.eye(n))
        assert o <= orth * n, o / n


# ------------------------------------------------------------------ one low-precision step
LOWP_CASES = [
    (256, 32, 0, [0, 3]),     # k = 64: one ragged 128-tile
    (512, 64, 0, [0, 5]),     # k = 128: exactly one tile
    (768, 128, 0, [0]),       # k = 256: 2 x 2 tiles, pivots in clusters / global scratch
    (80, 8, 1, [0, 1]),       # Algorithm 3 with a frozen entry
    (40, 5, 0, [0, 2]),       # odd b
    (4, 1, 0, [1]),           # b = 1
]


@pytest.mark.parametrize("prec", [MIXED, MIXED_F16, MIXED_TF32])
@pytest.mark.parametrize("np_,b,ordering,steps", LOWP_CASES)
def test_lowp_step_matches_oracle_within_split_bound(jg, np_, b, ordering, steps, prec):
    import torch
    d = np.linspace(1.0, 2.0 * np_, np_)
    A32 = (np.diag(d) + 0.05 * gen.sym_gaussian(np_, 4000 + np_ + b)).astype(np.float32)
    A32 = np.asfortranarray(A32)
    Q32 = gen.haar_q(np_, np_, gen.rng(4100, np_)).astype(np.float32)
    A64, Q64 = A32.astype(np.float64), Q32.astype(np.float64)
    tab = oracle.ordering(ordering, np_ // b)
    k = 2 * b
    for s in steps:
        A_or, Q_or, _ = oracle.syev_step(A64, Q64, b, tab[s])
        # the step's transform (block-diagonal over the pairs, with the sort)
        V = np.linalg.solve(Q64, Q_or) if np_ <= 1024 else None
        Ad = jg.colmajor(A32, device="cuda", dtype=torch.float32)
        Qd = jg.colmajor(Q32, device="cuda", dtype=torch.float32)
        rc = jg.jacobi_syev_step_lowp(Ad, Qd, s, jg.params(b=b, ordering=ordering, precision=prec))
        assert rc == 0
        Ag, Qg = _np(Ad).astype(np.float64), _np(Qd).astype(np.float64)
        assert np.array_equal(Ag, Ag.T)
        aV = np.abs(V)
        B = np.zeros((np_, np_))   # 1 inside each pair's k x k block
        for I, J in tab[s]:
            idx = np.r_[I * b:(I + 1) * b, J * b:(J + 1) * b]
            B[np.ix_(idx, idx)] = 1.0
        AV = np.abs(A64) @ aV
        vacc = 6 * k * U32 * (B @ AV + AV.T @ B)
        c = 2.0 ** -15 + 4 * k * U32
        boundA = c * (aV.T @ np.abs(A64) @ aV) + vacc + 1e-30
        boundQ = c * (np.abs(Q64) @ aV) + 6 * k * U32 * (np.abs(Q64) @ B) + 1e-30
        if prec == MIXED_F16:
            # fp16 splits: 22 bits in the normal range; entries of V and Q
            # below it (|x| < 2^-14) keep an absolute error of at most 2^-25
            c16 = 2.0 ** -20 + 4 * k * U32
            boundA = (c16 * (aV.T @ np.abs(A64) @ aV) + 2.0 ** -24 * (np.abs(A64) @ np.ones_like(aV)).max()
                      + vacc + 1e-30)
            boundQ = c16 * (np.abs(Q64) @ aV) + 2.0 ** -24 * k + 6 * k * U32 * (np.abs(Q64) @ B) + 1e-30
        ra = np.abs(Ag - A_or) / boundA
        rq = np.abs(Qg - Q_or) / boundQ
        assert ra.max() <= 1.0, ra.max()
        assert rq.max() <= 1.0, rq.max()


def test_lowp_step_without_q_and_arguments(jg):
    import torch
    np_, b = 128, 16
    A32 = np.asfortranarray(gen.sym_gaussian(np_, 4200).astype(np.float32))
    Ad = jg.colmajor(A32, device="cuda", dtype=torch.float32)
    assert jg.jacobi_syev_step_lowp(Ad, None, 1, jg.params(b=b, precision=MIXED)) == 0
    A_or, _, _ = oracle.syev_step(A32.astype(np.float64), None, b, oracle.ordering(0, np_ // b)[1])
    assert np.abs(_np(Ad) - A_or).max() <= 1e-4 * np.abs(A32).max()
    # FP64 precision is not a low-precision step; bad sizes and steps are rejected
    assert jg.jacobi_syev_step_lowp(Ad, None, 0, jg.params(b=b)) == jg.ERR_UNSUPPORTED
    assert jg.jacobi_syev_step_lowp(Ad, None, 99, jg.params(b=b, precision=MIXED)) == -7
    assert jg.jacobi_syev_step_lowp(Ad, None, 0, jg.params(b=48, precision=MIXED)) == -1


# ------------------------------------------------------------------ full mixed solves
@pytest.mark.parametrize("prec", [MIXED, MIXED_F16, MIXED_TF32])
@pytest.mark.parametrize("n,b", [(256, 32), (300, 32), (512, 64), (1024, 128)])
def test_mixed_solve_uniform_spectrum(jg, n, b, prec):
    A, lam = gen.sym_known(n, "uniform", seed=4300 + n)
    w, Q, _, st = jg.syev(A, b=b, precision=prec)
    assert st.status == 0
    assert st.sweeps_lowp >= 1 and st.flops_lowp > 0
    check(A, _np(w), _np(Q), np.sort(lam))


def test_mixed_matches_oracle_eigenvalues(jg):
    A = gen.sym_gaussian(192, 4400)
    w_or, *_ = oracle.syev(A, b=16)
    w, Q, _, st = jg.syev(A, b=16, precision=MIXED)
    assert st.status == 0
    check(A, _np(w), _np(Q), w_or)


@pytest.mark.parametrize("prec", [MIXED, MIXED_F16, MIXED_TF32])
def test_mixed_graded_spectrum(jg, prec):
    A, lam = gen.sym_known(256, "graded", seed=gen.SEEDS["c2g"])
    w_or, *_ = oracle.syev(A, b=32)
    w, Q, _, st = jg.syev(A, b=32, precision=prec)
    assert st.status == 0
    check(A, _np(w), _np(Q), w_or)


@pytest.mark.parametrize("refine", [0, 1, 2])
def test_mixed_refinement_steps(jg, refine):
    A, lam = gen.sym_known(384, "uniform", seed=4500)
    w, Q, _, st = jg.syev(A, b=64, precision=MIXED, refine_steps=refine)
    assert st.status == 0
    check(A, _np(w), _np(Q), np.sort(lam))


def test_mixed_clustered_eigenvalues(jg):
    """Pairs of equal eigenvalues: the refinement cannot separate them (its
    correction is left out for such pairs); the FP64 closing sweeps do."""
    n = 256
    lam = np.repeat(np.linspace(-1, 1, n // 2), 2)
    Qh = gen.haar_q(n, n, gen.rng(4600))
    A = np.asfortranarray((Qh * lam) @ Qh.T)
    A = 0.5 * (A + A.T)
    w, Q, _, st = jg.syev(A, b=32, precision=MIXED)
    assert st.status == 0
    check(A, _np(w), _np(Q), np.sort(lam))


def test_mixed_edge_cases(jg):
    # already diagonal: no sweep of either kind
    d = np.linspace(-2, 3, 64)
    w, Q, _, st = jg.syev(np.diag(d), b=16, precision=MIXED)
    assert st.status == 0 and st.sweeps == 0
    assert np.array_equal(_np(w), d) and np.array_equal(_np(Q), np.eye(64))
    # tiny order
    A = gen.sym_gaussian(3, 4700)
    w, Q, _, st = jg.syev(A, b=1, precision=MIXED)
    check(A, _np(w), _np(Q), np.linalg.eigvalsh(A))
    # non-finite input
    import torch
    A = gen.sym_gaussian(32, 4800)
    A[7, 3] = np.inf
    w = torch.empty(32, dtype=torch.float64, device="cuda")
    Qd = jg.colmajor_empty(32, 32, torch.float64, "cuda")
    Ad = jg.colmajor(A, device="cuda", dtype=torch.float64)
    rc, _ = jg.jacobi_syev(Ad, w, Qd, jg.params(b=8, precision=MIXED))
    assert rc == jg.ERR_NONFINITE
    # warm start is not offered with the mixed form; precision codes past FP64_EMU are rejected
    A[7, 3] = 0.0
    Ad = jg.colmajor(A, device="cuda", dtype=torch.float64)
    assert jg.jacobi_syev(Ad, w, Qd, jg.params(b=8, precision=MIXED, warm_start=1))[0] == jg.ERR_UNSUPPORTED
    assert jg.jacobi_syev(Ad, w, Qd, jg.params(b=8, precision=6))[0] == -7


def test_mixed_deterministic(jg):
    A, _ = gen.sym_known(256, "uniform", seed=4900)
    w1, Q1, _, _ = jg.syev(A, b=32, precision=MIXED)
    w2, Q2, _, _ = jg.syev(A, b=32, precision=MIXED)
    assert np.array_equal(_np(w1), _np(w2)) and np.array_equal(_np(Q1), _np(Q2))


@pytest.mark.parametrize("prec", [MIXED, MIXED_F16, MIXED_TF32])
def test_mixed_n4096_b64(jg, prec):
    """The benchmark's mixed workload size class: against the constructed
    spectrum, with fewer FP64 sweeps than the plain FP64 solve needs."""
    n, b = 4096, 64
    A, lam = gen.sym_known(n, "uniform", seed=gen.SEEDS["c2u"])
    w, Q, _, st = jg.syev(A, b=b, precision=prec)
    assert st.status == 0
    check(A, _np(w), _np(Q), np.sort(lam))
    assert st.sweeps - st.sweeps_lowp <= 4
