"""FP64-accurate products on the bf16 tensor cores (slicing; jacobi_f64emu_gemm)
against the exact product.  The model: every row of op(A) and column of B is
written as 2^{E-7} sum_p slice_p with eight 7-bit integer slices, and the
slice products of total significance p + q <= 9 are summed exactly.  Per
term of the dot product, rounding each operand to 56 fraction bits costs
< 2^{E+F-56} and the dropped products p + q >= 10 (balanced digits of at
most 64, weights 2^{-7(p+q-2)}) < 2^{E+F-56}, and the combination of the
accumulators rounds the three lowest levels to 2^{E+F-49} (half of it at
most); the bound per entry is taken as (9.1 K + 64) 2^-56 2^{E_m + F_n} with
2^{E_m} > max|op(A)(m, :)| and 2^{F_n} > max|B(:, n)|, the size of FP64
rounding (K 2^-53 |op(A)| |B|) for K >= 8."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_28952_gb300 as m
    m.lib()
    return m


def _pow2_above(x):
    m = np.abs(x).max()
    return 2.0 ** (np.floor(np.log2(m)) + 1) if m > 0 else 1.0


def _exact(A, B):
    # the product to well below FP64 rounding: long double where the platform
    # has it (x86), else FP64 (the bound's FP64 term covers it)
    if np.finfo(np.longdouble).eps < 1e-17:
        return (A.astype(np.longdouble) @ B.astype(np.longdouble)).astype(np.float64)
    return A @ B


@pytest.mark.parametrize("M,N,K,trans", [(128, 64, 32, False), (128, 64, 256, False), (300, 200, 128, False),
                                          (256, 130, 77, True), (1, 5, 3, False), (129, 65, 200, True),
                                          # K > 256: exact FP32 accumulation per 256 K, 64-bit running sums
                                          (128, 64, 300, False), (200, 130, 1000, True), (128, 64, 4096, False),
                                          (64, 40, 9000, True)])
def test_emu_gemm_is_fp64_accurate(jg, M, N, K, trans):
    import torch
    r = np.random.default_rng(M * 7 + N + K)
    A = r.standard_normal((K, M) if trans else (M, K))
    B = r.standard_normal((K, N))
    # graded rows and columns: the scaling is per row / column
    A *= (10.0 ** r.uniform(-8, 8, A.shape[1] if trans else A.shape[0]))[None, :] if trans else \
        (10.0 ** r.uniform(-8, 8, A.shape[0]))[:, None]
    B *= (10.0 ** r.uniform(-8, 8, N))[None, :]
    Ad = jg.colmajor(A, device="cuda", dtype=torch.float64)
    Bd = jg.colmajor(B, device="cuda", dtype=torch.float64)
    Cd = jg.colmajor_empty(M, N, torch.float64, "cuda")
    assert jg.jacobi_f64emu_gemm(Ad, Bd, Cd, transA=trans) == 0
    C = Cd.cpu().numpy()
    Aop = A.T if trans else A
    want = _exact(Aop, B)
    rs = np.array([_pow2_above(Aop[i]) for i in range(M)])
    cs = np.array([_pow2_above(B[:, j]) for j in range(N)])
    bound = (9.1 * K + 64) * 2.0 ** -56 * rs[:, None] * cs[None, :] + 4 * 2.0 ** -53 * np.abs(want)
    assert np.all(np.abs(C - want) <= bound), np.max(np.abs(C - want) / bound)


def test_emu_gemm_special_values(jg):
    import torch
    M, N, K = 64, 64, 16
    A = np.zeros((M, K))
    A[3, :] = 2.0 ** -1000 * np.arange(1, K + 1)   # tiny entries keep their row's own scale
    A[4, :] = (-1.0) ** np.arange(K) * 2.0 ** np.arange(K)   # signs and a 2^15 range in one row
    A[5, 7] = -2.0 ** 60
    B = np.eye(K, N)
    B[2, 9] = 3.0
    Ad = jg.colmajor(A, device="cuda", dtype=torch.float64)
    Bd = jg.colmajor(B, device="cuda", dtype=torch.float64)
    Cd = jg.colmajor_empty(M, N, torch.float64, "cuda")
    assert jg.jacobi_f64emu_gemm(Ad, Bd, Cd) == 0
    C = Cd.cpu().numpy()
    assert np.array_equal(C, A @ B)          # integers and powers of two are exact
    # the same across exact accumulations (K > 256): integer entries stay exact
    K2 = 700
    A2 = np.zeros((M, K2))
    A2[:, ::7] = np.arange(1, M + 1)[:, None]
    B2 = np.zeros((K2, 4))
    B2[::5, :] = -3.0
    Cd2 = jg.colmajor_empty(M, 4, torch.float64, "cuda")
    assert jg.jacobi_f64emu_gemm(jg.colmajor(A2, device="cuda", dtype=torch.float64),
                                 jg.colmajor(B2, device="cuda", dtype=torch.float64), Cd2) == 0
    assert np.array_equal(Cd2.cpu().numpy(), A2 @ B2)


# ------------------------------------------------------------------ the FP64 method with emulated products
import jacobi_inputs as gen  # noqa: E402
import oracle  # noqa: E402

EMU = 5


@pytest.mark.parametrize("np_,b,ordering,steps", [
    (256, 64, 0, [0, 1]), (512, 128, 0, [0]), (96, 16, 0, [0, 4]), (40, 5, 0, [0, 2]), (80, 8, 1, [0, 1]),
])
def test_emu_step_matches_oracle(jg, np_, b, ordering, steps):
    """One parallel step with the update products on the tensor cores gives
    the oracle's FP64 step to the same 1e-13 as the DFMA path (well
    separated pivots: a well-conditioned step)."""
    import torch
    d = np.linspace(1.0, 2.0 * np_, np_)
    A0 = np.asfortranarray(np.diag(d) + 0.05 * gen.sym_gaussian(np_, 5000 + np_ + b))
    tab = oracle.ordering(ordering, np_ // b)
    for s in steps:
        A_or, Q_or, _ = oracle.syev_step(A0, np.eye(np_), b, tab[s])
        Ad = jg.colmajor(A0, device="cuda", dtype=torch.float64)
        Qd = jg.colmajor(np.eye(np_), device="cuda", dtype=torch.float64)
        assert jg.jacobi_syev_step(Ad, Qd, s, jg.params(b=b, ordering=ordering, precision=EMU)) == 0
        Ag, Qg = Ad.cpu().numpy(), Qd.cpu().numpy()
        assert np.array_equal(Ag, Ag.T)
        assert np.abs(Ag - A_or).max() <= 1e-13 * np.abs(A0).max(), np.abs(Ag - A_or).max() / np.abs(A0).max()
        assert np.abs(Qg - Q_or).max() <= 1e-13, np.abs(Qg - Q_or).max()


def _check(A, w, Q, w_ref, eig=1e-13, res=1e-12, orth=1e-13):
    n = A.shape[0]
    nrm2 = np.abs(w_ref).max()
    assert np.abs(w - w_ref).max() <= eig * nrm2, np.abs(w - w_ref).max() / nrm2
    assert np.linalg.norm(A @ Q - Q * w[None, :]) <= res * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= orth * n


@pytest.mark.parametrize("n,b,kind", [(512, 64, "uniform"), (1024, 64, "uniform"), (300, 32, "uniform"),
                                       (256, 32, "graded"), (512, 128, "uniform")])
def test_emu_full_solve_meets_the_fp64_gates(jg, n, b, kind):
    A, lam = gen.sym_known(n, kind, seed=5100 + n)
    w, Q, _, st = jg.syev(A, b=b, precision=EMU)
    assert st.status == 0
    _check(A, w.cpu().numpy(), Q.cpu().numpy(), np.sort(lam) if kind == "uniform" else oracle.syev(A, b=b)[0])


def test_emu_n4096_b64(jg):
    """The benchmark matrix: the FP64 gates against the constructed spectrum."""
    n, b = 4096, 64
    A, lam = gen.sym_known(n, "uniform", seed=gen.SEEDS["c2u"])
    w, Q, _, st = jg.syev(A, b=b, precision=EMU)
    assert st.status == 0
    _check(A, w.cpu().numpy(), Q.cpu().numpy(), np.sort(lam))


def test_fp64_products_flag_is_the_emulated_path(jg):
    """precision FP64 with fp64_products = 1 runs the same solve as FP64_EMU."""
    A, lam = gen.sym_known(384, "uniform", seed=5300)
    w1, Q1, _, s1 = jg.syev(A, b=32, precision=EMU)
    w2, Q2, _, s2 = jg.syev(A, b=32, precision=0, fp64_products=1)
    assert s1.status == 0 and s2.status == 0 and s1.sweeps == s2.sweeps
    assert np.array_equal(w1.cpu().numpy(), w2.cpu().numpy()) and np.array_equal(Q1.cpu().numpy(), Q2.cpu().numpy())


@pytest.mark.parametrize("prec", [2, 3, 4])
def test_mixed_with_emulated_fp64_products_meets_the_fp64_gates(jg, prec):
    """The mixed forms with the refinement products and the closing sweeps'
    updates on the tensor cores (fp64_products = 1): the FP64 gates."""
    n = 1024
    A, lam = gen.sym_known(n, "uniform", seed=5400 + prec)
    w, Q, _, st = jg.syev(A, b=64, precision=prec, fp64_products=1)
    assert st.status == 0 and st.sweeps_lowp > 0
    _check(A, w.cpu().numpy(), Q.cpu().numpy(), np.sort(lam))


# ------------------------------------------------------------------ the one-sided method with emulated products
@pytest.mark.parametrize("m,np_,b", [(300, 64, 8), (1100, 96, 16), (700, 256, 64), (40, 12, 3)])
def test_emu_svd_step_matches_oracle(jg, m, np_, b):
    """One one-sided step (Gram partials over 512-row panels and the column
    update on the tensor cores, FP64 pivots) gives the oracle's FP64 step to
    the DFMA path's tolerances."""
    import torch
    G0 = gen.tall_gaussian(m, np_, 5500 + m, dtype=np.float64)
    tol = oracle.svd_tol(m)
    tab = oracle.ordering(0, np_ // b)
    for s in (0, len(tab) - 1):
        G_or, V_or, r_or = oracle.gesvd_step(G0, np.eye(np_), b, tab[s], tol_rel=tol, inner_max=30)
        Gd = jg.colmajor(G0, device="cuda", dtype=torch.float64)
        Vd = jg.colmajor(np.eye(np_), device="cuda", dtype=torch.float64)
        rc, r = jg.jacobi_gesvd_step(Gd, Vd, s, jg.params(b=b, tol=1e-15, precision=EMU))
        assert rc == 0 and abs(r - r_or) <= 1e-13
        assert np.abs(Gd.cpu().numpy() - G_or).max() <= 1e-12 * np.abs(G0).max()
        assert np.abs(Vd.cpu().numpy() - V_or).max() <= 1e-12


@pytest.mark.parametrize("m,n,b,qr", [(500, 96, 16, 0), (1030, 130, 32, 1), (2048, 256, 64, 0), (2048, 256, 64, 1)])
def test_emu_svd_meets_the_fp64_gates(jg, m, n, b, qr):
    G, sig = gen.svd_known(m, n, seed=5600 + n, decades=10.0)
    U, s, V, st = jg.gesvd(G, b=b, precision=EMU, svd_qr=qr)
    U, s, V = U.cpu().numpy(), s.cpu().numpy(), V.cpu().numpy()
    assert st.status == 0
    assert np.abs(s - sig).max() <= 1e-13 * sig[0]
    big = sig >= 1e-3 * sig[0]
    assert (np.abs(s - sig)[big] / sig[big]).max() <= 1e-12
    assert np.linalg.norm(U.T @ U - np.eye(n)) <= 1e-12 * n
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-12 * n
    assert np.linalg.norm(G @ V - U * s[None, :]) <= 1e-13 * np.linalg.norm(G) * np.sqrt(n)


def test_svd_rejects_the_mixed_precisions(jg):
    import torch
    G = gen.tall_gaussian(64, 16, 5700, dtype=np.float64)
    s = torch.empty(16, dtype=torch.float64, device="cuda")
    assert jg.jacobi_gesvd(jg.colmajor(G, device="cuda", dtype=torch.float64), s, None,
                           jg.params(b=4, want_vectors=0, precision=2))[0] == jg.ERR_UNSUPPORTED


def test_emu_graded_dhd_relative_criterion(jg):
    """A = D H D (kappa(H) <= 10, eigenvalues over ~12 decades) with the
    relative stop criterion: every eigenvalue to 1e-12 relative, as on the
    FP64 path (the emulated products balance the pair-blocks' columns by
    powers of two taken from the diagonal)."""
    U = 2.0 ** -53
    A, d, H = gen.graded_dhd(128, seed=gen.SEEDS["c2dhd"])
    w_or, *_ = oracle.syev(A, b=16, conv=oracle.CONV_REL, tol=4 * U)
    w, Q, _, st = jg.syev(A, b=16, conv=jg.CONV_REL, tol=4 * U, precision=EMU)
    w = w.cpu().numpy()
    assert st.status == 0
    assert (np.abs(w - w_or) / np.abs(w_or)).max() <= 1e-12


def test_emu_graded_spectrum_relative_gate(jg):
    A, lam = gen.sym_known(512, "graded", seed=5800)
    w_or, *_ = oracle.syev(A, b=32)
    w, Q, _, st = jg.syev(A, b=32, precision=EMU)
    w = w.cpu().numpy()
    assert st.status == 0
    assert np.abs(w - w_or).max() <= 1e-13 * np.abs(w_or).max()
    big = np.abs(w_or) >= 1e-3 * np.abs(w_or).max()
    assert (np.abs(w - w_or)[big] / np.abs(w_or[big])).max() <= 1e-12


@pytest.mark.parametrize("n,b", [(512, 64), (1024, 128), (300, 50)])
def test_step_image_of_v_is_bitwise_the_per_tile_slicing(jg, monkeypatch, n, b):
    """The emulated update slices V once per step into digit images that its
    tiles stage by bulk copies (default), or slices V inside every tile
    (JACOBI_EMU_IMAGE=0): the same slices and scales, so the step and the
    full solve agree bit for bit."""
    import torch

    import jacobi_inputs as gen

    def _dev(x):
        return jg.colmajor(x, device="cuda", dtype=torch.float64)

    def _np(t):
        return t.detach().cpu().numpy()

    A0 = gen.sym_gaussian(n, 6100 + n)
    out = {}
    for img in ("1", "0"):
        monkeypatch.setenv("JACOBI_EMU_IMAGE", img)
        Ad, Qd = _dev(A0), _dev(np.eye(n))
        for s in (0, 1):
            assert jg.jacobi_syev_step(Ad, Qd, s, jg.params(b=b, precision=jg.PREC_FP64_EMU)) == 0
        w, Q, _, st = jg.syev(A0, b=b, precision=jg.PREC_FP64_EMU)
        assert st.status == 0
        out[img] = (_np(Ad), _np(Qd), _np(w), _np(Q))
    for x, y in zip(out["1"], out["0"]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("n,b", [(512, 64), (700, 64)])
def test_refinement_images_are_bitwise_the_per_tile_slicing(jg, monkeypatch, n, b):
    """The mixed form with FP64-accurate refinement products: with the
    products' operands sliced once into images (default) or sliced in every
    tile (JACOBI_EMU_IMAGE=0), the solve agrees bit for bit (ragged n: the
    images' padding rows are zero)."""
    import jacobi_inputs as gen
    A, lam = gen.sym_known(n, "uniform", seed=6200 + n)
    out = {}
    for img in ("1", "0"):
        monkeypatch.setenv("JACOBI_EMU_IMAGE", img)
        w, Q, _, st = jg.syev(A, b=b, precision=jg.PREC_MIXED_BF16X3, fp64_products=1)
        assert st.status == 0 and st.ms_refine > 0
        out[img] = (w.cpu().numpy(), Q.cpu().numpy())
    assert np.array_equal(out["1"][0], out["0"][0]) and np.array_equal(out["1"][1], out["0"][1])
    assert np.abs(out["1"][0] - np.sort(lam)).max() <= 1e-13 * np.abs(lam).max()
