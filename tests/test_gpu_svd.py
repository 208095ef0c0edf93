"""GPU parity of the one-sided blocked Jacobi SVD (Algorithm 6) against the
CPU oracle: element-wise single steps (Gram block, FP64 pivot solve, column
update), then full solves on what is unique (singular values; U and V through
orthogonality and the residual ||G V - U Sigma||)."""
from __future__ import annotations

import numpy as np
import pytest

import jacobi_inputs as gen
import oracle

pytestmark = pytest.mark.gpu


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


def check_svd(G, U, s, V, s_ref, abs_tol=1e-13, rel_tol=1e-12, v_orth=1e-13):
    n = G.shape[1]
    smax = s_ref[0]
    assert np.abs(s - s_ref).max() <= abs_tol * smax, np.abs(s - s_ref).max() / smax
    big = s_ref >= 1e-3 * smax
    assert (np.abs(s - s_ref)[big] / s_ref[big]).max() <= rel_tol
    nz = s > 0
    assert np.linalg.norm(U[:, nz].T @ U[:, nz] - np.eye(nz.sum())) <= 1e-12 * n
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= v_orth * n
    assert np.linalg.norm(G @ V - U * s[None, :]) <= 1e-13 * np.linalg.norm(G) * np.sqrt(n)


@pytest.mark.parametrize("m,np_,b,ordering", [
    (300, 64, 8, 0), (1100, 96, 16, 0), (600, 128, 32, 0), (700, 160, 40, 1), (40, 12, 3, 0),
])
def test_step_parity_elementwise(jg, m, np_, b, ordering):
    G0 = gen.tall_gaussian(m, np_, 4000 + m, dtype=np.float64)
    tol = oracle.svd_tol(m)
    tab = oracle.ordering(ordering, np_ // b)
    p = jg.params(b=b, ordering=ordering, tol=1e-15)
    for s in (0, len(tab) - 1):
        G_or, V_or, r_or = oracle.gesvd_step(G0, np.eye(np_), b, tab[s], tol_rel=tol, inner_max=30)
        Gd, Vd = _dev(G0), _dev(np.eye(np_))
        rc, r = jg.jacobi_gesvd_step(Gd, Vd, s, p)
        assert rc == 0
        assert abs(r - r_or) <= 1e-13
        scale = np.abs(G0).max()
        assert np.abs(_np(Gd) - G_or).max() <= 1e-12 * scale
        assert np.abs(_np(Vd) - V_or).max() <= 1e-12


@pytest.mark.parametrize("m,n,b", [(500, 96, 16), (200, 70, 16), (260, 64, 64), (64, 64, 8)])
def test_known_singular_values(jg, m, n, b):
    G, sig = gen.svd_known(m, n, seed=4100 + n, decades=10.0)
    U_or, s_or, V_or, st_or, rc_or = oracle.gesvd(G, b=b)
    U, s, V, st = jg.gesvd(G, b=b)
    U, s, V = _np(U), _np(s), _np(V)
    assert st.status == 0 and rc_or == 0
    check_svd(G, U, s, V, s_or)
    assert np.abs(s - sig).max() <= 1e-13 * sig[0]


@pytest.mark.parametrize("cl", ["1", "4"])
def test_step_parity_cluster_sizes(jg, monkeypatch, cl):
    monkeypatch.setenv("JACOBI_PIVOT_CLUSTER", cl)
    m, np_, b = 900, 256, 32
    G0 = gen.tall_gaussian(m, np_, 4450, dtype=np.float64)
    tab = oracle.ordering(0, np_ // b)
    G_or, V_or, r_or = oracle.gesvd_step(G0, np.eye(np_), b, tab[1], tol_rel=oracle.svd_tol(m),
                                         inner_max=30)
    Gd, Vd = _dev(G0), _dev(np.eye(np_))
    rc, r = jg.jacobi_gesvd_step(Gd, Vd, 1, jg.params(b=b, tol=1e-15))
    assert rc == 0 and abs(r - r_or) <= 1e-13
    assert np.abs(_np(Gd) - G_or).max() <= 1e-12 * np.abs(G0).max()
    assert np.abs(_np(Vd) - V_or).max() <= 1e-12


def test_without_permutation(jg):
    G, sig = gen.svd_known(300, 48, seed=4150, decades=4.0)
    _, s_or, _, _, rc_or = oracle.gesvd(G, b=8, pivot_order=0)
    U, s, V, st = jg.gesvd(G, b=8, pivot_order=0)
    assert st.status == 0 and rc_or == 0
    check_svd(G, _np(U), _np(s), _np(V), s_or)


def test_zero_column_and_rank_deficiency(jg):
    G = gen.tall_gaussian(120, 40, 4200, dtype=np.float64)
    G[:, 3] = 0.0
    G[:, 17] = G[:, 5]
    U, s, V, st = jg.gesvd(G, b=8)
    U, s, V = _np(U), _np(s), _np(V)
    _, s_or, _, _, _ = oracle.gesvd(G, b=8)
    assert st.status == 0 and s[-1] == 0.0 and np.all(U[:, -1] == 0.0)
    assert np.abs(s - s_or).max() <= 1e-13 * s_or[0]
    assert np.all(np.isfinite(U))


def test_svd_nonfinite_and_args(jg):
    import torch
    G = gen.tall_gaussian(30, 10, 4300, dtype=np.float64)
    G[3, 3] = np.inf
    s = torch.empty(10, dtype=torch.float64, device="cuda")
    V = jg.colmajor_empty(10, 10, torch.float64, "cuda")
    assert jg.jacobi_gesvd(_dev(G), s, V, jg.params(b=2))[0] == jg.ERR_NONFINITE
    Gt = _dev(gen.tall_gaussian(10, 30, 4301, dtype=np.float64))
    s30 = torch.empty(30, dtype=torch.float64, device="cuda")
    assert jg.jacobi_gesvd(Gt, s30, None, jg.params(b=2, want_vectors=0))[0] == -2  # m < n


def test_full_size_16384x2048_b64(jg):
    """The one-sided workload at full size: sigma_i = 10^(-10 i/(n-1))."""
    m, n, b = 16384, 2048, 64
    G, sig = gen.svd_known(m, n, seed=gen.SEEDS["c3"], decades=10.0)
    U, s, V, st = jg.gesvd(G, b=b)
    U, s, V = _np(U), _np(s), _np(V)
    assert st.status == 0
    assert np.abs(s - sig).max() <= 1e-13 * sig[0]
    big = sig >= 1e-3 * sig[0]
    assert (np.abs(s - sig)[big] / sig[big]).max() <= 1e-12
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-13 * n
    assert np.linalg.norm(U.T @ U - np.eye(n)) <= 1e-12 * n


# ------------------------------------------------------------------ QR preconditioning (svd_qr = 1)
@pytest.mark.parametrize("m,n,b", [(500, 96, 16), (300, 45, 8), (64, 64, 8), (1030, 130, 32), (2000, 256, 32)])
def test_qr_preconditioned_known_singular_values(jg, m, n, b):
    """G = QR on the GPU (blocked Householder, ragged panels and row splits),
    the one-sided method on R^T, U = Q W: the oracle's QR-preconditioned
    singular values, orthonormal U and V, G V = U Sigma."""
    G, sig = gen.svd_known(m, n, seed=4500 + n, decades=10.0)
    _, s_or, _, _, rc_or = oracle.gesvd_qr(G, b=b)
    U, s, V, st = jg.gesvd(G, b=b, svd_qr=1)
    U, s, V = _np(U), _np(s), _np(V)
    assert st.status == 0 and rc_or == 0 and st.ms_precond > 0
    # V holds the normalised columns of the rotated R^T (orthogonal to the stop tolerance)
    check_svd(G, U, s, V, s_or, v_orth=1e-12)
    assert np.abs(s - sig).max() <= 1e-13 * sig[0]
    assert np.linalg.norm(U.T @ U - np.eye(n)) <= 1e-12 * n


def test_qr_preconditioned_rank_deficiency(jg):
    G = gen.tall_gaussian(160, 40, 4600, dtype=np.float64)
    G[:, 3] = 0.0
    G[:, 17] = G[:, 5]
    U, s, V, st = jg.gesvd(G, b=8, svd_qr=1)
    U, s, V = _np(U), _np(s), _np(V)
    s_or = oracle.gesvd_qr(G, b=8)[1]
    assert st.status == 0 and np.all(np.isfinite(U)) and np.all(np.isfinite(V))
    assert np.abs(s - s_or).max() <= 1e-13 * s_or[0]
    assert np.linalg.norm(U.T @ U - np.eye(40)) <= 1e-12 * 40      # U = Q W keeps orthonormal columns
    assert np.linalg.norm(G @ V - U * s[None, :]) <= 1e-13 * np.linalg.norm(G) * np.sqrt(40)


def test_qr_preconditioned_full_size_16384x2048_b64(jg):
    """The one-sided workload at full size through the QR form: the same
    gates as the direct form."""
    m, n, b = 16384, 2048, 64
    G, sig = gen.svd_known(m, n, seed=gen.SEEDS["c3"], decades=10.0)
    U, s, V, st = jg.gesvd(G, b=b, svd_qr=1)
    U, s, V = _np(U), _np(s), _np(V)
    assert st.status == 0
    assert np.abs(s - sig).max() <= 1e-13 * sig[0]
    big = sig >= 1e-3 * sig[0]
    assert (np.abs(s - sig)[big] / sig[big]).max() <= 1e-12
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-12 * n
    assert np.linalg.norm(U.T @ U - np.eye(n)) <= 1e-12 * n
