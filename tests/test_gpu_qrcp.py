"""The pivoting step of Sec. 2.1 (pivot_order = 2): column-pivoted QR of the
leading rows of each pivot's Vhat orders its eigenpairs, Vhat <- Vhat P.
Against the oracle's step element-wise (one CTA per pair and clusters, the
k = 256 pivots, padded blocks), and full two-sided and one-sided solves at
the FP64 gates."""
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


@pytest.mark.parametrize("cl", ["1", "4"])
@pytest.mark.parametrize("np_,b", [(96, 16), (256, 32), (512, 128), (384, 64)])
def test_qrcp_step_matches_oracle(jg, monkeypatch, cl, np_, b):
    monkeypatch.setenv("JACOBI_PIVOT_CLUSTER", cl)
    d = np.linspace(1.0, 2.0 * np_, np_)
    A0 = np.asfortranarray(np.diag(d) + 0.05 * gen.sym_gaussian(np_, 6100 + np_ + b))
    tab = oracle.ordering(0, np_ // b)
    for s in (0, 2):
        A_or, Q_or, _ = oracle.syev_step(A0, np.eye(np_), b, tab[s], pivot_order=2)
        Ad, Qd = _dev(A0), _dev(np.eye(np_))
        assert jg.jacobi_syev_step(Ad, Qd, s, jg.params(b=b, pivot_order=2)) == 0
        assert np.abs(Ad.cpu().numpy() - A_or).max() <= 1e-13 * np.abs(A0).max()
        assert np.abs(Qd.cpu().numpy() - Q_or).max() <= 1e-13


@pytest.mark.parametrize("n,b", [(256, 32), (200, 16), (130, 64)])
def test_qrcp_full_evd(jg, n, b):
    A, lam = gen.sym_known(n, "uniform", seed=6200 + n)
    w_or, *_, s_or = oracle.syev(A, b=b, pivot_order=2)
    w, Q, _, st = jg.syev(A, b=b, pivot_order=2)
    w, Q = w.cpu().numpy(), Q.cpu().numpy()
    assert st.status == 0 and s_or == 0
    assert np.abs(w - np.sort(lam)).max() <= 1e-13 * np.abs(lam).max()
    assert np.abs(w - w_or).max() <= 1e-13 * np.abs(lam).max()
    assert np.linalg.norm(A @ Q - Q * w[None, :]) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13 * n


def test_qrcp_svd_step_and_solve(jg):
    m, np_, b = 500, 96, 16
    G0 = gen.tall_gaussian(m, np_, 6300, dtype=np.float64)
    tab = oracle.ordering(0, np_ // b)
    G_or, V_or, r_or = oracle.gesvd_step(G0, np.eye(np_), b, tab[1], tol_rel=oracle.svd_tol(m), inner_max=30,
                                         pivot_order=2)
    Gd, Vd = _dev(G0), _dev(np.eye(np_))
    rc, r = jg.jacobi_gesvd_step(Gd, Vd, 1, jg.params(b=b, tol=1e-15, pivot_order=2))
    assert rc == 0 and abs(r - r_or) <= 1e-13
    assert np.abs(Gd.cpu().numpy() - G_or).max() <= 1e-12 * np.abs(G0).max()
    assert np.abs(Vd.cpu().numpy() - V_or).max() <= 1e-12
    G, sig = gen.svd_known(400, 80, seed=6301, decades=8.0)
    U, s, V, st = jg.gesvd(G, b=16, pivot_order=2)
    s = s.cpu().numpy()
    assert st.status == 0 and np.abs(s - sig).max() <= 1e-13 * sig[0]


def test_qrcp_mixed_form(jg):
    A, lam = gen.sym_known(512, "uniform", seed=6400)
    w, Q, _, st = jg.syev(A, b=64, precision=2, pivot_order=2)
    w = w.cpu().numpy()
    assert st.status == 0 and np.abs(w - np.sort(lam)).max() <= 1e-12 * np.abs(lam).max()
