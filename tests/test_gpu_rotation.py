"""The 2x2 Schur rotation of the FP64 pivot solves (Sec. 2.1, Algorithm 1 with
b = 1) against the textbook formulas in correctly rounded FP64 operations,
over inputs from the well-scaled to the extreme: t, s, tau agree to a few
units in the last place, c^2 + s^2 = 1 (c = 1 - s tau, the cosine the
Rutishauser form applies) to the same order, the rotated off-diagonal entry
is zero to working precision, and the rotation test agrees except at the
threshold itself."""
from __future__ import annotations

import numpy as np
import pytest

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


def _triples(seed):
    r = np.random.default_rng(seed)
    n = 20000
    # magnitudes from 1e-300 to 1e300 overall; within a triple mostly close, sometimes far apart
    base = 10.0 ** r.uniform(-300, 300, n)
    app = base * r.standard_normal(n) * 10.0 ** r.uniform(-3, 3, n)
    aqq = base * r.standard_normal(n) * 10.0 ** r.uniform(-3, 3, n)
    apq = base * r.standard_normal(n) * 10.0 ** r.choice([0.0, -5.0, -12.0, -20.0, -60.0, 4.0], n)
    # special structure: equal diagonals, negative diagonals, tiny and huge ratios, well scaled
    k = n // 8
    aqq[:k] = app[:k]
    app[k:2 * k] = -np.abs(app[k:2 * k])
    apq[2 * k:3 * k] = app[2 * k:3 * k] * 1e-200
    w = slice(3 * k, 4 * k)
    app[w], aqq[w], apq[w] = r.standard_normal(k), r.standard_normal(k), r.standard_normal(k)
    return app, aqq, apq


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rotation_matches_textbook(jg, seed):
    import torch
    app, aqq, apq = _triples(seed)
    ok = np.isfinite(aqq - app) & (apq != 0)
    app, aqq, apq = app[ok], aqq[ok], apq[ok]
    dev = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in (app, aqq, apq)]
    out = torch.empty((app.size, 8), dtype=torch.float64, device="cuda")
    tol = 2.0 ** -52
    assert jg.jacobi_rotation_params(dev[0], dev[1], dev[2], tol, out) == 0
    o = out.cpu().numpy()
    t, s, tau, on, t0, s0, tau0, on0 = o.T
    # both against the same formulas in long double (x86: 64-bit significand;
    # elsewhere quad), where the FP64 values are in the normal range
    L = np.longdouble
    with np.errstate(all="ignore"):
        zeta = (L(aqq) - L(app)) / (L(2) * L(apq))
        tt = np.where(zeta >= 0, L(1), L(-1)) / (np.abs(zeta) + np.sqrt(L(1) + zeta * zeta))
        cc = L(1) / np.sqrt(L(1) + tt * tt)
        ss = tt * cc
        ttau = ss / (L(1) + cc)
    sel = np.abs(t0) > 1e-290
    for a, b, x, name in ((t, t0, tt, "t"), (s, s0, ss, "s"), (tau, tau0, ttau, "tau")):
        err = (np.abs(L(a[sel]) - x[sel]) / np.abs(x[sel])).astype(np.float64)
        err0 = (np.abs(L(b[sel]) - x[sel]) / np.abs(x[sel])).astype(np.float64)
        assert err.max() <= 6 * U, (name, err.max() / U)
        assert err0.max() <= 6 * U, (name, "textbook", err0.max() / U)
    c = 1.0 - s * tau
    assert np.abs(c * c + s * s - 1.0).max() <= 8 * U
    # the rotated off-diagonal entry c s (app - aqq) + (c^2 - s^2) apq, relative
    # to the 2x2 block, in long double where the platform has it
    L = np.longdouble
    cl, sl = L(1) - L(s) * L(tau), L(s)
    off = cl * sl * (L(app) - L(aqq)) + (cl * cl - sl * sl) * L(apq)
    scale = np.maximum(np.maximum(np.abs(app), np.abs(aqq)), np.abs(apq))
    rel_off = np.abs(off.astype(np.float64)) / scale
    assert rel_off[sel].max() <= 32 * U
    # rotation test: equal except within a relative 1e-12 of the threshold
    thr = tol * np.sqrt(np.abs(app)) * np.sqrt(np.abs(aqq))
    near = np.abs(np.abs(apq) - thr) <= 1e-12 * thr
    assert np.array_equal(on[~near], on0[~near])


def test_rotation_special_values(jg):
    import torch
    # exactly equal diagonals: sgn(0) = +1 picks t = 1 for either sign of apq
    app = np.array([1.0, 1.0, -3.0, 5.0, 1e-300, 1e300])
    aqq = np.array([1.0, 1.0, -3.0, 5.0 + 2.0 ** -50, 1e-300, 1e300])
    apq = np.array([0.5, -0.5, 2.0, 1e-20, 1e-310, 1e290])
    dev = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in (app, aqq, apq)]
    out = torch.empty((app.size, 8), dtype=torch.float64, device="cuda")
    assert jg.jacobi_rotation_params(dev[0], dev[1], dev[2], 0.0, out) == 0
    o = out.cpu().numpy()
    assert o[0, 0] == 1.0 and o[1, 0] == 1.0 and o[2, 0] == 1.0
    for i in range(app.size):
        assert abs(o[i, 0] - o[i, 4]) <= 8 * U * abs(o[i, 4]), (i, o[i])
        assert o[i, 3] == o[i, 7] == 1.0
    assert jg.jacobi_rotation_params(dev[0], dev[1], dev[2], -1.0, out) == -5
