"""CPU model of the FP64 rotation parameters of the pivot solves: the same
steps as the GPU helper (FP32 seeds refined by Newton steps in FP64), with
numpy's correctly rounded float32 seeds in place of the GPU's approximate
ones and separate multiplies and adds in place of fused ones, against the
same formulas in long double
over values from 1e-300 to 1e300, equal and negative diagonals and
subnormal off-diagonals: t, s, tau within 6 units of 2^-53 and
c^2 + s^2 = 1 within 4, as the textbook chain of correctly rounded
operations.  The GPU kernel itself is checked the same way in
test_gpu_rotation.py."""
from __future__ import annotations

import numpy as np

U = 2.0 ** -53
f32 = np.float32


def _biased_exp(x):
    return ((np.asarray(x, np.float64).view(np.int64) >> 52) & 0x7FF).astype(np.int64)


def _model(app, aqq, apq):
    d = aqq - app
    E = np.clip(np.maximum(_biased_exp(d), _biased_exp(apq)), 2, 2044)
    sc = ((2045 - E).astype(np.int64) << 52).view(np.float64)        # 2^(1022 - E)
    ds, as_ = d * sc, apq * sc
    d32, a2 = ds.astype(f32), f32(2) * as_.astype(f32)
    dzero, dneg, aneg = d == 0, np.signbit(d), np.signbit(apq)
    with np.errstate(all="ignore"):
        R = np.sqrt(d32 * d32 + a2 * a2).astype(f32)
        sgz = np.where(dzero | (dneg == aneg), f32(1), f32(-1))
        t32 = (sgz * (np.abs(a2) / (np.abs(d32) + R))).astype(f32)
        sgg = np.where(dzero, np.where(aneg, f32(-1), f32(1)), np.where(dneg, f32(-1), f32(1)))
        r = (sgg / R).astype(f32).astype(np.float64)
        t = t32.astype(np.float64)
        for _ in range(2):
            t = t - ((as_ * t + ds) * t - as_) * r
        third = np.abs(a2) < 1e-30
        t = np.where(third, t - ((as_ * t + ds) * t - as_) * r, t)
        x = t * t + 1.0
        y0 = (f32(1) / np.sqrt(x.astype(f32))).astype(f32).astype(np.float64)
        h = 1.0 - (x * y0) * y0
        c = y0 + (y0 * h) * (0.5 + 0.375 * h)
        s = t * c
        u = 1.0 + c
        r0 = (f32(1) / u.astype(f32)).astype(np.float64)
        e = 1.0 - u * r0
        tau = s * (r0 + r0 * (e + e * e))
    return t, s, tau


def _truth(app, aqq, apq):
    L = np.longdouble
    with np.errstate(all="ignore"):
        zeta = (L(aqq) - L(app)) / (L(2) * L(apq))
        t = np.where(zeta >= 0, L(1), L(-1)) / (np.abs(zeta) + np.sqrt(L(1) + zeta * zeta))
        c = L(1) / np.sqrt(L(1) + t * t)
        s = t * c
        tau = s / (L(1) + c)
    return t, s, tau


def _triples(seed, n=20000):
    r = np.random.default_rng(seed)
    base = 10.0 ** r.uniform(-300, 300, n)
    app = base * r.standard_normal(n) * 10.0 ** r.uniform(-3, 3, n)
    aqq = base * r.standard_normal(n) * 10.0 ** r.uniform(-3, 3, n)
    apq = base * r.standard_normal(n) * 10.0 ** r.choice([0.0, -5.0, -12.0, -20.0, -60.0, 4.0], n)
    k = n // 8
    aqq[:k] = app[:k]                                  # equal diagonals
    app[k:2 * k] = -np.abs(app[k:2 * k])               # negative diagonals
    apq[2 * k:3 * k] = app[2 * k:3 * k] * 1e-200       # far below the diagonal
    w = slice(3 * k, 4 * k)
    app[w], aqq[w], apq[w] = r.standard_normal(k), r.standard_normal(k), r.standard_normal(k)
    ok = np.isfinite(aqq - app) & (apq != 0)
    return app[ok], aqq[ok], apq[ok]


def test_newton_step_rotation_matches_long_double():
    if np.finfo(np.longdouble).eps > 1e-17:
        import pytest
        pytest.skip("long double is not wider than double here")
    for seed in (1, 2, 3):
        app, aqq, apq = _triples(seed)
        got = _model(app, aqq, apq)
        want = _truth(app, aqq, apq)
        sel = np.abs(want[0].astype(np.float64)) > 1e-290
        for a, x, name in zip(got, want, ("t", "s", "tau")):
            err = (np.abs(np.longdouble(a[sel]) - x[sel]) / np.abs(x[sel])).astype(np.float64)
            assert err.max() <= 6 * U, (seed, name, err.max() / U)
        s, tau = got[1], got[2]
        c = 1.0 - s * tau
        assert np.abs(c * c + s * s - 1.0).max() <= 4 * U


def test_equal_diagonals_and_subnormal_off_diagonal():
    app = np.array([1.0, 1.0, 6.340876477936385e-259, -2.9e-300])
    aqq = np.array([1.0, 1.0, 6.340876477936385e-259, -2.9e-300])
    apq = np.array([0.5, -0.5, -2.826634e-318, -2.1e-321])
    t, s, tau = _model(app, aqq, apq)
    assert np.all(np.isfinite(t)) and np.all(t == 1.0)    # sgn(0) = +1 picks t = 1
    assert np.allclose(s, np.sqrt(0.5), rtol=4 * U, atol=0)
