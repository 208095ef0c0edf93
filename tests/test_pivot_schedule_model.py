"""CPU model of the two round schedules of the cluster pivot kernel
(k_pivot_cluster<false>, the split schedule, and k_pivot_cluster<true>, the
fused one), with the threads of a cluster run one after another between its
barriers.

The fused schedule lets the thread that rotates a "leading quad" of round g
(a quad holding one of round g + 1's pivot entries) choose round g + 1's
rotation and publish it with the two diagonal entries.  This model mirrors
its index arithmetic (the round-robin position / pair / partner rules, the
leader election, the split of the other quads and of V's rows over the bulk
threads, the zeroing of round g's pivot entries, the double-buffered
diagonal and parameters) and checks, for every round:

* every quad of round g is rotated exactly once (by its leader or by one bulk
  thread), every round-g pivot entry is zeroed once, every diagonal entry and
  every round-(g + 1) rotation is published exactly once;
* each leading quad holds the pivot entries its leader publishes;
* no thread index or slot leaves its array.

Then it runs both schedules with the same scalar operations (the textbook
rotation in Python floats stands in for the kernel's) and requires the
results to be equal bit for bit: the fused schedule changes who computes
what and when, not the arithmetic.
"""
from __future__ import annotations

import math

import numpy as np
import pytest


def rr_index_at(pos, rd, nr):
    if pos == 0:
        return 0
    v = pos - 1 + rd
    if v >= nr:
        v -= nr
    return 1 + v


def rr_position_of(x, rd, nr):
    if x == 0:
        return 0
    v = x - 1 - rd
    if v < 0:
        v += nr
    return 1 + v


def rr_pair_of(x, rd, k):
    pos = rr_position_of(x, rd, k - 1)
    return min(pos, k - 1 - pos)


def rr_partner_of(x, rd, k):
    return rr_index_at(k - 1 - rr_position_of(x, rd, k - 1), rd, k - 1)


def round_pairs(rd, k):
    """choose()'s rule: pair ee joins positions ee and k - 1 - ee."""
    out = []
    for ee in range(k // 2):
        pa, pb = ee, k - 1 - ee
        ia = 0 if pa == 0 else 1 + (pa - 1 + rd) % (k - 1)
        ib = 1 + (pb - 1 + rd) % (k - 1)
        out.append((min(ia, ib), max(ia, ib)))
    return out


def quads(half):
    """Quad table order (by e2, then e1)."""
    return [(e1, e2) for e2 in range(1, half) for e1 in range(e2)]


@pytest.mark.parametrize("k", [16, 18, 32, 64, 128, 256])
def test_round_robin_helpers_match_the_schedule(k):
    nr = k - 1
    for rd in range(nr):
        pr = round_pairs(rd, k)
        for ee, (p, q) in enumerate(pr):
            for x, y in ((p, q), (q, p)):
                assert rr_pair_of(x, rd, k) == ee
                assert rr_partner_of(x, rd, k) == y
        # every index once per round; every pair once per sweep
        assert sorted(x for pq in pr for x in pq) == list(range(k))
    allp = [pq for rd in range(nr) for pq in round_pairs(rd, k)]
    assert len(set(allp)) == k * (k - 1) // 2


@pytest.mark.parametrize("k,C,nt", [(16, 2, 64), (32, 4, 64), (64, 2, 96), (128, 4, 512),
                                    (256, 4, 512), (256, 2, 512), (48, 3, 64)])
def test_fused_round_covers_every_quad_entry_and_parameter_once(k, C, nt):
    half, nr = k // 2, k - 1
    upc = (half + C - 1) // C
    lw = (upc + 31) // 32 * 32
    assert lw < nt
    bt = nt - lw
    qt = quads(half)
    nq = len(qt)
    for rd in range(nr):
        for last in (False, True):
            rdn = 0 if rd + 1 == nr else rd + 1
            pr, prn = round_pairs(rd, k), round_pairs(rdn, k)
            quad_done = [0] * nq
            qidx = {q: i for i, q in enumerate(qt)}
            diag_pub = [0] * k
            par_pub = [0] * half
            zeroed = [0] * half
            for r in range(C):
                for tid in range(nt):
                    if tid < lw:
                        ep = r + C * tid
                        if ep < half:
                            x0 = rr_index_at(ep, rdn, nr)
                            y0 = rr_index_at(k - 1 - ep, rdn, nr)
                            assert {x0, y0} == set(prn[ep])
                            if last:
                                diag_pub[x0] += 1
                                diag_pub[y0] += 1
                            else:
                                ea, eb = rr_pair_of(x0, rd, k), rr_pair_of(y0, rd, k)
                                assert ea != eb
                                e1, e2 = min(ea, eb), max(ea, eb)
                                p1, q1 = pr[e1]
                                p2, q2 = pr[e2]
                                pp1, pq1 = rr_partner_of(p1, rdn, k), rr_partner_of(q1, rdn, k)
                                h1 = pp1 in (p2, q2)
                                h2 = pq1 in (p2, q2)
                                ep1 = rr_pair_of(p1, rdn, k) if h1 else half
                                ep2 = rr_pair_of(q1, rdn, k) if h2 else half
                                assert ep in (ep1, ep2)
                                if min(ep1, ep2) == ep:
                                    quad_done[qidx[(e1, e2)]] += 1
                                    for hh, x, y, epc in ((h1, p1, pp1, ep1), (h2, q1, pq1, ep2)):
                                        if hh:
                                            assert set(prn[epc]) == {x, y}
                                            diag_pub[x] += 1
                                            diag_pub[y] += 1
                                            par_pub[epc] += 1
                        if ep < half:
                            zeroed[ep] += 1
                    else:
                        btid = tid - lw
                        for qi in range(r * bt + btid, nq, C * bt):
                            e1, e2 = qt[qi]
                            p1, q1 = pr[e1]
                            p2, q2 = pr[e2]
                            if not last:
                                pp1, pq1 = rr_partner_of(p1, rdn, k), rr_partner_of(q1, rdn, k)
                                if pp1 in (p2, q2) or pq1 in (p2, q2):
                                    continue
                            quad_done[qi] += 1
            assert quad_done == [1] * nq, (rd, last)
            assert diag_pub == [1] * k
            assert zeroed == [1] * half
            assert par_pub == ([0] * half if last else [1] * half)


# ------------------------------------------------------------------ both schedules, same arithmetic
def schur(app, aqq, apq):
    zeta = (aqq - app) / (2.0 * apq)
    t = (1.0 if zeta >= 0 else -1.0) / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
    c = 1.0 / math.sqrt(1.0 + t * t)
    s = t * c
    return s, t, s / (1.0 + c)


def rot2(s, tau, x, y):
    a, b = x, y
    return a - s * (tau * a + b), b + s * (a - tau * b)


def wanted(app, aqq, apq, tol):
    return apq != 0.0 and abs(apq) > tol * math.sqrt(abs(app)) * math.sqrt(abs(aqq))


class Sym:
    """Packed symmetric storage (entry (i, j) and (j, i) are one cell)."""

    def __init__(self, A):
        self.k = A.shape[0]
        self.v = {(i, j): float(A[i, j]) for i in range(self.k) for j in range(i + 1)}

    def get(self, i, j):
        return self.v[(max(i, j), min(i, j))]

    def set(self, i, j, x):
        self.v[(max(i, j), min(i, j))] = x


def rotate_quad(S, par, e1, e2):
    p1, q1, on1, s1, tau1 = par[e1][:5]
    p2, q2, on2, s2, tau2 = par[e2][:5]
    x00, x01, x10, x11 = S.get(p1, p2), S.get(p1, q2), S.get(q1, p2), S.get(q1, q2)
    if on1:
        x00, x10 = rot2(s1, tau1, x00, x10)
        x01, x11 = rot2(s1, tau1, x01, x11)
    if on2:
        x00, x01 = rot2(s2, tau2, x00, x01)
        x10, x11 = rot2(s2, tau2, x10, x11)
    if on1 or on2:
        S.set(p1, p2, x00)
        S.set(p1, q2, x01)
        S.set(q1, p2, x10)
        S.set(q1, q2, x11)
    return x00, x01, x10, x11


def diag_step(d, p, q, t, apq):
    """The diagonal of the rotated 2 x 2 pivot (hi only; the kernel carries
    hi + lo with the same operation order in both schedules)."""
    return d[p] - t * apq, d[q] + t * apq


def choose(p, q, app, aqq, apq, tol):
    on = wanted(app, aqq, apq, tol)
    if on:
        s, t, tau = schur(app, aqq, apq)
        return (p, q, True, s, tau, t, apq)
    return (p, q, False, 0.0, 0.0, 0.0, 0.0)


def run_split(A, rounds, tol):
    k = A.shape[0]
    half, nr = k // 2, k - 1
    S = Sym(A)
    d = [S.get(i, i) for i in range(k)]
    V = np.eye(k)
    par = [choose(p, q, d[p], d[q], S.get(q, p), tol) for p, q in round_pairs(0, k)]
    for g in range(rounds):
        for e1, e2 in quads(half):
            if par[e1][2] or par[e2][2]:
                rotate_quad(S, par, e1, e2)
        for p, q, on, s, tau, t, apq in par:
            if on:
                d[p], d[q] = diag_step(d, p, q, t, apq)
        for p, q, on, *_ in par:
            if on:
                S.set(q, p, 0.0)
        nxt = None
        if g + 1 < rounds:
            nxt = [choose(p, q, d[p], d[q], S.get(q, p), tol) for p, q in round_pairs((g + 1) % nr, k)]
        for p, q, on, s, tau, t, apq in par:
            if on:
                for i in range(k):
                    V[i, p], V[i, q] = rot2(s, tau, V[i, p], V[i, q])
        par = nxt
    for i in range(k):
        S.set(i, i, d[i])
    return S, V


def run_fused(A, rounds, tol, C, nt):
    k = A.shape[0]
    half, nr = k // 2, k - 1
    upc = (half + C - 1) // C
    lw = (upc + 31) // 32 * 32
    bt = nt - lw
    S = Sym(A)
    D = [[S.get(i, i) for i in range(k)], [None] * k]
    V = np.eye(k)
    P = [[choose(p, q, D[0][p], D[0][q], S.get(q, p), tol) for p, q in round_pairs(0, k)], [None] * half]
    qt = quads(half)
    for g in range(rounds):
        rd, cb = g % nr, g & 1
        nb = cb ^ 1
        last = g + 1 == rounds
        rdn = (rd + 1) % nr
        par, d = P[cb], D[cb]

        def diag_after(x):
            eg = rr_pair_of(x, rd, k)
            p, q, on, s, tau, t, apq = par[eg]
            if not on:
                return d[x]
            return d[x] - t * apq if x == p else d[x] + t * apq

        for r in range(C):
            for tid in range(nt):
                if tid < lw:
                    ep = r + C * tid
                    if ep < half:
                        x0, y0 = rr_index_at(ep, rdn, nr), rr_index_at(k - 1 - ep, rdn, nr)
                        if last:
                            D[nb][x0], D[nb][y0] = diag_after(x0), diag_after(y0)
                        else:
                            ea, eb = rr_pair_of(x0, rd, k), rr_pair_of(y0, rd, k)
                            e1, e2 = min(ea, eb), max(ea, eb)
                            p1, q1 = par[e1][:2]
                            p2, q2 = par[e2][:2]
                            pp1, pq1 = rr_partner_of(p1, rdn, k), rr_partner_of(q1, rdn, k)
                            h1, h2 = pp1 in (p2, q2), pq1 in (p2, q2)
                            ep1 = rr_pair_of(p1, rdn, k) if h1 else half
                            ep2 = rr_pair_of(q1, rdn, k) if h2 else half
                            if min(ep1, ep2) == ep:
                                x00, x01, x10, x11 = rotate_quad(S, par, e1, e2)
                                for hh, x, y, epc, axy in ((h1, p1, pp1, ep1, x00 if pp1 == p2 else x01),
                                                           (h2, q1, pq1, ep2, x10 if pq1 == p2 else x11)):
                                    if hh:
                                        hx, hy = diag_after(x), diag_after(y)
                                        D[nb][x], D[nb][y] = hx, hy
                                        pp, qq = min(x, y), max(x, y)
                                        app, aqq = (hx, hy) if pp == x else (hy, hx)
                                        P[nb][epc] = choose(pp, qq, app, aqq, axy, tol)
                    if ep < half and par[ep][2]:
                        S.set(par[ep][1], par[ep][0], 0.0)
                else:
                    btid = tid - lw
                    for qi in range(r * bt + btid, len(qt), C * bt):
                        e1, e2 = qt[qi]
                        if not (par[e1][2] or par[e2][2]):
                            continue
                        p1, q1 = par[e1][:2]
                        p2, q2 = par[e2][:2]
                        if not last:
                            pp1, pq1 = rr_partner_of(p1, rdn, k), rr_partner_of(q1, rdn, k)
                            if pp1 in (p2, q2) or pq1 in (p2, q2):
                                continue
                        rotate_quad(S, par, e1, e2)
        # V (this model keeps all rows in one array; the kernel splits them by CTA)
        for p, q, on, s, tau, t, apq in par:
            if on:
                for i in range(k):
                    V[i, p], V[i, q] = rot2(s, tau, V[i, p], V[i, q])
    dfin = D[rounds & 1]
    for i in range(k):
        S.set(i, i, dfin[i])
    return S, V


@pytest.mark.parametrize("k,C,nt,seed", [(16, 2, 64, 1), (32, 4, 64, 2), (48, 3, 64, 3), (64, 4, 128, 4)])
def test_fused_and_split_schedules_agree_bit_for_bit(k, C, nt, seed):
    r = np.random.default_rng(seed)
    M = r.standard_normal((k, k))
    A = 0.5 * (M + M.T) + np.diag(np.linspace(1, 4, k))
    rounds = 4 * (k - 1) + 3           # four sweeps and a bit: sweep boundaries included
    S1, V1 = run_split(A, rounds, 4 * 2.0 ** -53)
    S2, V2 = run_fused(A, rounds, 4 * 2.0 ** -53, C, nt)
    assert S1.v == S2.v
    assert np.array_equal(V1, V2)
    # and the result is a Jacobi solve: V^T A V is the (nearly diagonal) iterate
    D = np.array([[S1.get(i, j) for j in range(k)] for i in range(k)])
    assert np.abs(V1.T @ A @ V1 - D).max() <= 1e-12 * np.abs(A).max()
    off = np.linalg.norm(D - np.diag(np.diag(D)))
    assert off <= 0.1 * np.linalg.norm(A - np.diag(np.diag(A)))
