"""GPU parity of the batched forms against the CPU oracle.

Each matrix of a batch is solved by the scalar parallel-ordered Jacobi of the
pivot solve (Algorithm 2 applied with b = 1 to the whole matrix); the oracle
for one matrix is therefore ``oracle.pivot_solve`` on it (zero-padded to an
even order: the padding row is never rotated and keeps the eigenvalue 0 at its
position).  FP64 batches are gated like the single-matrix path; FP32 batches
against the FP64 oracle with the FP64 bounds scaled by u32/u64 = 2^29
(eigenvalues 5.4e-5 ||A||_2, residual 5.4e-4 ||A||_F, orthogonality 5.4e-5 n).
"""
from __future__ import annotations

import numpy as np
import pytest

import jacobi_inputs as gen
import oracle

pytestmark = pytest.mark.gpu
SCALE32 = 2.0 ** 29


@pytest.fixture(scope="module")
def jg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_28952_gb300 as m
    m.lib()
    return m


def oracle_eig(A):
    n = A.shape[0]
    k = n + (n & 1)
    Ap = np.zeros((k, k))
    Ap[:n, :n] = A
    D, V, rot, sw = oracle.pivot_solve(Ap)
    return np.sort(np.diag(D)[:n])


def _mk(jg, mats, dtype):
    import torch
    As = [jg.colmajor(a, device="cuda", dtype=dtype) for a in mats]
    ws = [torch.empty(a.shape[0], dtype=dtype, device="cuda") for a in mats]
    Qs = [jg.colmajor_empty(a.shape[0], a.shape[0], dtype, "cuda") for a in mats]
    info = torch.full((len(mats),), -7, dtype=torch.int32, device="cuda")
    return As, ws, Qs, info


SIZES = [1, 2, 3, 8, 17, 31, 64, 65, 100, 127, 128, 129, 130, 190, 255, 300, 384, 511, 512]


@pytest.mark.parametrize("f32", [False, True])
def test_batched_evd_against_oracle(jg, f32):
    import torch
    r = np.random.default_rng(5)
    sizes = SIZES + list(r.integers(1, 200, 20))
    mats = [gen.sym_gaussian(int(n), 7, i) for i, n in enumerate(sizes)]
    dtype = torch.float32 if f32 else torch.float64
    As, ws, Qs, info = _mk(jg, mats, dtype)
    rc, st = jg.jacobi_syev_batched(As, ws, Qs, info, jg.params(), f32=f32)
    assert rc == 0
    assert torch.all(info == 0), info
    sc = SCALE32 if f32 else 1.0
    for A, w, Q in zip(mats, ws, Qs):
        n = A.shape[0]
        w = w.double().cpu().numpy()
        Q = Q.double().cpu().numpy()
        w_or = oracle_eig(A)
        nrm2 = max(np.abs(w_or).max(), 1e-300)
        assert np.abs(w - w_or).max() <= 1e-13 * sc * nrm2, (n, np.abs(w - w_or).max() / nrm2)
        assert np.linalg.norm(A @ Q - Q * w[None, :]) <= 1e-12 * sc * np.linalg.norm(A)
        assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13 * sc * n
        assert np.all(np.diff(w) >= 0)


def test_batched_evd_no_vectors_and_nonfinite(jg):
    import torch
    mats = [gen.sym_gaussian(n, 71, n) for n in (40, 90, 200)]
    mats[1][3, 2] = np.nan
    As, ws, _, info = _mk(jg, mats, torch.float64)
    rc, st = jg.jacobi_syev_batched(As, ws, None, info, jg.params(want_vectors=0))
    assert rc == 0
    assert info.cpu().tolist() == [0, -100, 0]
    for i in (0, 2):
        assert np.abs(ws[i].cpu().numpy() - oracle_eig(mats[i])).max() <= 1e-13 * 30


def test_batched_evd_deterministic_and_matches_single_pivot_path(jg):
    import torch
    mats = [gen.sym_gaussian(n, 72, n) for n in (64, 128, 200)]
    As, ws, Qs, info = _mk(jg, mats, torch.float64)
    jg.jacobi_syev_batched(As, ws, Qs, info, jg.params())
    w1 = [w.clone() for w in ws]
    jg.jacobi_syev_batched(As, ws, Qs, info, jg.params())
    assert all(torch.equal(a, b) for a, b in zip(w1, ws))


def test_plan_autotune_and_replay(jg):
    import torch
    r = np.random.default_rng(6)
    sizes = [int(x) for x in r.integers(8, 257, 300)]
    mats = [gen.sym_gaussian(n, 73, i) for i, n in enumerate(sizes)]
    As, ws, Qs, info = _mk(jg, mats, torch.float32)
    plan = jg.Plan(0, jg.PREC_FP32, sizes, p=jg.params())
    plan.autotune(As, ws, Qs, info)
    th, smk, grid = plan.shape()
    assert th in (128, 256, 512) and grid >= 152
    rc, st = plan.execute(As, ws, Qs, info)
    assert rc == 0 and torch.all(info == 0)
    w1 = [w.clone() for w in ws]
    rc, st2 = plan.execute(As, ws, Qs, info)   # graph replay
    assert rc == 0 and all(torch.equal(a, b) for a, b in zip(w1, ws))
    for i in (0, 17, 299):
        w_or = oracle_eig(mats[i])
        assert np.abs(ws[i].double().cpu().numpy() - w_or).max() <= 1e-13 * SCALE32 * np.abs(w_or).max()
    plan.close()


@pytest.mark.parametrize("f32", [True, False])
def test_plan_autotune_chooses_the_block_size_per_size_class(jg, f32):
    """The autotuner also chooses the order above which the blocked method
    (b = 16) takes over from the unblocked solve; the plan reports it, and
    every matrix on either side of it matches the oracle."""
    import torch
    r = np.random.default_rng(16)
    sizes = [int(x) for x in r.integers(150, 513, 200)] + [512, 500, 321, 320, 319, 257, 200]
    mats = [gen.sym_gaussian(n, 76, i) for i, n in enumerate(sizes)]
    dt = torch.float32 if f32 else torch.float64
    As, ws, Qs, info = _mk(jg, mats, dt)
    plan = jg.Plan(0, jg.PREC_FP32 if f32 else jg.PREC_FP64, sizes, p=jg.params())
    assert plan.blocking() == (16, plan.blocking()[1])      # default crossover before tuning
    plan.autotune(As, ws, Qs, info)
    b, mo = plan.blocking()
    assert b == 16 and (mo in (0, 192, 256, 320, 384, 448, 512) or mo == plan.shape()[1]), (b, mo)
    rc, st = plan.execute(As, ws, Qs, info)
    assert rc == 0 and torch.all(info == 0)
    tol = (1e-13 * SCALE32) if f32 else 1e-13
    for i in range(len(sizes) - 7, len(sizes)):
        w_or = oracle_eig(mats[i])
        assert np.abs(ws[i].double().cpu().numpy() - w_or).max() <= tol * np.abs(w_or).max(), sizes[i]
    plan.close()


def test_batched_tall_svd_f32(jg):
    import torch
    shapes = [(1024, 64)] * 12 + [(300, 40), (100, 100), (64, 1), (77, 33), (2, 2)]
    mats = [gen.tall_gaussian(m, n, 74, i, dtype=np.float64) for i, (m, n) in enumerate(shapes)]
    mats[13] = gen.svd_known(100, 100, seed=75, decades=3.0)[0]
    Gs = [jg.colmajor(g, device="cuda", dtype=torch.float32) for g in mats]
    ss = [torch.empty(g.shape[1], dtype=torch.float32, device="cuda") for g in mats]
    Vs = [jg.colmajor_empty(g.shape[1], g.shape[1], torch.float32, "cuda") for g in mats]
    info = torch.full((len(mats),), -7, dtype=torch.int32, device="cuda")
    rc, st = jg.jacobi_gesvd_batched_f32(Gs, ss, Vs, info, jg.params())
    assert rc == 0 and torch.all(info == 0), info
    for G, U, s, V in zip(mats, Gs, ss, Vs):
        n = G.shape[1]
        U = U.double().cpu().numpy()
        s = s.double().cpu().numpy()
        V = V.double().cpu().numpy()
        _, s_or, _, _, rc_or = oracle.gesvd(G, b=max(1, n // 2) if n > 1 else 1)
        assert np.abs(s - s_or).max() <= 1e-13 * SCALE32 * s_or[0]
        assert np.all(np.diff(s) <= 0)
        assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-13 * SCALE32 * n
        assert np.linalg.norm(U.T @ U - np.eye(n)) <= 1e-13 * SCALE32 * n
        assert np.linalg.norm(G @ V - U * s[None, :]) <= 1e-12 * SCALE32 * np.linalg.norm(G)


def test_batched_tall_svd_tiled_is_bitwise_the_rowwise_kernel(jg, monkeypatch):
    """The row-tiled kernel (the default) keeps every output's FMA chain in
    the order of the one-entry-per-thread kernel (JACOBI_BATCHED_SVD=rowwise):
    sigma, U, V and info agree bit for bit over a batch of tall, square,
    ragged and odd shapes."""
    import torch
    shapes = [(1024, 64)] * 6 + [(300, 40), (100, 100), (64, 1), (77, 33), (2, 2), (129, 65), (1000, 7)]
    mats = [gen.tall_gaussian(m, n, 78, i, dtype=np.float64) for i, (m, n) in enumerate(shapes)]
    outs = []
    for variant in ("rowwise", "tiled"):
        if variant == "rowwise":
            monkeypatch.setenv("JACOBI_BATCHED_SVD", "rowwise")
        else:
            monkeypatch.delenv("JACOBI_BATCHED_SVD", raising=False)
        Gs = [jg.colmajor(g, device="cuda", dtype=torch.float32) for g in mats]
        ss = [torch.empty(g.shape[1], dtype=torch.float32, device="cuda") for g in mats]
        Vs = [jg.colmajor_empty(g.shape[1], g.shape[1], torch.float32, "cuda") for g in mats]
        info = torch.full((len(mats),), -7, dtype=torch.int32, device="cuda")
        rc, st = jg.jacobi_gesvd_batched_f32(Gs, ss, Vs, info, jg.params())
        assert rc == 0 and torch.all(info == 0), (variant, info)
        outs.append((Gs, ss, Vs))
    for a, b in zip(outs[0], outs[1]):
        for x, y in zip(a, b):
            assert torch.equal(x, y)


@pytest.mark.parametrize("f32", [False, True])
def test_batched_large_orders_every_route_against_oracle(jg, monkeypatch, f32):
    """Orders above the shared-memory size: the blocked method, one CTA per
    matrix (default), thread-block clusters (one cluster per matrix, order
    padded to a multiple of the cluster size) and the L2-slot scalar solve
    (JACOBI_BATCHED_LARGE = blocked | cluster | l2) all meet the oracle's
    bounds and agree with each other."""
    import torch
    sizes = [512, 511, 384, 300, 257, 256, 200, 161, 130, 64, 9]
    mats = [gen.sym_gaussian(n, 76, n) for n in sizes]
    mats[3][17, 5] = np.inf        # a non-finite entry in a large matrix
    dtype = torch.float32 if f32 else torch.float64
    sc = SCALE32 if f32 else 1.0
    outs = []
    for route in ("blocked", "cluster", "l2"):
        monkeypatch.setenv("JACOBI_BATCHED_LARGE", route)
        As, ws, Qs, info = _mk(jg, mats, dtype)
        rc, st = jg.jacobi_syev_batched(As, ws, Qs, info, jg.params(), f32=f32)
        assert rc == 0
        inf = info.cpu().tolist()
        assert inf[3] == -100 and all(v == 0 for i, v in enumerate(inf) if i != 3), (route, inf)
        outs.append([w.double().cpu().numpy() for w in ws])
        for i, (A, w, Q) in enumerate(zip(mats, ws, Qs)):
            if i == 3:
                continue
            n = A.shape[0]
            w = w.double().cpu().numpy()
            Q = Q.double().cpu().numpy()
            w_or = oracle_eig(A)
            nrm2 = np.abs(w_or).max()
            assert np.abs(w - w_or).max() <= 1e-13 * sc * nrm2, (route, n, np.abs(w - w_or).max() / nrm2)
            assert np.linalg.norm(A @ Q - Q * w[None, :]) <= 1e-12 * sc * np.linalg.norm(A), (route, n)
            assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13 * sc * n, (route, n)
    for o in outs[1:]:
        for i in range(len(mats)):
            if i != 3:
                assert np.abs(outs[0][i] - o[i]).max() <= 2e-13 * sc * np.abs(o[i]).max()
