"""Seeded synthetic inputs shaped like the paper's workloads.

Shared by the tests, the benchmark and the smoke check, and the ONLY module that
both the CPU oracle side and the CUDA side use.  It holds no arithmetic of the
Jacobi method: it only draws random numbers (numpy PCG64) and builds matrices
with a prescribed spectrum through LAPACK's Householder QR.

Recipes (seed per workload is fixed by the caller):
  * ``sym_known(n, 'uniform')``   A = Q diag(lam) Q^T, lam ~ U[-1, 1] i.i.d.
  * ``sym_known(n, 'graded')``    lam_i = +-10^(-12 i/(n-1)), random signs, i = 0..n-1
  * ``graded_dhd(n)``             A = D H D, H unit-diagonal SPD with kappa(H) <= 10,
                                   D = diag(10^(-6 i/(n-1)))
  * ``svd_known(m, n)``           G = U diag(sigma) V^T, sigma_i = 10^(-10 i/(n-1))
  * ``sym_gaussian(n)``           (M + M^T)/2, M_ij ~ N(0, 1)
  * ``batch_sizes(count, lo, hi)``n ~ U{lo..hi} (inclusive)
  * ``tall_gaussian(m, n)``       G_ij ~ N(0, 1)
  * ``batch_flat_torch(...)``     the batched workloads drawn on the device (torch's
                                   Philox generator, seeded): many matrices packed
                                   into one flat column-major buffer
Q, U, V come from the Householder QR of a seeded N(0,1) matrix with the signs
fixed so that diag(R) > 0.
"""
from __future__ import annotations

import numpy as np

SEEDS = {"c1": 1, "c2u": 2, "c2g": 3, "c2dhd": 4, "c3": 5, "c4": 6, "c5": 7}


def rng(seed, *more) -> np.random.Generator:
    """PCG64 stream for (seed, *more)."""
    return np.random.default_rng([int(seed), *[int(x) for x in more]])


def haar_q(m: int, n: int, r: np.random.Generator) -> np.ndarray:
    """m x n (m >= n) matrix with orthonormal columns: Householder QR of a
    N(0,1) matrix, signs fixed so that diag(R) > 0."""
    X = r.standard_normal((m, n))
    Q, R = np.linalg.qr(X, mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def spectrum(n: int, kind: str, r: np.random.Generator) -> np.ndarray:
    if kind == "uniform":
        return r.uniform(-1.0, 1.0, n)
    if kind == "graded":
        i = np.arange(n, dtype=np.float64)
        mag = 10.0 ** (-12.0 * i / max(n - 1, 1))
        sgn = np.where(r.random(n) < 0.5, -1.0, 1.0)
        return sgn * mag
    raise ValueError(kind)


def sym_known(n: int, kind: str = "uniform", seed: int = 1):
    """(A, lam): symmetric A = Q diag(lam) Q^T (symmetrised, Fortran order)."""
    r = rng(seed)
    Q = haar_q(n, n, r)
    lam = spectrum(n, kind, r)
    A = (Q * lam[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    return np.asfortranarray(A), lam


def graded_dhd(n: int, seed: int = 4, decades: float = 6.0):
    """A = D H D with H unit-diagonal SPD (eigenvalues of the unscaled H in
    [1, 4]), D = diag(10^(-decades i/(n-1)))."""
    r = rng(seed)
    Q = haar_q(n, n, r)
    mu = r.uniform(1.0, 4.0, n)
    H = (Q * mu[None, :]) @ Q.T
    H = 0.5 * (H + H.T)
    s = 1.0 / np.sqrt(np.diag(H))
    H = H * s[:, None] * s[None, :]
    np.fill_diagonal(H, 1.0)
    i = np.arange(n, dtype=np.float64)
    d = 10.0 ** (-decades * i / max(n - 1, 1))
    A = H * d[:, None] * d[None, :]
    A = 0.5 * (A + A.T)
    return np.asfortranarray(A), d, H


def svd_known(m: int, n: int, seed: int = 5, decades: float = 10.0):
    """(G, sigma): G = U diag(sigma) V^T, sigma_i = 10^(-decades i/(n-1))."""
    r = rng(seed)
    U = haar_q(m, n, r)
    V = haar_q(n, n, r)
    i = np.arange(n, dtype=np.float64)
    sigma = 10.0 ** (-decades * i / max(n - 1, 1))
    G = (U * sigma[None, :]) @ V.T
    return np.asfortranarray(G), sigma


def sym_gaussian(n: int, seed: int, *more, dtype=np.float64) -> np.ndarray:
    """(M + M^T)/2 with M_ij ~ N(0,1), drawn from the stream (seed, *more)."""
    M = rng(seed, *more).standard_normal((n, n))
    return np.asfortranarray((0.5 * (M + M.T)).astype(dtype))


def batch_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """count sizes n ~ U{lo..hi} (inclusive)."""
    return rng(seed, 0).integers(lo, hi + 1, size=count).astype(np.int32)


def tall_gaussian(m: int, n: int, seed: int, *more, dtype=np.float32) -> np.ndarray:
    return np.asfortranarray(rng(seed, *more).standard_normal((m, n)).astype(dtype))


def batch_flat_torch(shapes, seed: int, device, dtype, symmetric: bool = True):
    """Many matrices drawn on the device, packed into one flat buffer.

    shapes: list of (m, n).  Each matrix is M_ij ~ N(0, 1) (torch's seeded
    device generator), symmetrised as (M + M^T)/2 when ``symmetric`` (m == n).
    Returns (flat, views, offsets): ``views[i]`` is matrix i as a column-major
    (m, n) view into ``flat`` (leading dimension m), offsets in elements.
    Drawn in float64 and rounded once to ``dtype``."""
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    offs, tot = [], 0
    for m, n in shapes:
        offs.append(tot)
        tot += m * n
    flat = torch.empty(tot, dtype=dtype, device=device)
    views = []
    for (m, n), o in zip(shapes, offs):
        M = torch.randn(n, m, generator=g, device=device, dtype=torch.float64)  # row-major n x m = col-major m x n
        if symmetric and m == n:
            M = 0.5 * (M + M.t())
        flat[o:o + m * n].copy_(M.reshape(-1))
        views.append(flat[o:o + m * n].view(n, m).t())
    return flat, views, offs
