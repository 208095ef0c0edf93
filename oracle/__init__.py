"""CPU FP64 oracle for blocked Jacobi (EVD and one-sided SVD).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2608_28952_gb300``) never imports it, and the two share no code.

Thin ctypes marshalling over ``jacobi_oracle.c`` (plain C, IEEE binary64).
Every function cites the passage of Demmel, Luo, Schneider & Wang, "Minimizing
the Arithmetic and Communication Complexity of Jacobi's Method ... Part Two"
that it follows; the C source states the readings taken where the paper is
silent.

Pinned by ``tests/test_oracle_pins.py`` against closed forms, invariants,
brute force (exact characteristic polynomial at n <= 4), the paper's printed
ordering tables, and LAPACK as an independent witness (singular values, the
QRCP column order of the pivoting step).  ``gesvd_qr`` composes LAPACK's QR
(a library step) with the pinned one-sided method.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

ORDER_ROUND_ROBIN = 0
ORDER_ANTI_DIAGONAL = 1
CONV_OFF_ABS = 0
CONV_REL = 1
U64 = 2.0 ** -53


class _Params(C.Structure):
    _fields_ = [("b", C.c_int), ("ordering", C.c_int), ("max_sweeps", C.c_int),
                ("inner_max_sweeps", C.c_int), ("conv", C.c_int), ("tol", C.c_double),
                ("inner_tol", C.c_double), ("want_vectors", C.c_int), ("threads", C.c_int),
                ("pivot_order", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("sweeps", C.c_int), ("stalled", C.c_int),
                ("steps", C.c_longlong), ("pair_solves", C.c_longlong),
                ("rotations", C.c_longlong), ("inner_sweeps", C.c_longlong),
                ("off_initial", C.c_double), ("off_final", C.c_double),
                ("norm_fro", C.c_double), ("off_hist", C.c_double * 64),
                ("rel_hist", C.c_double * 64)]


@dataclass
class Stats:
    status: int
    sweeps: int
    stalled: int
    steps: int
    pair_solves: int
    rotations: int
    inner_sweeps: int
    off_initial: float
    off_final: float
    norm_fro: float
    off_hist: list = field(default_factory=list)
    rel_hist: list = field(default_factory=list)


def _stats(s: _Stats) -> Stats:
    k = max(0, min(64, s.sweeps))
    return Stats(s.status, s.sweeps, s.stalled, s.steps, s.pair_solves, s.rotations,
                 s.inner_sweeps, s.off_initial, s.off_final, s.norm_fro,
                 list(s.off_hist)[:k], list(s.rel_hist)[:k])


_LIB = None
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)
_FP = C.POINTER(C.c_float)


def lib():
    global _LIB
    if _LIB is None:
        L = C.CDLL(_build.build())
        L.oracle_ordering.argtypes = [C.c_int, C.c_int, _IP, _IP]
        L.oracle_ordering.restype = C.c_int
        L.oracle_rotation.argtypes = [C.c_double, C.c_double, C.c_double, _DP, _DP, _DP]
        L.oracle_rotation.restype = None
        L.oracle_rotate.argtypes = [C.c_int, _DP, C.c_int, _DP, C.c_int, C.c_int, C.c_int]
        L.oracle_rotate.restype = C.c_int
        L.oracle_off_norm.argtypes = [C.c_int, _DP, C.c_int]
        L.oracle_off_norm.restype = C.c_double
        L.oracle_rel_off.argtypes = [C.c_int, _DP, C.c_int]
        L.oracle_rel_off.restype = C.c_double
        L.oracle_pivot_solve.argtypes = [C.c_int, _DP, _DP, C.c_double, C.c_int, _IP]
        L.oracle_pivot_solve.restype = C.c_int
        L.oracle_padded_blocks.argtypes = [C.c_int, C.c_int, C.c_int]
        L.oracle_padded_blocks.restype = C.c_int
        L.oracle_syev_step.argtypes = [C.c_int, C.c_int, _DP, _DP, C.c_int, _IP, C.c_double,
                                       C.c_int, C.c_int]
        L.oracle_syev_step.restype = C.c_longlong
        for name in ("oracle_syev_blocked", "oracle_syev_scalar"):
            f = getattr(L, name)
            f.argtypes = [C.c_int, _DP, C.c_int, _DP, _DP, C.c_int, C.POINTER(_Params),
                          C.POINTER(_Stats)]
            f.restype = C.c_int
        for name in ("oracle_gesvd_blocked", "oracle_gesvd_scalar"):
            f = getattr(L, name)
            f.argtypes = [C.c_int, C.c_int, _DP, C.c_int, _DP, _DP, C.c_int,
                          C.POINTER(_Params), C.POINTER(_Stats)]
            f.restype = C.c_int
        L.oracle_gram_pair.argtypes = [C.c_int, C.c_int, _DP, C.c_int, C.c_int, C.c_int, _DP]
        L.oracle_gram_pair.restype = None
        L.oracle_gesvd_step.argtypes = [C.c_int, C.c_int, C.c_int, _DP, C.c_int, _DP, C.c_int,
                                        _IP, C.c_double, C.c_int, C.c_int]
        L.oracle_gesvd_step.restype = C.c_double
        L.oracle_split_bf16.argtypes = [C.c_int, _FP, _FP, _FP]
        L.oracle_split_bf16.restype = None
        L.oracle_qrcp_perm.argtypes = [C.c_int, C.c_int, _DP, _IP]
        L.oracle_qrcp_perm.restype = C.c_int
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(_DP)


def _f64F(a) -> np.ndarray:
    """Column-major float64 copy."""
    return np.array(a, dtype=np.float64, order="F", copy=True)


# ---------------------------------------------------------------- orderings
def ordering(kind: int, N: int) -> list[list[tuple[int, int]]]:
    """Ordering table as a list of steps, each a list of 0-based pairs (I<J).

    kind 0: round-robin tournament; kind 1: Algorithm 3 ("cyclic by
    anti-diagonals", groups K = 0..N-1)."""
    maxp = N * (N - 1) // 2
    pairs = np.zeros(2 * max(maxp, 1), dtype=np.int32)
    ptr = np.zeros(N + 1, dtype=np.int32)
    S = lib().oracle_ordering(kind, N, pairs.ctypes.data_as(_IP), ptr.ctypes.data_as(_IP))
    if S < 0:
        raise ValueError("bad ordering arguments")
    return [[(int(pairs[2 * e]), int(pairs[2 * e + 1])) for e in range(ptr[s], ptr[s + 1])]
            for s in range(S)]


def padded_blocks(n: int, b: int, kind: int = ORDER_ROUND_ROBIN) -> int:
    return lib().oracle_padded_blocks(n, b, kind)


# ---------------------------------------------------------------- scalar pieces
def rotation(app: float, aqq: float, apq: float) -> tuple[float, float, float]:
    """(c, s, t) of the textbook 2x2 symmetric Schur rotation (Sec. 1)."""
    c, s, t = C.c_double(), C.c_double(), C.c_double()
    lib().oracle_rotation(app, aqq, apq, C.byref(c), C.byref(s), C.byref(t))
    return c.value, s.value, t.value


def rotate(A: np.ndarray, Q: np.ndarray | None, p: int, q: int):
    """Apply one textbook rotation annihilating A(p,q) (Sec. 1).  Returns (A', Q', applied)."""
    A = _f64F(A)
    n = A.shape[0]
    Qc = _f64F(Q) if Q is not None else None
    r = lib().oracle_rotate(n, _dp(A), n, _dp(Qc) if Qc is not None else None, n, p, q)
    return A, Qc, bool(r)


def off_norm(A: np.ndarray) -> float:
    """Xi(A) = sqrt(sum_{i != j} A(i,j)^2), Sec. 2.1 eq. (Omega_A)."""
    A = _f64F(A)
    return lib().oracle_off_norm(A.shape[0], _dp(A), A.shape[0])


def rel_off(A: np.ndarray) -> float:
    """max_{i != j} |A(i,j)| / sqrt(|A(i,i)| |A(j,j)|), the relative stop
    measure (an entry over a zero diagonal product counts as 0 when it is 0,
    else +inf)."""
    A = _f64F(A)
    return lib().oracle_rel_off(A.shape[0], _dp(A), A.shape[0])


def pivot_solve(Ahat: np.ndarray, tol_rel: float = 4 * U64, max_sweeps: int = 30):
    """Diagonalise a k x k symmetric pivot by Jacobi on 1x1 blocks in the
    round-robin parallel order (Algorithm 2 with b = 1).

    Returns (D, V, rotations, sweeps) with V^T Ahat V ~= D."""
    A = _f64F(Ahat)
    k = A.shape[0]
    V = np.zeros((k, k), order="F")
    sw = C.c_int()
    rot = lib().oracle_pivot_solve(k, _dp(A), _dp(V), tol_rel, max_sweeps, C.byref(sw))
    return A, V, rot, sw.value


# ---------------------------------------------------------------- EVD
def _params(b, ordering, max_sweeps, inner_max_sweeps, conv, tol, inner_tol, want_vectors,
            threads, pivot_order=1):
    return _Params(b, ordering, max_sweeps, inner_max_sweeps, conv, tol, inner_tol,
                   int(want_vectors), threads, pivot_order)


def qrcp_perm(X: np.ndarray) -> np.ndarray:
    """The column order chosen by column-pivoted QR of X (Businger-Golub,
    norms recomputed at every step, ties to the smaller index): the rule of
    the pivoting step (Sec. 2.1) applied to the leading rows of Vhat."""
    X = _f64F(X)
    r, c = X.shape
    perm = np.zeros(c, dtype=np.int32)
    if lib().oracle_qrcp_perm(r, c, _dp(X), perm.ctypes.data_as(_IP)) != 0:
        raise ValueError("oracle qrcp: bad argument")
    return perm


def syev_step(A: np.ndarray, Q: np.ndarray | None, b: int, pairs, tol_rel=4 * U64,
              inner_max=1, pivot_order=1):
    """One parallel step (Algorithm 2 structure) on a full np x np matrix;
    pivot_order 1 sorts each pivot's eigenpairs descending, 2 orders them by
    QRCP of Vhat's leading rows (the pivoting step of Sec. 2.1); either way
    Qhat <- Qhat P.

    Returns (A', Q', rotations)."""
    A = _f64F(A)
    npd = A.shape[0]
    Qc = _f64F(Q) if Q is not None else None
    pr = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1))
    rot = lib().oracle_syev_step(npd, b, _dp(A), _dp(Qc) if Qc is not None else None,
                                 len(pairs), pr.ctypes.data_as(_IP), tol_rel, inner_max,
                                 pivot_order)
    return A, Qc, int(rot)


def syev(A: np.ndarray, b: int = 16, *, scalar: bool = False, tol: float = 1e-14,
         ordering: int = ORDER_ROUND_ROBIN, max_sweeps: int = 60, inner_max_sweeps: int = 1,
         conv: int = CONV_OFF_ABS, inner_tol: float = 4 * U64, want_vectors: bool = True,
         threads: int = 0, pivot_order: int = 1):
    """Blocked (Algorithm 1 in the parallel order of Algorithm 2) or scalar
    cyclic Jacobi EVD of the symmetric A (lower triangle read).

    Returns (w ascending, Q or None, A_final, Stats, status)."""
    A = _f64F(A)
    n = A.shape[0]
    w = np.zeros(n)
    Q = np.zeros((n, n), order="F") if want_vectors else None
    p = _params(b, ordering, max_sweeps, inner_max_sweeps, conv, tol, inner_tol, want_vectors,
                threads, pivot_order)
    st = _Stats()
    f = lib().oracle_syev_scalar if scalar else lib().oracle_syev_blocked
    status = f(n, _dp(A), n, _dp(w), _dp(Q) if Q is not None else None, n, C.byref(p),
               C.byref(st))
    if status < 0:
        raise ValueError(f"oracle syev: bad argument {status}")
    return w, Q, A, _stats(st), status


# ---------------------------------------------------------------- SVD
def svd_tol(m: int) -> float:
    """Effective one-sided stop tolerance max(1e-15, sqrt(m) u64)."""
    return max(1e-15, np.sqrt(m) * U64)


def gram_pair(G: np.ndarray, b: int, I: int, J: int) -> np.ndarray:
    """Gram block G(:,[I,J])^T G(:,[I,J]) (Sec. 6, eq. (SVD_subproblem))."""
    G = _f64F(G)
    m = G.shape[0]
    out = np.zeros((2 * b, 2 * b), order="F")
    lib().oracle_gram_pair(m, b, _dp(G), m, I, J, _dp(out))
    return out


def gesvd_step(G: np.ndarray, V: np.ndarray | None, b: int, pairs, tol_rel: float,
               inner_max: int = 30, pivot_order: int = 1):
    """One one-sided step over disjoint column pairs.  Returns (G', V', max_rel_off)."""
    G = _f64F(G)
    m, npd = G.shape
    Vc = _f64F(V) if V is not None else None
    pr = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1))
    r = lib().oracle_gesvd_step(m, npd, b, _dp(G), m, _dp(Vc) if Vc is not None else None,
                                len(pairs), pr.ctypes.data_as(_IP), tol_rel, inner_max,
                                pivot_order)
    return G, Vc, r


def gesvd(G: np.ndarray, b: int = 16, *, scalar: bool = False, tol: float | None = None,
          ordering: int = ORDER_ROUND_ROBIN, max_sweeps: int = 60, inner_max_sweeps: int = 30,
          want_vectors: bool = True, threads: int = 0, pivot_order: int = 1):
    """Blocked one-sided Jacobi SVD (Algorithm 6 in the parallel order) or the
    scalar Hestenes form.  Returns (U, sigma descending, V or None, Stats, status)."""
    G = _f64F(G)
    m, n = G.shape
    if tol is None:
        tol = svd_tol(m)
    s = np.zeros(n)
    V = np.zeros((n, n), order="F") if want_vectors else None
    p = _params(b, ordering, max_sweeps, inner_max_sweeps, CONV_REL, tol, tol, want_vectors,
                threads, pivot_order)
    st = _Stats()
    f = lib().oracle_gesvd_scalar if scalar else lib().oracle_gesvd_blocked
    status = f(m, n, _dp(G), m, _dp(s), _dp(V) if V is not None else None, n, C.byref(p),
               C.byref(st))
    if status < 0:
        raise ValueError(f"oracle gesvd: bad argument {status}")
    return G, s, V, _stats(st), status


def gesvd_qr(G: np.ndarray, b: int = 16, *, transpose: bool = True, **kw):
    """One-sided SVD preconditioned by a reduced QR factorisation (Sec. 6,
    subsection "Preprocessing with QR"): G = QR, the blocked one-sided method
    on X = R^T (transpose, default) or on R, and the SVD of G from Q times the
    left singular vectors of R.  The QR factorisation is LAPACK's Householder
    QR through numpy (a library step).  On X = R^T: X W = U_X Sigma, so
    R = W Sigma U_X^T and G = (Q W) Sigma U_X^T.  Returns (U, sigma
    descending, V, Stats, status) like gesvd."""
    G = _f64F(G)
    Q, R = np.linalg.qr(G, mode="reduced")
    R = np.triu(R)
    kw = dict(kw)
    kw["want_vectors"] = True
    kw.setdefault("inner_max_sweeps", 2)   # on R^T: the same sweeps with half the inner work
    if transpose:
        UX, s, W, st, status = gesvd(np.asfortranarray(R.T), b=b, **kw)
        return np.asfortranarray(Q @ W), s, UX, st, status
    UR, s, VR, st, status = gesvd(np.asfortranarray(R), b=b, **kw)
    return np.asfortranarray(Q @ UR), s, VR, st, status


# ---------------------------------------------------------------- split precision
def split_bf16(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """hi = bf16_rn(x), lo = bf16_rn(x - hi), both returned as float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    hi = np.empty_like(x)
    lo = np.empty_like(x)
    lib().oracle_split_bf16(x.size, x.ctypes.data_as(_FP), hi.ctypes.data_as(_FP),
                            lo.ctypes.data_as(_FP))
    return hi, lo
