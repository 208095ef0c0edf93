"""GB300 (sm_103a) blocked Jacobi: symmetric EVD and one-sided SVD.

Thin ctypes binding over the C ABI in ``include/jacobi.h`` (library
``_build/libjacobi_gb300.so``, built by ``build.py``).  Every step of the
computation runs in the library's CUDA kernels; this module only marshals
arguments.  PyTorch provides device memory and streams.

The same names as the C ABI are exported (``jacobi_syev``, ``jacobi_gesvd``,
...), each taking column-major tensors; ``syev`` / ``gesvd`` are convenience
wrappers that allocate the outputs.  If the library is missing the import of
any entry point raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libjacobi_gb300.so")

ORDER_ROUND_ROBIN = 0
ORDER_ANTI_DIAGONAL = 1
PREC_FP64 = 0
PREC_FP32 = 1
PREC_MIXED_BF16X3 = 2
PREC_MIXED_FP16X3 = 3
PREC_MIXED_TF32 = 4
PREC_FP64_EMU = 5
CONV_OFF_ABS = 0
CONV_REL = 1
ERR_NONFINITE = -100
ERR_CUDA = -101
ERR_ALLOC = -102
ERR_TIMEOUT = -103
ERR_UNSUPPORTED = -104


class jacobi_params(C.Structure):
    _fields_ = [("b", C.c_int), ("ordering", C.c_int), ("max_sweeps", C.c_int),
                ("inner_max_sweeps", C.c_int), ("tol", C.c_double), ("inner_tol", C.c_double),
                ("precision", C.c_int), ("conv", C.c_int), ("want_vectors", C.c_int),
                ("warm_start", C.c_int), ("switch_tol", C.c_double), ("refine_steps", C.c_int),
                ("pivot_order", C.c_int), ("fp64_products", C.c_int), ("svd_qr", C.c_int)]


class jacobi_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("sweeps", C.c_int), ("sweeps_lowp", C.c_int),
                ("stalled", C.c_int), ("steps", C.c_longlong), ("pair_solves", C.c_longlong),
                ("rotations", C.c_longlong), ("inner_sweeps", C.c_longlong),
                ("norm_fro", C.c_double), ("off_initial", C.c_double), ("off_final", C.c_double),
                ("off_hist", C.c_double * 64), ("ms_total", C.c_double),
                ("ms_pivot", C.c_double), ("ms_update", C.c_double),
                ("launches", C.c_longlong), ("pivot_launches", C.c_longlong),
                ("update_launches", C.c_longlong),
                ("flops_fp64", C.c_double), ("flops_update", C.c_double),
                ("flops_fp32", C.c_double), ("flops_lowp", C.c_double),
                ("ms_lowp", C.c_double), ("ms_refine", C.c_double),
                ("ms_pivot_lowp", C.c_double), ("ms_update_lowp", C.c_double),
                ("flops_refine", C.c_double), ("ms_precond", C.c_double),
                ("flops_precond", C.c_double), ("rel_final", C.c_double),
                ("rel_hist", C.c_double * 64)]


@dataclass
class Stats:
    status: int
    sweeps: int
    sweeps_lowp: int
    stalled: int
    steps: int
    pair_solves: int
    rotations: int
    inner_sweeps: int
    norm_fro: float
    off_initial: float
    off_final: float
    ms_total: float
    ms_pivot: float
    ms_update: float
    launches: int
    pivot_launches: int
    update_launches: int
    flops_fp64: float
    flops_update: float
    flops_fp32: float
    flops_lowp: float
    ms_lowp: float
    ms_refine: float
    ms_pivot_lowp: float
    ms_update_lowp: float
    flops_refine: float
    ms_precond: float
    flops_precond: float
    rel_final: float = 0.0
    off_hist: list = field(default_factory=list)
    rel_hist: list = field(default_factory=list)


def _stats(s: jacobi_stats) -> Stats:
    return Stats(s.status, s.sweeps, s.sweeps_lowp, s.stalled, s.steps, s.pair_solves,
                 s.rotations, s.inner_sweeps, s.norm_fro, s.off_initial, s.off_final,
                 s.ms_total, s.ms_pivot, s.ms_update, s.launches, s.pivot_launches,
                 s.update_launches, s.flops_fp64, s.flops_update, s.flops_fp32, s.flops_lowp,
                 s.ms_lowp, s.ms_refine, s.ms_pivot_lowp, s.ms_update_lowp, s.flops_refine,
                 s.ms_precond, s.flops_precond, s.rel_final,
                 list(s.off_hist)[: max(0, min(64, s.sweeps))],
                 list(s.rel_hist)[: max(0, min(64, s.sweeps))])


# Every symbol include/jacobi.h declares, with its ctypes signature.
_I, _D, _P = C.c_int, C.c_double, C.c_void_p
_PP = C.POINTER(jacobi_params)
_SP = C.POINTER(jacobi_stats)
SIGNATURES = {
    "jacobi_params_default": (_I, [_PP]),
    "jacobi_status_string": (C.c_char_p, [_I]),
    "jacobi_syev": (_I, [_I, _P, _I, _P, _P, _I, _PP, _SP, _P]),
    "jacobi_syev_h": (_I, [_I, _P, _I, _P, _P, _I, _PP, _SP, _P]),
    "jacobi_syev_f32": (_I, [_I, _P, _I, _P, _P, _I, _PP, _SP, _P]),
    "jacobi_gesvd": (_I, [_I, _I, _P, _I, _P, _P, _I, _PP, _SP, _P]),
    "jacobi_gesvd_h": (_I, [_I, _I, _P, _I, _P, _P, _I, _PP, _SP, _P]),
    "jacobi_ordering_table": (_I, [_I, _I, _P, _P]),
    "jacobi_syev_step": (_I, [_I, _P, _I, _P, _I, _PP, _I, _P]),
    "jacobi_gesvd_step": (_I, [_I, _I, _P, _I, _P, _I, _PP, _I, C.POINTER(C.c_double), _P]),
    "jacobi_syev_batched": (_I, [_I, _P, _P, _P, _P, _P, _P, _PP, _P, _SP, _P]),
    "jacobi_syev_batched_f32": (_I, [_I, _P, _P, _P, _P, _P, _P, _PP, _P, _SP, _P]),
    "jacobi_gesvd_batched_f32": (_I, [_I, _P, _P, _P, _P, _P, _P, _P, _PP, _P, _SP, _P]),
    "jacobi_plan_create_batched": (_I, [C.POINTER(_P), _I, _I, _I, _P, _P, _P, _P, _PP, _P]),
    "jacobi_plan_autotune": (_I, [_P, _P, _P, _P, _P, _P]),
    "jacobi_plan_execute": (_I, [_P, _P, _P, _P, _P, _SP, _P]),
    "jacobi_plan_shape": (_I, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "jacobi_plan_blocking": (_I, [_P, C.POINTER(_I), C.POINTER(_I)]),
    "jacobi_plan_destroy": (None, [_P]),
    "jacobi_syev_step_noalloc": (_I, [_I, _P, _I, _P, _I, _PP, _I, _P]),
    "jacobi_lowp_gemm": (_I, [_I, _I, _I, _P, _I, _I, _P, _I, _P, _I, _P]),
    "jacobi_syev_step_lowp": (_I, [_I, _P, _I, _P, _I, _PP, _I, _P]),
    "jacobi_f64emu_gemm": (_I, [_I, _I, _I, _P, _I, _I, _P, _I, _P, _I, _P]),
    "jacobi_rotation_params": (_I, [_I, _P, _P, _P, _D, _P, _P]),
    "jacobi_off_norm": (_I, [_I, _P, _I, _I, C.POINTER(C.c_double), _P]),
    "jacobi_wait_selftest": (_I, [_I, _D, _P]),
}

_LIB = None


def lib() -> C.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA extension {LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


# ------------------------------------------------------------------ marshalling helpers
def params(**kw) -> jacobi_params:
    """Default parameters with keyword overrides (names as in jacobi_params)."""
    p = jacobi_params()
    lib().jacobi_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def status_string(code: int) -> str:
    return lib().jacobi_status_string(code).decode()


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _colmajor_ld(t) -> int:
    """Leading dimension of a column-major 2-D tensor (stride(0) == 1)."""
    if t.dim() != 2 or (t.stride(0) != 1 and t.shape[0] > 1):
        raise ValueError("expected a column-major 2-D tensor (stride(0) == 1)")
    return max(t.stride(1), t.shape[0], 1)


def colmajor(x, device=None, dtype=None):
    """Column-major copy of a 2-D tensor or array (as a torch tensor)."""
    import torch
    t = torch.as_tensor(x)
    if dtype is not None:
        t = t.to(dtype)
    if device is not None:
        t = t.to(device)
    return t.t().contiguous().t()


def colmajor_empty(rows, cols, dtype, device):
    import torch
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _fits(rows: int, cols: int, *mats):
    """Raise when a matrix argument holds fewer than rows x cols elements in
    its column-major layout (the library would read or write past it)."""
    for t in mats:
        if t is None:
            continue
        if t.dim() != 2 or t.shape[0] < rows or t.shape[1] < cols:
            raise ValueError(f"expected at least a {rows} x {cols} matrix, got {tuple(t.shape)}")


def _holds(count: int, *vecs):
    for t in vecs:
        if t is not None and t.numel() < count:
            raise ValueError(f"expected at least {count} elements, got {t.numel()}")


def _need(dtype: str, device: str, *tensors):
    """Raise before the C call when a tensor's element type or memory space is
    not the one the entry point reads: the C side receives bare pointers and
    cannot tell (a float32 buffer read as float64 runs past its end)."""
    import torch
    want = getattr(torch, dtype)
    for t in tensors:
        if t is None:
            continue
        if t.dtype != want:
            raise TypeError(f"expected {dtype} tensors, got {t.dtype}")
        if t.device.type != device:
            raise ValueError(f"expected tensors on {device}, got {t.device}")


# ------------------------------------------------------------------ C-ABI names
def jacobi_syev(A, w, Q, p: jacobi_params | None = None, stream=None):
    """C ``jacobi_syev`` on CUDA tensors: A (n x n, column-major, float64,
    overwritten by D), w (n), Q (n x n column-major or None).
    Returns (status, Stats)."""
    _need("float64", "cuda", A, w, Q)
    n = A.shape[0]
    _fits(n, n, A, Q)
    _holds(n, w)
    st = jacobi_stats()
    rc = lib().jacobi_syev(n, _ptr(A), _colmajor_ld(A), _ptr(w), _ptr(Q),
                           _colmajor_ld(Q) if Q is not None else n,
                           C.byref(p) if p is not None else None, C.byref(st), _stream_ptr(stream))
    return rc, _stats(st)


def jacobi_syev_h(A, w, Q, p: jacobi_params | None = None, stream=None):
    """C ``jacobi_syev_h`` on HOST buffers (torch CPU tensors, ideally
    pinned): same layout as jacobi_syev."""
    _need("float64", "cpu", A, w, Q)
    n = A.shape[0]
    _fits(n, n, A, Q)
    _holds(n, w)
    st = jacobi_stats()
    rc = lib().jacobi_syev_h(n, _ptr(A), _colmajor_ld(A), _ptr(w), _ptr(Q),
                             _colmajor_ld(Q) if Q is not None else n,
                             C.byref(p) if p is not None else None, C.byref(st),
                             _stream_ptr(stream))
    return rc, _stats(st)


def jacobi_syev_f32(A, w, Q, p: jacobi_params | None = None, stream=None):
    """C ``jacobi_syev_f32`` on CUDA float32 tensors: same layout as
    jacobi_syev (A column-major n x n, overwritten by D; w (n); Q or None)."""
    _need("float32", "cuda", A, w, Q)
    n = A.shape[0]
    _fits(n, n, A, Q)
    _holds(n, w)
    st = jacobi_stats()
    rc = lib().jacobi_syev_f32(n, _ptr(A), _colmajor_ld(A), _ptr(w), _ptr(Q),
                               _colmajor_ld(Q) if Q is not None else n,
                               C.byref(p) if p is not None else None, C.byref(st),
                               _stream_ptr(stream))
    return rc, _stats(st)


def jacobi_gesvd(G, sigma, V, p: jacobi_params | None = None, stream=None):
    """C ``jacobi_gesvd`` on CUDA tensors: G (m x n column-major float64, out:
    U), sigma (n), V (n x n or None).  Returns (status, Stats)."""
    _need("float64", "cuda", G, sigma, V)
    m, n = G.shape
    _fits(n, n, V)
    _holds(n, sigma)
    st = jacobi_stats()
    rc = lib().jacobi_gesvd(m, n, _ptr(G), _colmajor_ld(G), _ptr(sigma), _ptr(V),
                            _colmajor_ld(V) if V is not None else n,
                            C.byref(p) if p is not None else None, C.byref(st), _stream_ptr(stream))
    return rc, _stats(st)


def jacobi_gesvd_h(G, sigma, V, p: jacobi_params | None = None, stream=None):
    _need("float64", "cpu", G, sigma, V)
    m, n = G.shape
    _fits(n, n, V)
    _holds(n, sigma)
    st = jacobi_stats()
    rc = lib().jacobi_gesvd_h(m, n, _ptr(G), _colmajor_ld(G), _ptr(sigma), _ptr(V),
                              _colmajor_ld(V) if V is not None else n,
                              C.byref(p) if p is not None else None, C.byref(st),
                              _stream_ptr(stream))
    return rc, _stats(st)


def jacobi_off_norm(A, want_rel: bool = True, stream=None):
    """C ``jacobi_off_norm`` on a column-major float64 CUDA tensor A (n x n):
    returns (status, off(A), ||A||_F, relative measure)."""
    _need("float64", "cuda", A)
    n = A.shape[0]
    _fits(n, n, A)
    out = (C.c_double * 3)()
    rc = lib().jacobi_off_norm(n, _ptr(A), _colmajor_ld(A), int(want_rel), out, _stream_ptr(stream))
    return rc, out[0], out[1], out[2]


def jacobi_syev_step(A, Q, step: int, p: jacobi_params | None = None, stream=None):
    """C ``jacobi_syev_step``: one parallel step in place on the full
    symmetric np x np column-major CUDA tensor A (and Q or None)."""
    _need("float64", "cuda", A, Q)
    np_ = A.shape[0]
    _fits(np_, np_, A, Q)
    return lib().jacobi_syev_step(np_, _ptr(A), _colmajor_ld(A), _ptr(Q),
                                  _colmajor_ld(Q) if Q is not None else np_,
                                  C.byref(p) if p is not None else None, step,
                                  _stream_ptr(stream))


def jacobi_syev_step_noalloc(A, Q, step: int, p: jacobi_params | None = None, stream=None):
    """C ``jacobi_syev_step_noalloc``: ``jacobi_syev_step`` for callers that
    cannot allocate device memory (np <= 768, b <= 128); the library keeps its
    working buffers in one fixed device array instead."""
    _need("float64", "cuda", A, Q)
    np_ = A.shape[0]
    _fits(np_, np_, A, Q)
    return lib().jacobi_syev_step_noalloc(np_, _ptr(A), _colmajor_ld(A), _ptr(Q),
                                          _colmajor_ld(Q) if Q is not None else np_,
                                          C.byref(p) if p is not None else None, step,
                                          _stream_ptr(stream))


def jacobi_gesvd_step(G, V, step: int, p: jacobi_params | None = None, stream=None):
    """C ``jacobi_gesvd_step``: one one-sided step in place on G (m x np) and
    V (np x np or None).  Returns (status, relmax)."""
    _need("float64", "cuda", G, V)
    m, np_ = G.shape
    _fits(np_, np_, V)
    r = C.c_double(0.0)
    rc = lib().jacobi_gesvd_step(m, np_, _ptr(G), _colmajor_ld(G), _ptr(V),
                                 _colmajor_ld(V) if V is not None else np_,
                                 C.byref(p) if p is not None else None, step, C.byref(r),
                                 _stream_ptr(stream))
    return rc, r.value


def jacobi_lowp_gemm(A, B, C, transA: bool = False, stream=None):
    """C ``jacobi_lowp_gemm``: C = op(A) B (FP32, column-major CUDA tensors)
    on the tensor cores with bf16 hi/lo operand splits."""
    _need("float32", "cuda", A, B, C)
    K, N = B.shape
    M = C.shape[0]
    _fits(K, M, A if transA else None)
    _fits(M, K, None if transA else A)
    _fits(M, N, C)
    return lib().jacobi_lowp_gemm(M, N, K, _ptr(A), _colmajor_ld(A), int(transA), _ptr(B),
                                  _colmajor_ld(B), _ptr(C), _colmajor_ld(C), _stream_ptr(stream))


def jacobi_rotation_params(app, aqq, apq, tol: float, out, stream=None):
    """C ``jacobi_rotation_params``: for each triple, out[i] = (t, s, tau,
    rotate) as the FP64 pivot solves compute them, then the same four by the
    textbook formulas (contiguous FP64 CUDA tensors; out is count x 8)."""
    _need("float64", "cuda", app, aqq, apq, out)
    _holds(app.numel(), aqq, apq)
    _holds(8 * app.numel(), out)
    return lib().jacobi_rotation_params(app.numel(), _ptr(app), _ptr(aqq), _ptr(apq), float(tol), _ptr(out),
                                        _stream_ptr(stream))


def jacobi_f64emu_gemm(A, B, C, transA: bool = False, stream=None):
    """C ``jacobi_f64emu_gemm``: C = op(A) B (FP64, column-major CUDA tensors,
    K <= 256) on the tensor cores from eight bf16 slices per operand."""
    _need("float64", "cuda", A, B, C)
    K, N = B.shape
    M = C.shape[0]
    _fits(K, M, A if transA else None)
    _fits(M, K, None if transA else A)
    _fits(M, N, C)
    return lib().jacobi_f64emu_gemm(M, N, K, _ptr(A), _colmajor_ld(A), int(transA), _ptr(B),
                                    _colmajor_ld(B), _ptr(C), _colmajor_ld(C), _stream_ptr(stream))


def jacobi_syev_step_lowp(A, Q, step: int, p: jacobi_params | None = None, stream=None):
    """C ``jacobi_syev_step_lowp``: one low-precision step of the mixed form
    in place on FP32 column-major CUDA tensors A (np x np, symmetric) and Q
    (or None); p.precision must be JACOBI_PREC_MIXED_BF16X3."""
    _need("float32", "cuda", A, Q)
    np_ = A.shape[0]
    _fits(np_, np_, A, Q)
    return lib().jacobi_syev_step_lowp(np_, _ptr(A), _colmajor_ld(A), _ptr(Q),
                                       _colmajor_ld(Q) if Q is not None else np_,
                                       C.byref(p) if p is not None else None, step,
                                       _stream_ptr(stream))


def jacobi_wait_selftest(arrive: bool, limit_ms: float, stream=None) -> int:
    """C ``jacobi_wait_selftest``: one CTA waits on an mbarrier with the
    tensor-core kernels' bounded wait (limit_ms); 0 when arrive, else
    JACOBI_ERR_TIMEOUT once the limit has passed."""
    return lib().jacobi_wait_selftest(int(arrive), float(limit_ms), _stream_ptr(stream))


def jacobi_ordering_table(kind: int, N: int):
    """The library's pair schedule: list of steps, each a list of (I, J)."""
    import numpy as np
    pairs = np.zeros(max(1, N * (N - 1)), dtype=np.int32)
    ptr = np.zeros(N + 1, dtype=np.int32)
    S = lib().jacobi_ordering_table(kind, N, pairs.ctypes.data, ptr.ctypes.data)
    if S < 0:
        raise ValueError("bad ordering arguments")
    return [[(int(pairs[2 * e]), int(pairs[2 * e + 1])) for e in range(ptr[s], ptr[s + 1])]
            for s in range(S)]


# ------------------------------------------------------------------ convenience
def syev(A, b: int = 32, *, want_vectors: bool = True, stream=None, **kw):
    """Eigen-decomposition of the symmetric A (any 2-D tensor/array; only its
    lower triangle is read).  Returns (w, Q, D, Stats) as CUDA tensors
    (Q column-major, None without vectors); raises on an error status."""
    import torch
    dev = torch.device("cuda")
    Ad = colmajor(A, device=dev, dtype=torch.float64)
    n = Ad.shape[0]
    w = torch.empty(n, dtype=torch.float64, device=dev)
    Q = colmajor_empty(n, n, torch.float64, dev) if want_vectors else None
    p = params(b=b, want_vectors=int(want_vectors), **kw)
    rc, st = jacobi_syev(Ad, w, Q, p, stream)
    if rc < 0:
        raise RuntimeError(f"jacobi_syev: {rc} ({status_string(rc)})")
    return w, Q, Ad, st


def gesvd(G, b: int = 32, *, want_vectors: bool = True, stream=None, **kw):
    """One-sided Jacobi SVD of G (m x n, m >= n).  Returns (U, sigma, V, Stats)."""
    import torch
    dev = torch.device("cuda")
    Gd = colmajor(G, device=dev, dtype=torch.float64)
    m, n = Gd.shape
    s = torch.empty(n, dtype=torch.float64, device=dev)
    V = colmajor_empty(n, n, torch.float64, dev) if want_vectors else None
    p = params(b=b, want_vectors=int(want_vectors), **kw)
    rc, st = jacobi_gesvd(Gd, s, V, p, stream)
    if rc < 0:
        raise RuntimeError(f"jacobi_gesvd: {rc} ({status_string(rc)})")
    return Gd, s, V, st


# ------------------------------------------------------------------ batched forms
def _ptr_array(tensors):
    """Host array of device pointers (None -> NULL array)."""
    if tensors is None:
        return None
    arr = (C.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])
    return arr


def _int_array(vals):
    return (C.c_int * len(vals))(*[int(v) for v in vals])


class Plan:
    """Batched plan (jacobi_plan_*): kind 0 EVD, 1 one-sided SVD."""

    def __init__(self, kind, precision, n, m=None, lda=None, ldq=None, p=None, stream=None):
        self.kind, self.batch = kind, len(n)
        self._h = C.c_void_p()
        self._keep = [_int_array(n), _int_array(m) if m is not None else None,
                      _int_array(lda) if lda is not None else None,
                      _int_array(ldq) if ldq is not None else None]
        rc = lib().jacobi_plan_create_batched(C.byref(self._h), kind, precision, len(n),
                                              self._keep[1], self._keep[0], self._keep[2],
                                              self._keep[3], C.byref(p) if p is not None else None,
                                              _stream_ptr(stream))
        if rc != 0:
            raise RuntimeError(f"jacobi_plan_create_batched: {rc} ({status_string(rc)})")

    def autotune(self, X, y, Z, info, stream=None):
        rc = lib().jacobi_plan_autotune(self._h, _ptr_array(X), _ptr_array(y), _ptr_array(Z),
                                        C.c_void_p(info.data_ptr()), _stream_ptr(stream))
        if rc != 0:
            raise RuntimeError(f"jacobi_plan_autotune: {rc}")

    def execute(self, X, y, Z, info, stream=None):
        st = jacobi_stats()
        rc = lib().jacobi_plan_execute(self._h, _ptr_array(X), _ptr_array(y), _ptr_array(Z),
                                       C.c_void_p(info.data_ptr()), C.byref(st),
                                       _stream_ptr(stream))
        return rc, _stats(st)

    def shape(self):
        t, k, g = C.c_int(), C.c_int(), C.c_int()
        lib().jacobi_plan_shape(self._h, C.byref(t), C.byref(k), C.byref(g))
        return t.value, k.value, g.value

    def blocking(self):
        """(b, min_order): orders above min_order use the blocked method with
        block size b; at or below it, the unblocked solve (0, 0: no blocked
        route in this plan)."""
        b, mo = C.c_int(), C.c_int()
        lib().jacobi_plan_blocking(self._h, C.byref(b), C.byref(mo))
        return b.value, mo.value

    def close(self):
        if self._h:
            lib().jacobi_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def jacobi_syev_batched(As, ws, Qs, info, p=None, stream=None, f32=False):
    """C ``jacobi_syev_batched`` / ``_f32`` on lists of column-major CUDA tensors."""
    _need("float32" if f32 else "float64", "cuda", *As, *ws, *(Qs or []))
    _need("int32", "cuda", info)
    n = [a.shape[0] for a in As]
    st = jacobi_stats()
    f = lib().jacobi_syev_batched_f32 if f32 else lib().jacobi_syev_batched
    rc = f(len(As), _int_array(n), _ptr_array(As), _int_array([_colmajor_ld(a) for a in As]),
           _ptr_array(ws), _ptr_array(Qs),
           _int_array([_colmajor_ld(q) for q in Qs]) if Qs is not None else None,
           C.byref(p) if p is not None else None, C.c_void_p(info.data_ptr()), C.byref(st),
           _stream_ptr(stream))
    return rc, _stats(st)


def jacobi_gesvd_batched_f32(Gs, sigmas, Vs, info, p=None, stream=None):
    """C ``jacobi_gesvd_batched_f32`` on lists of column-major CUDA tensors."""
    _need("float32", "cuda", *Gs, *sigmas, *(Vs or []))
    _need("int32", "cuda", info)
    m = [g.shape[0] for g in Gs]
    n = [g.shape[1] for g in Gs]
    st = jacobi_stats()
    rc = lib().jacobi_gesvd_batched_f32(
        len(Gs), _int_array(m), _int_array(n), _ptr_array(Gs),
        _int_array([_colmajor_ld(g) for g in Gs]), _ptr_array(sigmas), _ptr_array(Vs),
        _int_array([_colmajor_ld(v) for v in Vs]) if Vs is not None else None,
        C.byref(p) if p is not None else None, C.c_void_p(info.data_ptr()), C.byref(st),
        _stream_ptr(stream))
    return rc, _stats(st)
