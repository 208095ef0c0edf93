"""C ABI checks that need no GPU: the library loads, exports every function
include/jacobi.h declares, and its host-side logic (the pair schedule of
Sec. 3 / Algorithm 3, parameter defaults, status strings) matches the oracle
and the header."""
from __future__ import annotations

import ctypes as C
import os
import re

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(jacobi_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def jg():
    from paper_2608_28952_gb300 import build
    build.build()
    import paper_2608_28952_gb300 as m
    m.lib()
    return m


def test_every_declared_symbol_is_exported(jg):
    names = _declared()
    assert {"jacobi_syev", "jacobi_gesvd", "jacobi_params_default"} <= names
    L = C.CDLL(jg.LIB_PATH)
    for n in sorted(names):
        assert hasattr(L, n), n
    assert names == set(jg.SIGNATURES), names ^ set(jg.SIGNATURES)


def test_params_default_matches_header(jg):
    p = jg.params()
    assert p.b == 32 and p.max_sweeps == 60 and p.inner_max_sweeps == 0  # 0 = automatic
    assert p.tol == 1e-14 and p.inner_tol == 4 * 2.0 ** -53
    assert p.precision == jg.PREC_FP64 and p.conv == jg.CONV_OFF_ABS
    assert p.want_vectors == 1 and p.warm_start == 0 and p.pivot_order == 1
    assert p.fp64_products == 0 and p.svd_qr == 0   # DFMA products, the direct one-sided SVD


def test_status_strings(jg):
    assert jg.status_string(0) == "converged"
    assert "max_sweeps" in jg.status_string(3)
    assert "non-finite" in jg.status_string(jg.ERR_NONFINITE)
    assert "invalid" in jg.status_string(-2)


@pytest.mark.parametrize("kind", [oracle.ORDER_ROUND_ROBIN, oracle.ORDER_ANTI_DIAGONAL])
def test_library_schedule_equals_oracle_schedule(jg, kind):
    for N in range(2, 70):
        if kind == oracle.ORDER_ROUND_ROBIN and N % 2:
            with pytest.raises(ValueError):
                jg.jacobi_ordering_table(kind, N)
            continue
        assert jg.jacobi_ordering_table(kind, N) == oracle.ordering(kind, N)


def test_invalid_schedule_arguments(jg):
    with pytest.raises(ValueError):
        jg.jacobi_ordering_table(0, 1)
    with pytest.raises(ValueError):
        jg.jacobi_ordering_table(7, 8)


def _header_struct_fields(name):
    txt = open(os.path.join(ROOT, "include", "jacobi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    m = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r";", txt)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype = decl.split()[0] if not decl.startswith("long long") else "long long"
        names = decl[len(ctype):].split(",")
        for nm in names:
            nm = nm.strip()
            arr = re.match(r"(\w+)\[(\d+)\]", nm)
            fields.append((arr.group(1), ctype, int(arr.group(2))) if arr else (nm, ctype, 1))
    return fields


@pytest.mark.parametrize("name", ["jacobi_params", "jacobi_stats"])
def test_binding_structs_mirror_the_header(jg, name):
    """Field names, order, C types and array lengths of the ctypes mirrors
    equal the header's, so the library never writes past the Python struct."""
    want = _header_struct_fields(name)
    got = getattr(jg, name)._fields_
    ctmap = {"int": C.c_int, "double": C.c_double, "long long": C.c_longlong}
    assert [f[0] for f in want] == [g[0] for g in got]
    for (nm, ct, ln), (gnm, gty) in zip(want, got):
        base = ctmap[ct]
        assert gty == (base * ln if ln > 1 else base), nm


@pytest.mark.parametrize("fn", ["jacobi_syev", "jacobi_syev_f32", "jacobi_syev_h"])
def test_syev_argument_errors_come_before_any_device_work(jg, fn):
    """The argument checks of the EVD entry points return -k (k the argument's
    position) or JACOBI_ERR_UNSUPPORTED before touching the device, so they
    run here without a GPU; the buffers are never dereferenced."""
    f = getattr(jg.lib(), fn)
    fake = C.c_void_p(0x1000)   # never dereferenced on these paths
    null = C.c_void_p(0)
    p = jg.params(b=16)

    def call(n, A, lda, w, Q, ldq, prm):
        return f(n, A, lda, w, Q, ldq, C.byref(prm), None, null)

    assert call(0, fake, 4, fake, fake, 4, p) == -1
    assert call(4, null, 4, fake, fake, 4, p) == -2
    assert call(4, fake, 3, fake, fake, 4, p) == -3
    assert call(4, fake, 4, null, fake, 4, p) == -4
    assert call(4, fake, 4, fake, null, 4, p) == -5
    assert call(4, fake, 4, fake, fake, 3, p) == -6
    if fn != "jacobi_syev_h":   # the host-buffer form validates its parameters on the device path
        for bad in (dict(b=0), dict(precision=9), dict(pivot_order=3), dict(tol=-1.0), dict(conv=4)):
            assert call(4, fake, 4, fake, fake, 4, jg.params(**{"b": 16, **bad})) == -7, bad
        assert call(4, fake, 4, fake, fake, 4, jg.params(b=129)) == jg.ERR_UNSUPPORTED


def test_batched_argument_errors_come_before_any_device_work(jg):
    """The batched calls validate sizes on the host before any CUDA call,
    with jacobi_plan_create_batched's codes: -4 batch, -5 h_m (one-sided:
    NULL or m n >= 2^31, the kernels' int index range), -6 h_n, -7 a
    leading dimension."""
    L = jg.lib()
    null = C.c_void_p(0)
    fake = C.c_void_p(0x1000)       # pointer arrays: never read on these paths
    p = jg.params()

    def ints(*v):
        return (C.c_int * len(v))(*v)

    def svd(batch, hm, hn, hld=None):
        return L.jacobi_gesvd_batched_f32(batch, hm, hn, fake, hld, fake, fake, None, C.byref(p),
                                          fake, None, null)

    def evd(batch, hn, hld=None):
        return L.jacobi_syev_batched(batch, hn, fake, hld, fake, fake, None, C.byref(p), fake, None, null)

    assert svd(0, ints(8), ints(4)) == -4
    assert svd(1, None, ints(4)) == -5
    assert svd(1, ints(1 << 26), ints(64)) == -5           # m n = 2^32
    assert svd(2, ints(100, 40000000), ints(10, 60)) == -5  # one matrix past the int range
    assert svd(1, ints(8), None) == -6
    assert svd(1, ints(8), ints(9)) == -6                   # n > m
    assert svd(1, ints(8), ints(0)) == -6
    assert svd(1, ints(8), ints(4), ints(7)) == -7          # ldg < m
    assert evd(0, ints(4)) == -4
    assert evd(1, None) == -6
    assert evd(1, ints(513)) == -6
    assert evd(1, ints(5), ints(4)) == -7


@pytest.mark.parametrize("fn", ["jacobi_syev", "jacobi_syev_f32", "jacobi_gesvd"])
def test_workspace_fault_injection_returns_alloc_before_any_launch(jg, fn, monkeypatch):
    """JACOBI_WORKSPACE_LIMIT caps one call's workspace: the drivers check the
    allocation before their first launch and return JACOBI_ERR_ALLOC, so this
    runs here without a GPU (the device pointers are never dereferenced)."""
    monkeypatch.setenv("JACOBI_WORKSPACE_LIMIT", "16")
    f = getattr(jg.lib(), fn)
    fake = C.c_void_p(0x1000)
    p = jg.params(b=16)
    st = jg.jacobi_stats()
    if fn == "jacobi_gesvd":
        rc = f(200, 64, fake, 200, fake, fake, 64, C.byref(p), C.byref(st), C.c_void_p(0))
    else:
        rc = f(64, fake, 64, fake, fake, 64, C.byref(p), C.byref(st), C.c_void_p(0))
    assert rc == jg.ERR_ALLOC
    assert st.status == jg.ERR_ALLOC


def test_binding_rejects_wrong_element_type_or_memory_space(jg):
    """The C entry points receive bare pointers: the binding refuses tensors
    of another element type or memory space before the call (here without a
    GPU: the check comes first)."""
    import torch
    A = torch.zeros(8, 8, dtype=torch.float64)
    w = torch.zeros(8, dtype=torch.float64)
    with pytest.raises(ValueError):
        jg.jacobi_syev(A, w, None)                       # host tensors to a device entry point
    with pytest.raises(TypeError):
        jg.jacobi_syev_h(A.float(), w, None)             # float32 to an FP64 entry point
    with pytest.raises(TypeError):
        jg.jacobi_syev_f32(A, w, None)                   # float64 to the FP32-storage entry point
    with pytest.raises(ValueError):
        jg.jacobi_syev_batched([A], [w], None, torch.zeros(1, dtype=torch.int32))
    with pytest.raises(TypeError):
        jg.jacobi_lowp_gemm(A, A, A)                     # the FP32 product given FP64 operands


def test_binding_rejects_buffers_too_small_for_the_call(jg):
    """A w shorter than n or a Q smaller than n x n would be written past its
    end by the library: the binding refuses it first (host tensors through
    the host-buffer entry points, so no GPU is involved)."""
    import torch
    A = torch.zeros(8, 8, dtype=torch.float64)
    with pytest.raises(ValueError):
        jg.jacobi_syev_h(A, torch.zeros(7, dtype=torch.float64), None)
    with pytest.raises(ValueError):
        jg.jacobi_syev_h(A, torch.zeros(8, dtype=torch.float64), torch.zeros(8, 7, dtype=torch.float64))
    with pytest.raises(ValueError):
        jg.jacobi_syev_h(A[:, :7], torch.zeros(8, dtype=torch.float64), None)
    G = torch.zeros(20, 6, dtype=torch.float64)
    with pytest.raises(ValueError):
        jg.jacobi_gesvd_h(G, torch.zeros(5, dtype=torch.float64), None)
    with pytest.raises(ValueError):
        jg.jacobi_gesvd_h(G, torch.zeros(6, dtype=torch.float64), torch.zeros(6, 5, dtype=torch.float64))


def test_noalloc_argument_checks_come_before_any_device_work(jg):
    """jacobi_syev_step_noalloc checks its parameters as jacobi_syev_step does
    (-6 for an invalid one) and refuses, with JACOBI_ERR_UNSUPPORTED, what its
    fixed array does not hold (orders above 768, b above 128, emulated FP64
    products, the QRCP pivoting step) before any CUDA call."""
    f = jg.lib().jacobi_syev_step_noalloc
    fake = C.c_void_p(0x1000)   # never dereferenced on these paths
    null = C.c_void_p(0)

    def call(np_, A, lda, Q, ldq, prm):
        return f(np_, A, lda, Q, ldq, C.byref(prm), 0, null)

    for bad in (dict(b=0), dict(ordering=3), dict(tol=-1.0), dict(conv=5), dict(pivot_order=4),
                dict(precision=11), dict(inner_max_sweeps=-1)):
        assert call(64, fake, 64, fake, 64, jg.params(**{"b": 8, **bad})) == -6, bad
    for unsup in (dict(precision=jg.PREC_FP64_EMU), dict(precision=jg.PREC_MIXED_BF16X3),
                  dict(precision=jg.PREC_MIXED_TF32), dict(fp64_products=1), dict(pivot_order=2),
                  dict(b=129)):
        assert call(64, fake, 64, fake, 64, jg.params(**{"b": 8, **unsup})) == jg.ERR_UNSUPPORTED, unsup
    assert call(1024, fake, 1024, fake, 1024, jg.params(b=64)) == jg.ERR_UNSUPPORTED
    assert call(60, fake, 64, fake, 64, jg.params(b=8)) == -1     # np not a multiple of b
    assert call(24, fake, 24, fake, 24, jg.params(b=8)) == -1     # N = 3 blocks: odd
    assert call(64, null, 64, fake, 64, jg.params(b=8)) == -2
    assert call(64, fake, 63, fake, 64, jg.params(b=8)) == -3
    assert call(64, fake, 64, fake, 63, jg.params(b=8)) == -5


def test_wait_selftest_argument_checks(jg):
    """The self-test of the bounded wait checks its arguments on the host."""
    L = jg.lib()
    assert L.jacobi_wait_selftest(2, 10.0, C.c_void_p(0)) == -1
    assert L.jacobi_wait_selftest(0, 0.5, C.c_void_p(0)) == -2
    assert L.jacobi_wait_selftest(0, 5000.0, C.c_void_p(0)) == -2
    assert L.jacobi_wait_selftest(1, float("nan"), C.c_void_p(0)) == -2
