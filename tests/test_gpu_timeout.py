"""The timeout path of the tensor-core kernels' bounded mbarrier wait, on the
GPU and without a fault: a wait on a barrier that nothing arrives at runs
out after the given limit and the call returns JACOBI_ERR_TIMEOUT; the tensor
memory it held is freed and the context stays usable, so the next
tensor-core call (a split-precision GEMM and an FP64-accurate emulated GEMM)
succeeds with correct results."""
from __future__ import annotations

import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_28952_gb300 as m
    m.lib()
    return m


def _gemms_still_work(jg):
    import torch
    r = np.random.default_rng(77)
    A = r.standard_normal((256, 96))
    B = r.standard_normal((96, 200))
    C32 = jg.colmajor_empty(256, 200, torch.float32, "cuda")
    assert jg.jacobi_lowp_gemm(jg.colmajor(A, "cuda", torch.float32), jg.colmajor(B, "cuda", torch.float32), C32) == 0
    ref = A.astype(np.float32).astype(np.float64) @ B.astype(np.float32).astype(np.float64)
    assert np.abs(C32.cpu().numpy() - ref).max() <= 1e-4 * np.abs(ref).max()
    C64 = jg.colmajor_empty(256, 200, torch.float64, "cuda")
    assert jg.jacobi_f64emu_gemm(jg.colmajor(A, "cuda", torch.float64), jg.colmajor(B, "cuda", torch.float64), C64) == 0
    assert np.abs(C64.cpu().numpy() - A @ B).max() <= 1e-13 * np.abs(A @ B).max()


def test_wait_that_nothing_arrives_at_times_out_and_leaves_the_context_usable(jg):
    import torch
    torch.cuda.synchronize()
    assert jg.jacobi_wait_selftest(True, 50.0) == 0          # the barrier completes: no timeout
    t0 = time.perf_counter()
    rc = jg.jacobi_wait_selftest(False, 50.0)
    dt = time.perf_counter() - t0
    assert rc == jg.ERR_TIMEOUT
    assert 0.045 <= dt <= 2.0, dt                              # it waited about the limit, then gave up
    _gemms_still_work(jg)
    # a second timeout in a row, then a normal solve
    assert jg.jacobi_wait_selftest(False, 10.0) == jg.ERR_TIMEOUT
    assert jg.jacobi_wait_selftest(True, 10.0) == 0
    _gemms_still_work(jg)
