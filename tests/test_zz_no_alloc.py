"""The allocation-free single step, jacobi_syev_step_noalloc.

Some callers cannot allocate device memory -- code inside a framework that
owns the whole device through its own memory pool, or a latency-critical loop
that cannot absorb an allocation.  For them the library offers a variant of
the one-step entry point whose working buffers live in a fixed device array.
These tests call it through the C ABI and compare it with the allocating
jacobi_syev_step on the same inputs, two calls in a row with different sizes,
block sizes and orderings (so a stale buffer from the first call would show
in the second), plus its size limit.  Its pivot solves always run one CTA
per pair; with the allocating step forced to one CTA per pair as well
(JACOBI_PIVOT_CLUSTER=1) the two agree bit for bit, otherwise to rounding
(1e-13 of the largest entry, the step-parity tolerance).  This file is
collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

import jacobi_inputs as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_28952_gb300 as m
    m.lib()
    return m


def _case(np_, seed):
    d = np.linspace(1.0, 2.0 * np_, np_)
    return np.asfortranarray(np.diag(d) + 0.05 * gen.sym_gaussian(np_, seed))


def _both(jg, A0, step, p):
    import torch
    dev = "cuda"
    A1 = jg.colmajor(A0, device=dev, dtype=torch.float64)
    Q1 = jg.colmajor(np.eye(A0.shape[0]), device=dev, dtype=torch.float64)
    A2, Q2 = A1.clone().t().contiguous().t(), Q1.clone().t().contiguous().t()
    assert jg.jacobi_syev_step(A1, Q1, step, p) == 0
    assert jg.jacobi_syev_step_noalloc(A2, Q2, step, p) == 0
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (A1, Q1, A2, Q2)]


def test_noalloc_step_matches_allocating_step_twice_in_a_row(jg):
    # first call: n = 512, b = 64 (pivots in shared memory), round-robin
    A0 = _case(512, 4401)
    a1, q1, a2, q2 = _both(jg, A0, 3, jg.params(b=64))
    scale = np.abs(A0).max()
    assert np.abs(a2 - a1).max() <= 1e-13 * scale
    assert np.abs(q2 - q1).max() <= 1e-13
    assert not np.array_equal(a2, A0)  # the step did something
    # second call: n = 256, b = 128 (pivots in global scratch), Algorithm 3
    A0 = _case(256, 4402)
    a1, q1, a2, q2 = _both(jg, A0, 1, jg.params(b=128, ordering=jg.ORDER_ANTI_DIAGONAL))
    assert np.abs(a2 - a1).max() <= 1e-13 * np.abs(A0).max()
    assert np.abs(q2 - q1).max() <= 1e-13


def test_noalloc_without_q_and_size_limit(jg):
    import torch
    A0 = _case(96, 4403)
    A1 = jg.colmajor(A0, device="cuda", dtype=torch.float64)
    A2 = A1.clone().t().contiguous().t()
    assert jg.jacobi_syev_step(A1, None, 2, jg.params(b=16)) == 0
    assert jg.jacobi_syev_step_noalloc(A2, None, 2, jg.params(b=16)) == 0
    assert np.abs(A2.cpu().numpy() - A1.cpu().numpy()).max() <= 1e-13 * np.abs(A0).max()
    big = jg.colmajor(np.eye(1024), device="cuda", dtype=torch.float64)
    assert jg.jacobi_syev_step_noalloc(big, None, 0, jg.params(b=64)) == jg.ERR_UNSUPPORTED


def test_noalloc_step_is_bitwise_the_one_cta_step(jg, monkeypatch):
    """With one CTA per pair on both sides the two steps are the same
    arithmetic: equal bit for bit.  Cases: round-robin, and an even step of
    Algorithm 3 with N = 8 blocks, which leaves two blocks out (the frozen
    entry of the schedule), with the k = 256 pivots in global scratch."""
    monkeypatch.setenv("JACOBI_PIVOT_CLUSTER", "1")
    for np_, b, ordering, step, seed in ((512, 64, 0, 5, 4404), (512, 64, 1, 2, 4405),
                                         (768, 128, 1, 4, 4406), (96, 8, 1, 6, 4407)):
        A0 = _case(np_, seed)
        a1, q1, a2, q2 = _both(jg, A0, step, jg.params(b=b, ordering=ordering))
        assert np.array_equal(a1, a2) and np.array_equal(q1, q2), (np_, b, ordering, step)
        assert not np.array_equal(a2, A0)


def test_noalloc_rejects_modes_it_has_no_buffers_for(jg):
    """Emulated products and the QRCP pivoting step need buffers the fixed
    array does not hold: JACOBI_ERR_UNSUPPORTED, the caller's A untouched."""
    import torch
    A0 = _case(64, 4408)
    A = jg.colmajor(A0, device="cuda", dtype=torch.float64)
    for kw in (dict(precision=jg.PREC_FP64_EMU), dict(precision=jg.PREC_MIXED_BF16X3),
               dict(fp64_products=1), dict(pivot_order=2)):
        assert jg.jacobi_syev_step_noalloc(A, None, 0, jg.params(b=8, **kw)) == jg.ERR_UNSUPPORTED, kw
    assert np.array_equal(A.cpu().numpy(), A0)
