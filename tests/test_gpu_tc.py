"""Tensor-core split-precision GEMM (tcgen05, kind::f16) against its exact
model from the oracle: every operand value x enters as hi = bf16(x),
lo = bf16(x - hi) (oracle.split_bf16), every product as hi*hi + hi*lo +
lo*hi; the model sums these in FP64, the tensor cores in FP32, so the bound
is the FP32 accumulation error 2 K u32 (|A| |B|) element-wise."""
from __future__ import annotations

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def jg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_28952_gb300 as m
    m.lib()
    return m


def _model(A, B):
    ah, al = oracle.split_bf16(A)
    bh, bl = oracle.split_bf16(B)
    ah, al, bh, bl = (x.astype(np.float64) for x in (ah, al, bh, bl))
    return ah @ bh + ah @ bl + al @ bh


@pytest.mark.parametrize("M,N,K,trans", [(128, 128, 32, False), (128, 128, 256, False),
                                          (300, 200, 100, False), (256, 384, 77, True),
                                          (1, 5, 3, False), (129, 130, 33, True)])
def test_lowp_gemm_matches_split_model(jg, M, N, K, trans):
    import torch
    r = np.random.default_rng(M * 1000 + N + K)
    A = r.standard_normal((K, M) if trans else (M, K)).astype(np.float32)
    B = r.standard_normal((K, N)).astype(np.float32)
    Ad = jg.colmajor(A, device="cuda", dtype=torch.float32)
    Bd = jg.colmajor(B, device="cuda", dtype=torch.float32)
    Cd = jg.colmajor_empty(M, N, torch.float32, "cuda")
    assert jg.jacobi_lowp_gemm(Ad, Bd, Cd, transA=trans) == 0
    C = Cd.cpu().numpy().astype(np.float64)
    Aop = A.T if trans else A
    want = _model(Aop, B)
    bound = 2 * K * U32 * (np.abs(Aop).astype(np.float64) @ np.abs(B).astype(np.float64)) + 1e-30
    assert np.all(np.abs(C - want) <= bound), np.max(np.abs(C - want) / bound)
    # and close to the exact product: the split keeps ~16 bits per operand
    exact = Aop.astype(np.float64) @ B.astype(np.float64)
    assert np.all(np.abs(C - exact) <= 2 * K * U32 * (np.abs(Aop) @ np.abs(B)) + 2.0 ** -15 * (np.abs(Aop) @ np.abs(B)))
