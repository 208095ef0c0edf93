// k_tc.cu -- split-precision rotation-update GEMMs on the 5th-generation
// tensor cores (tcgen05) of sm_103a.
//
// C[M x N] = Aop[M x K] * Bop[K x N] from FP32 (or FP64) operands: each
// operand value x is split into hi = bf16(x) and lo = bf16(x - hi), and the
// product is formed as hi*hi + hi*lo + lo*hi (lo*lo dropped) by three
// tcgen05.mma.kind::f16 instructions per K step, accumulating in FP32 in
// tensor memory (TMEM).  One CTA computes a 128 x 128 tile:
//   * 128 threads stage a 128 x 32 slice of Aop and a 32 x 128 slice of Bop
//     per K chunk, split them, and store the four bf16 tiles in shared memory
//     in the tensor cores' canonical K-major layout without swizzle (8 x 8
//     "core matrices" of 128 contiguous bytes);
//   * one thread issues the 6 MMAs of the chunk (2 K steps of 16 x 3
//     products) and commits them to the chunk's mbarrier; the chunk's buffers
//     are reused two chunks later, after that barrier completes, so staging
//     of chunk c+1 overlaps the MMAs of chunk c;
//   * the epilogue reads the 128 x 128 FP32 accumulator out of TMEM
//     (tcgen05.ld, warp w reads lanes 32w..32w+31 = rows) and stores it.
// Every wait on an mbarrier is bounded (about 2 s by the global timer); a wait
// that runs out sets the error word, skips the remaining work, and the CTA
// still frees its TMEM before returning.
//
// Operands are read through loader functors (index maps), so the same tile
// code serves the plain GEMM, the pair-column update X(:,P) <- X(:,P) V_P
// and the pair-row update X(P,:) <- V_P^T X(P,:) of the mixed-precision
// sweeps.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "tc_common.cuh"

namespace jac {

// C tile (128 x 128 at tile origin) = Aop * Bop over K; fa(m, k) and fb(k, n)
// return FP32 operand values (0 outside the operands); st(m, n, v) stores.
template <class FA, class FB, class ST>
__device__ void tc_gemm_tile(int K, FA fa, FB fb, ST st, TcErr err)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // 1024-byte aligned base for the operand tiles
    unsigned char* base = (unsigned char*)(((uintptr_t)tsm + 1023) & ~(uintptr_t)1023);

    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < 2; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TC_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = idesc_bf16(TC_BM, TC_BN);
    const int nchunks = (K + TC_BK - 1) / TC_BK;
    uint32_t uses[2] = {0, 0};

    for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        unsigned char* st_base = base + s * TC_STAGE_BYTES;
        // the MMAs that last read this stage (chunk c - 2) must be complete
        if (c >= 2) {
            if (!mbar_wait(smem_u32(&s_bar[s]), (uses[s] - 1) & 1)) {
                if (tid == 0) s_fail = 1;
            }
        }
        __syncthreads();
        if (s_fail) break;
        const int k0 = c * TC_BK;
        // stage Aop (128 x 32): thread -> rows, 32 values each
        for (int idx = tid; idx < TC_BM * TC_BK; idx += TC_T) {
            const int m = idx % TC_BM, kk = idx / TC_BM;
            const float x = (k0 + kk < K) ? fa(m, k0 + kk) : 0.f;
            __nv_bfloat16 h, l;
            split_bf16(x, h, l);
            const uint32_t o = tile_off(m, kk);
            *(__nv_bfloat16*)(st_base + o) = h;
            *(__nv_bfloat16*)(st_base + TC_TILE_BYTES + o) = l;
        }
        // stage Bop (32 x 128) stored as N rows x K
        for (int idx = tid; idx < TC_BN * TC_BK; idx += TC_T) {
            const int kk = idx % TC_BK, n = idx / TC_BK;
            const float x = (k0 + kk < K) ? fb(k0 + kk, n) : 0.f;
            __nv_bfloat16 h, l;
            split_bf16(x, h, l);
            const uint32_t o = tile_off(n, kk);
            *(__nv_bfloat16*)(st_base + 2 * TC_TILE_BYTES + o) = h;
            *(__nv_bfloat16*)(st_base + 3 * TC_TILE_BYTES + o) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(st_base), a_lo = a_hi + TC_TILE_BYTES;
            const uint32_t b_hi = a_hi + 2 * TC_TILE_BYTES, b_lo = a_hi + 3 * TC_TILE_BYTES;
            for (int ks = 0; ks < TC_BK / 16; ++ks) {
                const uint32_t koff = ks * 2 * 128;  // two core matrices along K per 16
                const uint64_t dah = smem_desc(a_hi + koff, 128, 512), dal = smem_desc(a_lo + koff, 128, 512);
                const uint64_t dbh = smem_desc(b_hi + koff, 128, 512), dbl = smem_desc(b_lo + koff, 128, 512);
                const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(dal), "l"(dbh), "r"(idesc), "r"(1u));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&s_bar[s]))
                         : "memory");
        }
        uses[s]++;
    }
    // all MMAs complete: wait for the last commit of each used stage
    __syncthreads();
    if (!s_fail) {
        for (int s = 0; s < 2; ++s)
            if (uses[s] > 0 && !mbar_wait(smem_u32(&s_bar[s]), (uses[s] - 1) & 1))
                if (tid == 0) s_fail = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fail) {
        // epilogue: warp w holds rows 32w..32w+31; 8 columns per load
        for (int j0 = 0; j0 < TC_BN; j0 += 8) {
            uint32_t v[8];
            const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int m = warp * 32 + lane;
#pragma unroll
            for (int u = 0; u < 8; ++u) st(m, j0 + u, __uint_as_float(v[u]));
        }
    } else if (tid == 0) {
        atomicExch(err.flag, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN) : "memory");
}

// ---------------------------------------------------------------- plain GEMM (test / library primitive)
// C (M x N, ldc) = op(A) (M x K) * B (K x N), column-major FP32; op(A) = A
// (lda >= M) or A^T (A stored K x M, lda >= K).
__global__ void __launch_bounds__(TC_T) k_tc_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                                  int transA, const float* __restrict__ B, int ldb,
                                                  float* __restrict__ C, int ldc, int* err)
{
    const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * TC_BN;
    tc_gemm_tile(
        K,
        [&](int m, int k) {
            const int mm = m0 + m;
            if (mm >= M) return 0.f;
            return transA ? A[k + (size_t)lda * mm] : A[mm + (size_t)lda * k];
        },
        [&](int k, int n) {
            const int nn = n0 + n;
            return nn < N ? B[k + (size_t)ldb * nn] : 0.f;
        },
        [&](int m, int n, float v) {
            const int mm = m0 + m, nn = n0 + n;
            if (mm < M && nn < N) C[mm + (size_t)ldc * nn] = v;
        },
        TcErr{err});
}

cudaError_t launch_tc_gemm(int M, int N, int K, const float* A, int lda, int transA, const float* B,
                           int ldb, float* C, int ldc, int* err, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((M + TC_BM - 1) / TC_BM, (N + TC_BN - 1) / TC_BN);
    k_tc_gemm<<<grid, TC_T, TC_SMEM, s>>>(M, N, K, A, lda, transA, B, ldb, C, ldc, err);
    return cudaGetLastError();
}

}  // namespace jac

// Split-precision tensor-core GEMM as a library primitive: C = op(A) * B in
// FP32 from BF16 hi/lo operand splits (three products, FP32 accumulation).
extern "C" int jacobi_lowp_gemm(int M, int N, int K, const float* A, int lda, int transA,
                                const float* B, int ldb, float* C, int ldc, void* stream)
{
    if (M < 0 || N < 0 || K < 0) return -1;
    if (!A || !B || !C) return -5;
    if ((!transA && lda < M) || (transA && lda < K) || ldb < K || ldc < M) return -5;
    if (M == 0 || N == 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (K == 0) {
        if (cudaMemset2DAsync(C, (size_t)ldc * 4, 0, (size_t)M * 4, N, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        return 0;
    }
    int* err = nullptr;
    if (cudaMallocAsync(&err, sizeof(int), s) != cudaSuccess) return JACOBI_ERR_ALLOC;
    int h = 0;
    int rc = 0;
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess ||
        jac::launch_tc_gemm(M, N, K, A, lda, transA, B, ldb, C, ldc, err, s) != cudaSuccess ||
        cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        rc = JACOBI_ERR_CUDA;
    cudaFreeAsync(err, s);
    cudaStreamSynchronize(s);
    if (rc == 0 && h) rc = JACOBI_ERR_TIMEOUT;
    return rc;
}
