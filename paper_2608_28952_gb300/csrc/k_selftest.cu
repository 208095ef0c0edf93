// k_selftest.cu -- the timeout path of the tensor-core kernels' bounded
// mbarrier wait, exercised on purpose.
//
// The tcgen05 kernels wait on mbarriers that their own MMAs arrive at; each
// wait is bounded (mbar_wait), and a wait that runs out sets the call's error
// word, skips the rest of the tile, frees the CTA's tensor memory and
// returns, so the host reports JACOBI_ERR_TIMEOUT and the context stays
// usable.  k_wait_selftest goes through the same steps with a barrier that
// nothing arrives at (arrive = 0) or that one thread arrives at (arrive = 1):
// allocate tensor memory, initialise the barrier, wait with the given limit,
// record a timeout, free the tensor memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "host.h"
#include "tc_common.cuh"

namespace jac {
namespace {

__global__ void __launch_bounds__(32) k_wait_selftest(int arrive, uint64_t limit_ns, int* err)
{
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar;
    const int tid = threadIdx.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)), "r"(32)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    if (arrive && tid == 0) {
        asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(&s_bar))
                     : "memory");
    }
    __syncthreads();
    if (tid == 0 && !mbar_wait(smem_u32(&s_bar), 0, limit_ns)) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
}

}  // namespace
}  // namespace jac

using namespace jac;

extern "C" int jacobi_wait_selftest(int arrive, double limit_ms, void* stream)
{
    if (arrive != 0 && arrive != 1) return -1;
    if (!(limit_ms >= 1.0 && limit_ms <= 2000.0)) return -2;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    int* err = ws.get<int>(1);
    if (ws.failed) return JACOBI_ERR_ALLOC;
    int h_err = 0;
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return JACOBI_ERR_CUDA;
    k_wait_selftest<<<1, 32, 0, s>>>(arrive, (uint64_t)(limit_ms * 1e6), err);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    return h_err ? JACOBI_ERR_TIMEOUT : 0;
}
