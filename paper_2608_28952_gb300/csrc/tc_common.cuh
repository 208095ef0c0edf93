// tc_common.cuh -- shared pieces of the tcgen05 kernels: the canonical
// no-swizzle K-major operand layout, shared-memory and instruction
// descriptors, the bf16 hi/lo split, and the bounded mbarrier wait.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace jac {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 32, TC_T = 128;
constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 2;          // one bf16 128 x 32 tile (8 KB)
constexpr int TC_STAGE_BYTES = 4 * TC_TILE_BYTES;          // A hi, A lo, B hi, B lo
constexpr int TC_SMEM = 2 * TC_STAGE_BYTES + 1024;         // two stages + barriers, alignment

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (r, k) of a 128 x 32 K-major bf16 tile in the
// canonical no-swizzle layout: core matrix (r/8, k/8) at (r/8)*SBO + (k/8)*LBO,
// row r%8 at 16 bytes, element k%8 at 2 bytes; LBO = 128 (next core matrix
// along K), SBO = 512 (next 8-row group).
__device__ __forceinline__ uint32_t tile_off(int r, int k)
{
    return (uint32_t)((r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (tcgen05): start address >> 4 in bits
// [0,14), leading-dimension byte offset >> 4 in [16,30), stride byte offset
// >> 4 in [32,46), version 1 in [46,48), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of tcgen05.mma.kind::f16: FP32 accumulator (bits
// [4,6) = 1), A and B bf16 (bits [7,10) and [10,13) = 1), both K-major,
// N >> 3 in [17,23), M >> 4 in [24,29).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The same with both operands fp16 (type field 0).
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// kind::tf32: A and B tf32 (type field 2).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// hi = fp16(x), lo = fp16(x - hi): for |x| in fp16's normal range the pair
// carries 22 significant bits; the caller scales x by a power of two so that
// |x| <= 1 (no overflow) and the entries that matter stay normal.
__device__ __forceinline__ void split_f16(float x, __half& hi, __half& lo)
{
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait until the mbarrier at `bar` completes the phase with parity `par`;
// false if limit_ns (default about 2 s) pass first by the global timer, or
// after 2^28 polls whatever the timer says.
constexpr uint64_t kMbarWaitNs = 2000000000ull;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t par, uint64_t limit_ns = kMbarWaitNs)
{
    const uint64_t t0 = global_ns();
    for (uint32_t polls = 0;; ++polls) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(par)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > limit_ns || polls >= (1u << 28)) return false;
    }
}

struct TcErr {
    int* flag;   // device error word (set to 1 on a timed-out wait)
};

}  // namespace jac
