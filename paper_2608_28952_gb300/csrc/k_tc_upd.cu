// k_tc_upd.cu -- the block updates of one low-precision step of the mixed
// form on the tcgen05 tensor cores (Algorithm 2's row and column updates,
// with the symmetric pair-block formulation of the FP64 path):
//
//   stage 1: T_pb = A_{P1P2} V2 for every pair-block pb = (P1 < P2), and
//            Q'(:,P) = Q(:,P) V_P for every pair P;
//   stage 2: A'_{P1P2} = V1^T T_pb, written with its mirror A'_{P2P1}.
//
// The pivot blocks themselves receive D from the pivot kernel.  Every
// product is formed from splits hi = r(x), lo = r(x - hi) as
// hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory, r = bf16
// (BF16x3) or fp16 (FP16x3).  fp16 has 5 exponent bits, so in the FP16x3
// form the FP32 operands are scaled by powers of two (exact) before the
// split: every row of a stage-1 A tile by its own row maximum over K, every
// column of T by its column maximum (collected by stage 1's epilogue); the
// products are scaled back in the epilogues.  V and Q (|entries| <= 1) are
// split unscaled.
//
// Data movement, per 128 x 128 output tile of a CTA (256 threads):
//   * V_P (FP64, from the pivot kernel) is split once per step by
//     k_tc_split_v into an "image": for every (128-column tile, 32-row
//     chunk) the bf16 hi and lo tiles in the MMA operand layout (16 KB).  The
//     same image is the B operand of stage 1 (V2(kk, n)) and the A operand of
//     stage 2 (V1^T(m, kk) = V1(kk, m)), so stages copy it with 16-byte loads;
//   * FP32 operands (A blocks, Q columns, T) are loaded eight values per
//     thread item with all loads of a chunk issued back to back into
//     registers two chunks ahead (two register slots), then split (paired
//     conversions) and stored to shared memory;
//   * two pipeline stages of 32 KB (three CTAs per SM; tf32: three stages of
//     64 KB, one CTA per SM); one thread issues the chunk's six MMAs
//     and commits them to the stage's mbarrier, which the stage's next
//     filling waits for (bounded wait: a timeout sets the error word, the
//     CTA skips the remaining work and still frees its TMEM);
//   * the epilogue reads the accumulator with tcgen05.ld (8 warps: lane
//     quarter w % 4, column half w / 4) and stores coalesced; the mirrored
//     store of stage 2 writes 8 consecutive rows per thread.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "tc_common.cuh"

namespace jac {

namespace {

constexpr int U_T = 256;
constexpr int U_NS = 3;   // most pipeline stages of any kind

// Operand kinds: 0 bf16 hi/lo, 1 fp16 hi/lo (power-of-two scaled), 2 tf32
// big/small (x = big + small, big = x with its low 13 mantissa bits cleared,
// the tensor core reading the top 19 bits of each).
template <int KIND>
struct KT {
    static constexpr int EB = KIND == 2 ? 4 : 2;            // bytes per element in shared memory
    static constexpr int TILE = TC_BM * TC_BK * EB;          // one 128 x 32 part (8 or 16 KB)
    static constexpr int STAGE = 4 * TILE;                   // A hi, A lo, B hi, B lo
    // bf16 / fp16: two 32 KB stages, so three CTAs share an SM (one's
    // epilogue and set-up overlap the others' main loops); tf32 (64 KB
    // stages, one CTA per SM either way): three.  At least two: the next
    // chunk's bulk copy goes into the other stage while this one computes.
    static constexpr int NS = KIND == 2 ? 3 : 2;
    static constexpr int SMEM = NS * STAGE + 1024;
    static constexpr int IMG = 2 * TILE;                     // hi + lo of one operand tile
    static constexpr int SBO = KIND == 2 ? 1024 : 512;       // next 8-row group of core matrices
    static constexpr int KSTEP = KIND == 2 ? 8 : 16;         // K of one MMA
};

// Byte offset of element (r, k) in a part: 8 x 16-byte core matrices, K-major
// (8 bf16/fp16 or 4 tf32 values per core-matrix row), no swizzle.
template <int KIND>
__device__ __forceinline__ uint32_t toff(int r, int k)
{
    if constexpr (KIND == 2)
        return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
    else
        return tile_off(r, k);
}

__device__ __forceinline__ int umap(int I, int J, int b, int x) { return x < b ? I * b + x : J * b + (x - b); }

__device__ __forceinline__ bool uentry(const int2* pairs, int e, int& I, int& J)
{
    const int2 pr = pairs[e];
    const bool fz = pr.x < 0;
    I = fz ? -1 - pr.x : pr.x;
    J = fz ? -1 - pr.y : pr.y;
    return fz;
}

__device__ __forceinline__ void decode_pb(int pb, int& e1, int& e2)
{
    int t = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)pb)) * 0.5f);
    while (t * (t - 1) / 2 > pb) --t;
    while ((t + 1) * t / 2 <= pb) ++t;
    e2 = t;
    e1 = pb - t * (t - 1) / 2;
}

// Eight bf16 values as one 16-byte word.
struct Pack8 {
    uint4 hi, lo;
};

// hi = r(x), lo = r(x - hi) for eight values, two per conversion (the paired
// round-to-nearest conversions give the same bits as one value at a time);
// fp16 values are scaled first, bf16 values are not (scale is 1 there).
template <bool F16>
__device__ __forceinline__ Pack8 split8(const float (&x)[8], float scale = 1.f)
{
    Pack8 p;
    uint32_t hw[4], lw[4];
    if (F16) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float a = x[2 * u] * scale, b = x[2 * u + 1] * scale;
            const __half2 h = __floats2half2_rn(a, b);
            const float2 hf = __half22float2(h);
            const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
            hw[u] = *reinterpret_cast<const uint32_t*>(&h);
            lw[u] = *reinterpret_cast<const uint32_t*>(&l);
        }
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float a = x[2 * u], b = x[2 * u + 1];
            const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            const float2 hf = __bfloat1622float2(h);
            const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
            hw[u] = *reinterpret_cast<const uint32_t*>(&h);
            lw[u] = *reinterpret_cast<const uint32_t*>(&l);
        }
    }
    p.hi = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    p.lo = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    return p;
}

// Eight consecutive K values (r, kk0..kk0+7) of an operand split into the
// hi part at dst and the lo part at dst + TILE.
template <int KIND>
__device__ __forceinline__ void store8(unsigned char* dst, int r, int kk0, const float (&x)[8], float scale)
{
    if constexpr (KIND == 2) {
        float big[8], sml[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float v = x[u] * scale;
            big[u] = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
            sml[u] = v - big[u];
        }
        const uint32_t o0 = toff<2>(r, kk0), o1 = toff<2>(r, kk0 + 4);
        *reinterpret_cast<float4*>(dst + o0) = make_float4(big[0], big[1], big[2], big[3]);
        *reinterpret_cast<float4*>(dst + o1) = make_float4(big[4], big[5], big[6], big[7]);
        *reinterpret_cast<float4*>(dst + KT<2>::TILE + o0) = make_float4(sml[0], sml[1], sml[2], sml[3]);
        *reinterpret_cast<float4*>(dst + KT<2>::TILE + o1) = make_float4(sml[4], sml[5], sml[6], sml[7]);
    } else {
        const Pack8 p = split8<KIND == 1>(x, scale);
        const uint32_t o = tile_off(r, kk0);
        *reinterpret_cast<uint4*>(dst + o) = p.hi;
        *reinterpret_cast<uint4*>(dst + KT<KIND>::TILE + o) = p.lo;
    }
}

// Power-of-two scaling: e with mx * 2^-e in [0.5, 1) (0 for mx == 0), and 2^e.
__device__ __forceinline__ int exp_of(float mx)
{
    if (!(mx > 0.f)) return 0;
    const int e = ilogbf(mx) + 1;
    return e < -100 ? -100 : (e > 100 ? 100 : e);
}
__device__ __forceinline__ float pow2(int e) { return __int_as_float((127 + e) << 23); }

// ---------------------------------------------------------------- operand loaders
// A loader fills one 128 x 32 operand tile (hi at dst, lo at dst + 8 KB) of
// chunk c in two phases: load(c) into registers, store() into shared memory.
// Element (r, kk) of the tile is stored at tile_off(r, kk); r is the M (or N)
// index, kk the K index.

// FP32 gather: element (r, kk) = base[row(r) + ld * col(c * 32 + kk)], 0 where
// row < 0 or col < 0.  Thread items (r, g): r = item % 128, g = item / 128
// (eight consecutive K values), items tid and tid + 256.
template <int KIND>
struct GatherF32 {
    const float* base;
    size_t ld;
    int rows[2];        // global row of the thread's two items (or -1)
    float scale[2];     // power-of-two scale of the two items' rows (FP16x3)
    float v[2][2][8];   // register slot (chunk parity), item, value
    template <int S, class COL>
    __device__ __forceinline__ void load(int c, COL col)
    {
        const int tid = threadIdx.x;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int g = (tid + U_T * i) >> 7;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int cc = col(c * TC_BK + g * 8 + u);
                v[S][i][u] = (rows[i] >= 0 && cc >= 0) ? __ldg(base + rows[i] + ld * (size_t)cc) : 0.f;
            }
        }
    }
    template <int S>
    __device__ __forceinline__ void store(unsigned char* dst) const
    {
        const int tid = threadIdx.x;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int item = tid + U_T * i, r = item & 127, g = item >> 7;
            store8<KIND>(dst, r, g * 8, v[S][i], scale[i]);
        }
    }
};

// The gather over the columns (K) of the pair (I, J): column x of the
// operand is global column umap(I, J, b, x).
template <int KIND>
struct GatherPairCols {
    GatherF32<KIND>& g;
    int I, J, b, k;
    template <int S>
    __device__ __forceinline__ void load(int c)
    {
        g.template load<S>(c, [&](int x) { return x < k ? umap(I, J, b, x) : -1; });
    }
    template <int S>
    __device__ __forceinline__ void store(unsigned char* d) const { g.template store<S>(d); }
};

// K-major FP32 (T of stage 2 as the B operand): element (n, kk) =
// T[(c * 32 + kk) + k * (n0 + n)], 0 outside k x k.  Items (n, g) with
// g = item % 4, n = item / 4, so a warp reads 128 contiguous bytes per n.
template <int KIND>
struct KMajorF32 {
    const float* T;
    int k, n0;
    bool vec4;
    const float* cscale;   // shared memory: power-of-two scale of column n (FP16x3), or null
    float v[2][2][8];      // register slot (chunk parity), item, value
    template <int S>
    __device__ __forceinline__ void load(int c)
    {
        const int tid = threadIdx.x;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int item = tid + U_T * i, g = item & 3, n = item >> 2;
            const int kk0 = c * TC_BK + g * 8, col = n0 + n;
            const float* src = T + kk0 + (size_t)k * col;
            if (col < k && vec4 && kk0 + 8 <= k) {
                const float4 a = __ldg(reinterpret_cast<const float4*>(src));
                const float4 b = __ldg(reinterpret_cast<const float4*>(src + 4));
                v[S][i][0] = a.x; v[S][i][1] = a.y; v[S][i][2] = a.z; v[S][i][3] = a.w;
                v[S][i][4] = b.x; v[S][i][5] = b.y; v[S][i][6] = b.z; v[S][i][7] = b.w;
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) v[S][i][u] = (col < k && kk0 + u < k) ? __ldg(src + u) : 0.f;
            }
        }
    }
    template <int S>
    __device__ __forceinline__ void store(unsigned char* dst) const
    {
        const int tid = threadIdx.x;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int item = tid + U_T * i, g = item & 3, n = item >> 2;
            store8<KIND>(dst, n, g * 8, v[S][i], cscale ? cscale[n] : 1.f);
        }
    }
};

// Pre-split image tile (hi and lo parts, 16 or 32 KB, contiguous in global
// memory in the MMA operand layout): staged by the tensor memory accelerator
// (one cp.async.bulk per chunk, completing on the stage's "full" mbarrier),
// not through registers.
template <int KIND>
struct ImageTile {
    static constexpr bool kBulk = true;
    const unsigned char* img;   // tile (tile index t, chunk c) at img + (t * nchk + c) * IMG
    int nchk;
    int t;
    __device__ __forceinline__ const unsigned char* src(int c) const
    {
        return img + ((size_t)t * nchk + c) * KT<KIND>::IMG;
    }
    template <int S>
    __device__ __forceinline__ void load(int) {}
    template <int S>
    __device__ __forceinline__ void store(unsigned char*) const {}
};

template <class L, class = void>
struct IsBulk {
    static constexpr bool value = false;
};
template <class L>
struct IsBulk<L, decltype((void)L::kBulk)> {
    static constexpr bool value = L::kBulk;
};

template <int S>
struct Slot {
    static constexpr int value = S;
};

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global memory into this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// ---------------------------------------------------------------- the tile
// acc(128 x 128) = Aop * Bop over nchk chunks of 32.  LA / LB: loaders with
// load(c) / store(dst); EP(m, j0, v[8]): the epilogue for row m, columns
// j0..j0+7.
template <int KIND, class LA, class LB, class EP>
__device__ void tc_tile(int nchk, LA& la, LB& lb, EP ep, int* err)
{
    extern __shared__ __align__(1024) unsigned char usm[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[U_NS];
    __shared__ __align__(8) uint64_t s_full[U_NS];   // bulk (TMA) operand copies of a stage landed
    __shared__ int s_fail;
    constexpr int U_NS = KT<KIND>::NS;   // this kind's stages (the arrays above have room for the most)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* base = (unsigned char*)(((uintptr_t)usm + 1023) & ~(uintptr_t)1023);
    constexpr bool kBA = IsBulk<LA>::value, kBB = IsBulk<LB>::value, kAnyBulk = kBA || kBB;
    constexpr uint32_t kBulkBytes = (kBA ? KT<KIND>::IMG : 0) + (kBB ? KT<KIND>::IMG : 0);

    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < U_NS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_full[s])) : "memory");
        }
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
    const uint32_t idesc = KIND == 2 ? idesc_tf32(TC_BM, TC_BN)
                                     : (KIND == 1 ? idesc_f16(TC_BM, TC_BN) : idesc_bf16(TC_BM, TC_BN));
    constexpr int TB = KT<KIND>::TILE, SBO = KT<KIND>::SBO;
    uint32_t uses[U_NS];
#pragma unroll
    for (int s = 0; s < U_NS; ++s) uses[s] = 0;

    // thread 0: the bulk operand copies of chunk c into stage c % U_NS (the
    // stage must be free: its previous MMAs complete)
    int bulk_issued = 0, bulk_waited = 0;
    auto issue_bulk = [&](int c) {
        const int s = c % U_NS;
        unsigned char* st = base + s * KT<KIND>::STAGE;
        const uint32_t fb = smem_u32(&s_full[s]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kBulkBytes) : "memory");
        if constexpr (kBA) bulk_g2s(smem_u32(st), la.src(c), KT<KIND>::IMG, fb);
        if constexpr (kBB) bulk_g2s(smem_u32(st + 2 * TB), lb.src(c), KT<KIND>::IMG, fb);
        ++bulk_issued;
    };
    if (kAnyBulk && tid == 0) issue_bulk(0);
    // register-staged operands: chunk c in register slot c % 2, its loads
    // issued two chunks ahead (a slot is refilled right after its store), so
    // their latency spans two chunks' MMAs; the slot is a compile-time index
    la.template load<0>(0);
    lb.template load<0>(0);
    if (nchk > 1) {
        la.template load<1>(1);
        lb.template load<1>(1);
    }
    auto step = [&](int c, auto slot) -> bool {
        constexpr int S = decltype(slot)::value;
        const int s = c % U_NS;
        unsigned char* st = base + s * KT<KIND>::STAGE;
        // the MMAs that last read this stage (chunk c - U_NS) must be complete
        if (c >= U_NS && !mbar_wait(smem_u32(&s_bar[s]), (uses[s] - 1) & 1)) s_fail = 1;
        la.template store<S>(st);
        lb.template store<S>(st + 2 * TB);
        if (c + 2 < nchk) {  // the loads of chunk c + 2 into the slot just stored
            la.template load<S>(c + 2);
            lb.template load<S>(c + 2);
        }
        if (c + 1 < nchk) {
            if (kAnyBulk && tid == 0 && !s_fail) {
                const int s1 = (c + 1) % U_NS;
                if (c + 1 >= U_NS && !mbar_wait(smem_u32(&s_bar[s1]), (uses[s1] - 1) & 1)) s_fail = 1;
                else issue_bulk(c + 1);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s_fail) return false;
        if (tid == 0) {
            bool landed = true;
            if (kAnyBulk) {
                landed = mbar_wait(smem_u32(&s_full[s]), (uint32_t)(c / U_NS) & 1u);
                ++bulk_waited;
                if (!landed) s_fail = 1;   // no MMA on a stage whose copy did not land; the commit below still arrives
            }
            if (landed) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(st), a_lo = a_hi + TB;
            const uint32_t b_hi = a_hi + 2 * TB, b_lo = a_hi + 3 * TB;
#pragma unroll
            for (int ks = 0; ks < TC_BK / KT<KIND>::KSTEP; ++ks) {
                const uint32_t koff = ks * 2 * 128;   // two core matrices along K per MMA
                const uint64_t dah = smem_desc(a_hi + koff, 128, SBO), dal = smem_desc(a_lo + koff, 128, SBO);
                const uint64_t dbh = smem_desc(b_hi + koff, 128, SBO), dbl = smem_desc(b_lo + koff, 128, SBO);
                const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
                if constexpr (KIND == 2) {
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(dal), "l"(dbh), "r"(idesc), "r"(1u));
                } else {
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
            }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&s_bar[s]))
                         : "memory");
        }
        uses[s]++;
        return true;
    };
    for (int c = 0; c < nchk; c += 2) {
        if (!step(c, Slot<0>{})) break;
        if (c + 1 < nchk && !step(c + 1, Slot<1>{})) break;
    }
    // bulk copies issued but not waited for (a failed tile breaks early):
    // wait for them (bounded) before the shared memory is given up
    if (kAnyBulk && tid == 0)
        for (int c = bulk_waited; c < bulk_issued; ++c) mbar_wait(smem_u32(&s_full[c % U_NS]), (uint32_t)(c / U_NS) & 1u);
    // every MMA complete: wait for the last commit of each used stage
    __syncthreads();
    if (!s_fail) {
        for (int s = 0; s < U_NS; ++s)
            if (uses[s] > 0 && !mbar_wait(smem_u32(&s_bar[s]), (uses[s] - 1) & 1)) s_fail = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fail) {
        const int q = warp & 3, h = warp >> 2, m = q * 32 + lane;
        for (int j0 = h * 64; j0 < h * 64 + 64; j0 += 8) {
            uint32_t v[8];
            const uint32_t addr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)j0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float f[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) f[u] = __uint_as_float(v[u]);
            ep(m, j0, f);
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN) : "memory");
}

// ---------------------------------------------------------------- kernels
// Image of V_P per pair (skipped for pairs without rotation): tile (nt, c)
// holds element (kk, n) = V_P(c * 32 + kk, nt * 128 + n), rounded to FP32
// then split, at tile_off(n, kk).
template <int KIND>
__global__ void __launch_bounds__(U_T) k_tc_split_v(const double* __restrict__ V, const int* __restrict__ rot,
                                                    int k, int ntk, int nchk, unsigned char* __restrict__ img)
{
    const int tile = blockIdx.x, e = tile / (ntk * nchk), rem = tile % (ntk * nchk);
    const int nt = rem / nchk, c = rem % nchk;
    if (rot[e] == 0) return;
    const double* Ve = V + (size_t)e * 2 * k * k;
    unsigned char* dst = img + (size_t)tile * KT<KIND>::IMG;
    for (int i = 0; i < 2; ++i) {
        const int item = threadIdx.x + U_T * i, g = item & 3, nn = item >> 2;
        const int n = nt * TC_BN + nn, kk0 = c * TC_BK + g * 8;
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = (n < k && kk0 + u < k) ? (float)Ve[(kk0 + u) + (size_t)k * n] : 0.f;
        store8<KIND>(dst, nn, kk0 - c * TC_BK, x, 1.f);
    }
}

// Stage 1.  Items [0, n_sand): tile (mt, nt) of T_pb = A_{P1P2} V2; items
// beyond: tile (rt, nt) of Q'(:, P) = Q(:, P) V_P.  A pivot without rotation
// (V = I) gives an exact copy instead of a product.  FP16x3: the rows of the
// A tile are scaled by their maxima over K (a first pass over the tile's
// rows), and the epilogue records every T column's maximum for stage 2.
template <int KIND>
__global__ void __launch_bounds__(U_T) k_tc_upd1(TcUpdArgs a, int n_sand)
{
    constexpr bool F16 = KIND == 1;
    __shared__ float s_rmax[2][TC_BM];
    const int k = a.k, b = a.b, ntk = (k + TC_BN - 1) / TC_BN, nchk = (k + TC_BK - 1) / TC_BK;
    int item = blockIdx.x;
    if (item < n_sand) {
        const int pb = item / (ntk * ntk), rem = item % (ntk * ntk), mt = rem / ntk, nt = rem % ntk;
        int e1, e2, I1, J1, I2, J2;
        decode_pb(pb, e1, e2);
        uentry(a.pairs, e1, I1, J1);
        uentry(a.pairs, e2, I2, J2);
        float* T = a.T + (size_t)pb * k * k;
        unsigned* tmax = F16 ? a.tmax + (size_t)pb * k : nullptr;
        const int m0 = mt * TC_BM, n0 = nt * TC_BN;
        if (a.rot[e2] == 0) {
            for (int idx = threadIdx.x; idx < TC_BM * TC_BN; idx += U_T) {
                const int m = m0 + idx % TC_BM, j = n0 + idx / TC_BM;
                if (m < k && j < k) {
                    const float v = a.Ain[umap(I1, J1, b, m) + (size_t)a.lda * umap(I2, J2, b, j)];
                    T[m + (size_t)k * j] = v;
                    if (F16 && v != 0.f) atomicMax(tmax + j, __float_as_uint(fabsf(v)));
                }
            }
            return;
        }
        GatherF32<KIND> la;
        la.base = a.Ain;
        la.ld = (size_t)a.lda;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = (threadIdx.x + U_T * i) & 127;
            la.rows[i] = m0 + r < k ? umap(I1, J1, b, m0 + r) : -1;
            la.scale[i] = 1.f;
        }
        if (F16) {
            // row maxima over all K: thread (r, half h) scans columns h, h + 2, ...
            const int r = threadIdx.x & 127, h = threadIdx.x >> 7;
            const int row = m0 + r < k ? umap(I1, J1, b, m0 + r) : -1;
            float mx = 0.f;
            if (row >= 0)
                for (int x = h; x < k; x += 2) mx = fmaxf(mx, fabsf(__ldg(a.Ain + row + (size_t)a.lda * umap(I2, J2, b, x))));
            s_rmax[h][r] = mx;
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int rr = (threadIdx.x + U_T * i) & 127;
                la.scale[i] = pow2(-exp_of(fmaxf(s_rmax[0][rr], s_rmax[1][rr])));
            }
        }
        ImageTile<KIND> lb{a.vimg + (size_t)e2 * ntk * nchk * KT<KIND>::IMG, nchk, nt};
        GatherPairCols<KIND> lawrap{la, I2, J2, b, k};
        tc_tile<KIND>(nchk, lawrap, lb,
                     [&](int m, int j0, const float (&v)[8]) {
                         const bool live = m0 + m < k;
                         const float up = F16 ? pow2(exp_of(fmaxf(s_rmax[0][m], s_rmax[1][m]))) : 1.f;
                         float w[8];
#pragma unroll
                         for (int u = 0; u < 8; ++u) {
                             w[u] = v[u] * up;
                             if (live && n0 + j0 + u < k) T[(m0 + m) + (size_t)k * (n0 + j0 + u)] = w[u];
                         }
                         if (F16) {
                             // column maxima over the warp's 32 rows, one atomic per column
#pragma unroll
                             for (int u = 0; u < 8; ++u) {
                                 float x = live ? fabsf(w[u]) : 0.f;
                                 for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
                                 if ((threadIdx.x & 31) == 0 && x > 0.f && n0 + j0 + u < k)
                                     atomicMax(tmax + n0 + j0 + u, __float_as_uint(x));
                             }
                         }
                     },
                     a.err);
        if (threadIdx.x == 0) atomicAdd(&a.cnt->flops_lowp, 6ull * TC_BM * TC_BN * k);
        return;
    }
    item -= n_sand;
    const int nrt = (a.qrows + TC_BM - 1) / TC_BM;
    const int e = item / (nrt * ntk), rem = item % (nrt * ntk), rt = rem / ntk, nt = rem % ntk;
    int I, J;
    uentry(a.pairs, e, I, J);
    const int r0 = rt * TC_BM, n0 = nt * TC_BN;
    if (a.rot[e] == 0) {
        for (int idx = threadIdx.x; idx < TC_BM * TC_BN; idx += U_T) {
            const int m = r0 + idx % TC_BM, j = n0 + idx / TC_BM;
            if (m < a.qrows && j < k) {
                const size_t o = m + (size_t)a.ldq * umap(I, J, b, j);
                a.Qout[o] = a.Qin[o];
            }
        }
        return;
    }
    GatherF32<KIND> la;
    la.base = a.Qin;
    la.ld = (size_t)a.ldq;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int r = (threadIdx.x + U_T * i) & 127;
        la.rows[i] = r0 + r < a.qrows ? r0 + r : -1;
        la.scale[i] = 1.f;
    }
    ImageTile<KIND> lb{a.vimg + (size_t)e * ntk * nchk * KT<KIND>::IMG, nchk, nt};
    GatherPairCols<KIND> lawrap{la, I, J, b, k};
    tc_tile<KIND>(nchk, lawrap, lb,
                 [&](int m, int j0, const float (&v)[8]) {
                     if (r0 + m >= a.qrows) return;
#pragma unroll
                     for (int u = 0; u < 8; ++u)
                         if (n0 + j0 + u < k) a.Qout[(r0 + m) + (size_t)a.ldq * umap(I, J, b, n0 + j0 + u)] = v[u];
                 },
                 a.err);
    if (threadIdx.x == 0) atomicAdd(&a.cnt->flops_lowp, 6ull * TC_BM * TC_BN * k);
}

// Stage 2: tile (mt, nt) of O_pb = V1^T T_pb, written to A' at (P1 rows, P2
// columns) and mirrored to (P2 rows, P1 columns), so A' stays symmetric.
// FP16x3: T's columns are scaled by their maxima from stage 1 and the
// products scaled back.
template <int KIND>
__global__ void __launch_bounds__(U_T) k_tc_upd2(TcUpdArgs a)
{
    constexpr bool F16 = KIND == 1;
    __shared__ float s_cscale[TC_BN];
    const int k = a.k, b = a.b, ntk = (k + TC_BN - 1) / TC_BN, nchk = (k + TC_BK - 1) / TC_BK;
    const int item = blockIdx.x;
    const int pb = item / (ntk * ntk), rem = item % (ntk * ntk), mt = rem / ntk, nt = rem % ntk;
    int e1, e2, I1, J1, I2, J2;
    decode_pb(pb, e1, e2);
    uentry(a.pairs, e1, I1, J1);
    uentry(a.pairs, e2, I2, J2);
    const float* T = a.T + (size_t)pb * k * k;
    const int m0 = mt * TC_BM, n0 = nt * TC_BN;
    float* Ao = a.Aout;
    const size_t lda = (size_t)a.lda;
    if (a.rot[e1] == 0) {
        for (int idx = threadIdx.x; idx < TC_BM * TC_BN; idx += U_T) {
            const int m = m0 + idx % TC_BM, j = n0 + idx / TC_BM;
            if (m < k && j < k) {
                const int gi = umap(I1, J1, b, m), gj = umap(I2, J2, b, j);
                const float v = T[m + (size_t)k * j];
                Ao[gi + lda * gj] = v;
                Ao[gj + lda * gi] = v;
            }
        }
        return;
    }
    if (F16) {
        for (int j = threadIdx.x; j < TC_BN; j += U_T)
            s_cscale[j] = n0 + j < k ? pow2(-exp_of(__uint_as_float(a.tmax[(size_t)pb * k + n0 + j]))) : 1.f;
        __syncthreads();
    }
    ImageTile<KIND> la{a.vimg + (size_t)e1 * ntk * nchk * KT<KIND>::IMG, nchk, mt};
    KMajorF32<KIND> lb;
    lb.T = T;
    lb.k = k;
    lb.n0 = n0;
    lb.vec4 = (k & 3) == 0;
    lb.cscale = F16 ? s_cscale : nullptr;
    // 8 consecutive output columns land in 8 consecutive rows of the mirror
    // when they stay inside one block of the pair and the address is 16-byte
    // aligned
    const bool mvec = (b & 7) == 0 && (lda & 3) == 0;
    tc_tile<KIND>(nchk, la, lb,
                 [&](int m, int j0, const float (&v0)[8]) {
                     if (m0 + m >= k) return;
                     float v[8];
#pragma unroll
                     for (int u = 0; u < 8; ++u) v[u] = F16 ? v0[u] / s_cscale[j0 + u] : v0[u];
                     const int gi = umap(I1, J1, b, m0 + m);
                     const int jb = n0 + j0;
#pragma unroll
                     for (int u = 0; u < 8; ++u)
                         if (jb + u < k) Ao[gi + lda * umap(I2, J2, b, jb + u)] = v[u];
                     if (mvec && jb + 8 <= k) {
                         float* dst = Ao + umap(I2, J2, b, jb) + lda * gi;
                         reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
                         reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
                     } else {
#pragma unroll
                         for (int u = 0; u < 8; ++u)
                             if (jb + u < k) Ao[umap(I2, J2, b, jb + u) + lda * gi] = v[u];
                     }
                 },
                 a.err);
    if (threadIdx.x == 0) atomicAdd(&a.cnt->flops_lowp, 6ull * TC_BM * TC_BN * k);
}

}  // namespace

size_t tc_update_tbuf_floats(int npairs, int k) { return (size_t)(npairs * (npairs - 1) / 2) * k * k; }

size_t tc_update_tmax_words(int npairs, int k) { return (size_t)(npairs * (npairs - 1) / 2) * k; }

size_t tc_update_vimg_bytes(int npairs, int k)
{
    const size_t ntk = (k + TC_BN - 1) / TC_BN, nchk = (k + TC_BK - 1) / TC_BK;
    return (size_t)npairs * ntk * nchk * KT<2>::IMG;   // the largest kind
}

template <int KIND>
static cudaError_t launch_tc_update_t(const TcUpdArgs& a, cudaStream_t s)
{
    constexpr bool F16 = KIND == 1;
    constexpr int U_SMEM = KT<KIND>::SMEM;
    const int ntk = (a.k + TC_BN - 1) / TC_BN, nchk = (a.k + TC_BK - 1) / TC_BK;
    const int npb = a.npairs * (a.npairs - 1) / 2;
    const int n_sand = npb * ntk * ntk;
    const int n_q = a.Qin ? a.npairs * ((a.qrows + TC_BM - 1) / TC_BM) * ntk : 0;
    cudaError_t e = cudaFuncSetAttribute(k_tc_upd1<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, U_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_upd2<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, U_SMEM);
    if (e != cudaSuccess) return e;
    if (F16 && npb > 0 && (e = cudaMemsetAsync(a.tmax, 0, sizeof(unsigned) * (size_t)npb * a.k, s)) != cudaSuccess)
        return e;
    if (a.npairs > 0) k_tc_split_v<KIND><<<a.npairs * ntk * nchk, U_T, 0, s>>>(a.V, a.rot, a.k, ntk, nchk, a.vimg);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n_sand + n_q > 0) k_tc_upd1<KIND><<<n_sand + n_q, U_T, U_SMEM, s>>>(a, n_sand);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n_sand > 0) k_tc_upd2<KIND><<<n_sand, U_T, U_SMEM, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tc_update(const TcUpdArgs& a, cudaStream_t s)
{
    return a.kind == 2 ? launch_tc_update_t<2>(a, s)
                       : (a.kind == 1 ? launch_tc_update_t<1>(a, s) : launch_tc_update_t<0>(a, s));
}

}  // namespace jac
