// k_emu.cu -- FP64-accurate products on the bf16 tensor cores (tcgen05) by
// slicing: the error-free splitting of Ozaki, Ogita, Oishi and Rump
// ("Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer.
// Algorithms 59, 2012), with integer-valued bf16 slices.
//
// Every row m of Aop is scaled by 2^{E_m}, E_m > the exponent of its largest
// entry, and written in fixed point with 56 fraction bits, X = |a| 2^{56-E_m}
// (rounded), written with eight balanced base-2^7 digits d_1..d_8, and slice
// p holds d_p 2^{-7(p-1)} (exact in bf16).  Columns of Bop likewise with F_n.
// Then a = 2^{E_m - 7} sum_p A_p and
//     C(m, n) = 2^{E_m + F_n - 14} sum_{p + q <= 9} sum_k A_p(m, k) B_q(k, n).
// A product A_p B_q is an integer times 2^{-7(p + q - 2)}; with K <= 512 the
// sums of level l = p + q - 2 <= 4 stay below 2^24 in magnitude (|d_1| <= 128,
// |d_p| <= 64 for p > 1: level 4, the largest, has 2 * 128 * 64 + 3 * 64 * 64
// = 28672 per K value, 28672 * 512 < 2^24) and are exact in the FP32
// accumulators of the tensor cores, one accumulator per level; levels 5..7 (relative weight <= 2^-35)
// share one.  The accumulators are combined exactly in 64-bit integers (units
// of 2^-35) and converted once.  The dropped products (p + q > 9), the
// rounding to 56 fraction bits and the rounding of the lowest levels in the
// combination leave an error below about (9 K + 64) 2^-56 2^{E_m + F_n}, the
// size of FP64 rounding in a K-term dot product of the scaled rows and
// columns.
//
// One CTA computes a 128 x 64 tile (six 64-column accumulators in 512 TMEM
// columns); K is streamed in chunks of 32 through two 96 KB stages (8 slices
// of A, 128 x 32, and of B, 64 x 32, in the canonical no-swizzle K-major
// layout); one thread issues the 72 MMAs of a chunk (2 K steps x 36 slice
// products) and commits them to the stage's mbarrier (bounded waits).  For
// K > 256 (emu_tile<true>) the accumulators are drained into 64-bit integer
// running sums every 512 K values.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "tc_common.cuh"

namespace jac {

namespace {

constexpr int EM = 128, EN = 64, EK = 32, ENS = 8, ENACC = 6, E_T = 256;
constexpr int E_KSUPER = 512;   // K values per exact FP32 accumulation (the bound above)
constexpr int E_ATILE = EM * EK * 2;                      // one A slice tile (8 KB)
constexpr int E_BTILE = EN * EK * 2;                      // one B slice tile (4 KB)
constexpr int E_STAGE = ENS * (E_ATILE + E_BTILE);        // 96 KB
constexpr int E_SMEM = 2 * E_STAGE + 1024;

// unbiased exponent e with |x| in [2^e, 2^{e+1}) (-1100 for 0); integer
// operations only (GB300's FP64 pipe runs at 1/64 rate)
__device__ __forceinline__ int exp2_of(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    if ((b << 1) == 0) return -1100;
    const int ea = (int)((b >> 52) & 0x7FF);
    if (ea) return ea - 1023;
    return -1075 + (64 - __clzll((long long)(b & 0xFFFFFFFFFFFFFull)));   // subnormal
}

// x 2^-c for a power-of-two shift by integer operations on the exponent
// field (exact; the FP64 path only where the result leaves the normal range).
__device__ __forceinline__ double pow2_shift(double x, int c)
{
    const long long bits = __double_as_longlong(x);
    const int ea = (int)((bits >> 52) & 0x7FF);
    if (c == 0 || (bits << 1) == 0) return x;
    if (ea == 0) return ldexp(x, -c);   // subnormal
    if (ea - c >= 1 && ea - c <= 2046) return __longlong_as_double(bits - (long long)c * (1ll << 52));
    return ldexp(x, -c);
}

// The eight slices of x for the row/column scale 2^E (|x| < 2^E): the
// fixed-point value X = |x| 2^{56-E} (rounded to nearest where x is more than
// four binades below the scale; exact otherwise) written with balanced
// base-2^7 digits, X = sum_p d_p 2^{56-7p}, d_1 in [0, 128], the others in
// [-64, 63], and the sign of x on every digit.
// Balanced digits keep the discarded low-order products unbiased; with
// truncated digits they always shrink |a b| and the bias builds up over the
// hundreds of update steps of a solve.
__device__ __forceinline__ void slice8(double x, int E, __nv_bfloat16 (&s)[ENS])
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int ea = (int)((b >> 52) & 0x7FF);
    uint64_t M = b & 0xFFFFFFFFFFFFFull;
    int e = -1022;
    if (ea) {
        M |= 1ull << 52;
        e = ea - 1023;
    }
    const int sh = e - E + 4;   // |X| = M 2^sh < 2^56
    uint64_t X;
    if (sh >= 0) X = M << sh;
    else if (sh > -54) X = (M + (1ull << (-sh - 1))) >> -sh;
    else X = 0ull;
    // Balanced digits by one offset: with H = 64 sum_{p=2..8} 2^{56-7p},
    // the base-128 digits u_p of Y = X + H give d_p = u_p - 64 (p >= 2) and
    // d_1 = Y >> 49; the sign of x is applied to every digit.
    const uint64_t H = 64ull * ((1ull << 42) + (1ull << 35) + (1ull << 28) + (1ull << 21) + (1ull << 14) + (1ull << 7) + 1ull);
    const uint64_t Y = X + H;
    const bool neg = (b >> 63) != 0;
#pragma unroll
    for (int p = 1; p <= ENS; ++p) {
        int d = p == 1 ? (int)(Y >> 49) : (int)((Y >> (56 - 7 * p)) & 127ull) - 64;
        if (neg) d = -d;
        s[p - 1] = __float2bfloat16_rn(__int2float_rn(d) * __int_as_float((127 - 7 * (p - 1)) << 23));
    }
}

// Eight consecutive K values of one row r of a slice tile set: slice p of
// value u to tile p at tile_off(r, kk0 + u).
__device__ __forceinline__ void store_slices(unsigned char* base, int tile_bytes, int r, int kk0,
                                             const double (&x)[8], int E)
{
    __nv_bfloat16 sl[8][ENS];
#pragma unroll
    for (int u = 0; u < 8; ++u) slice8(x[u], E, sl[u]);
    const uint32_t o = tile_off(r, kk0);
#pragma unroll
    for (int p = 0; p < ENS; ++p) {
        __nv_bfloat16 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = sl[u][p];
        *reinterpret_cast<uint4*>(base + p * tile_bytes + o) = *reinterpret_cast<const uint4*>(v);
    }
}

}  // namespace

// S 2^e in FP64, rounded to nearest even, by integer operations (the FP64
// pipe runs at 1/64 rate); the ldexp path is for results outside the normal
// range (not met in Jacobi updates).
__device__ __forceinline__ double i64_scaled(long long sv, int e)
{
    if (sv == 0) return 0.0;
    const uint64_t sg = sv < 0 ? (1ull << 63) : 0ull;
    const uint64_t mag = sv < 0 ? (uint64_t)(-sv) : (uint64_t)sv;
    const int lz = __clzll((long long)mag);
    const uint64_t mm = mag << lz;                    // leading one at bit 63
    uint64_t mant = mm >> 11;                         // 53 bits
    const uint64_t low = mm & 0x7FFull;
    if (low > 0x400ull || (low == 0x400ull && (mant & 1ull))) ++mant;
    const int ex = 63 - lz + e + 1023;               // biased exponent of the result
    if (ex > 0 && ex < 2047)
        return __longlong_as_double((long long)(sg | (((uint64_t)ex << 52) + (mant - (1ull << 52)))));
    return ldexp(__ll2double_rn(sv), e);
}

// C tile (128 x 64) = Aop (128 x K) * Bop (K x 64) in FP64 accuracy.
// fa(m, k), fb(k, n): FP64 operand values (0 outside); eA[m], eB[n]: the
// row / column scale exponents in shared memory (filled by the caller, all
// threads synchronised); st(m, n, v) stores.  K <= 256 unless BIG: then the
// accumulators are drained every E_KSUPER = 512 K values (so every level sum
// stays exact in FP32) into 64-bit integer running sums held in registers, in
// units of 2^{sh - 35} with sh = the shift that keeps |sum| below 2^63
// (sh = 0 up to K = 8192: 16 drains of |S| < 2^58.02).
//
// AIMG / BIMG: the operand's slices come pre-made from an image in global
// memory instead (slice p of chunk c: E_ATILE / E_BTILE bytes in the MMA
// layout at img + (8 c + p) stride, the tile's rows first; img_stride for A,
// img_stride_b for B, which defaults to img_stride), staged by
// bulk copies of the tensor memory accelerator that complete on the stage's
// "full" mbarrier; fa / fb are not called for that operand.
template <bool BIG, bool AIMG = false, bool BIMG = false, class FA, class FB, class ST>
__device__ void emu_tile(int K, FA fa, FB fb, const int* eA, const int* eB, ST st, int* err,
                         const unsigned char* imgA = nullptr, const unsigned char* imgB = nullptr,
                         size_t img_stride = 0, size_t img_stride_b = 0)
{
    if (img_stride_b == 0) img_stride_b = img_stride;
    constexpr bool kImg = AIMG || BIMG;
    constexpr uint32_t kImgBytes = (AIMG ? ENS * E_ATILE : 0) + (BIMG ? ENS * E_BTILE : 0);
    extern __shared__ __align__(1024) unsigned char esm[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ __align__(8) uint64_t s_full[2];
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* base = (unsigned char*)(((uintptr_t)esm + 1023) & ~(uintptr_t)1023);
    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_full[s])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = idesc_bf16(EM, EN);
    const int nchk = (K + EK - 1) / EK;
    constexpr int CH = E_KSUPER / EK;   // chunks per exact accumulation
    int sh = 0;
    if (BIG)
        while ((long long)K > (8192ll << sh)) ++sh;
    // epilogue mapping: thread (quadrant qd, half h) owns row m, columns h*32 .. h*32+31
    const int qd = warp & 3, h = warp >> 2, m = qd * 32 + lane;
    long long R[BIG ? 32 : 1];
#pragma unroll
    for (int u = 0; u < (BIG ? 32 : 1); ++u) R[u] = 0;
    // The exact levels hold integers I_l 2^{-7l} (|I_l| < 2^24): their sum is
    // the integer S = sum_l I_l 2^{7(5-l)} in units of 2^-35 (|I_0| <= 2^23,
    // so |S| < 2^58.02 for K <= 512), formed exactly in 64-bit integers; the shared low levels
    // (weights 2^-35 .. 2^-49) are rounded to that unit, 2^-57 of the level-0
    // unit.  One conversion to FP64, the scale 2^{E_m + F_n - 49} in the
    // exponent field.
    auto drain = [&](bool last) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int j0 = h * 32 + g * 8;
            long long S[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) S[u] = 0;
#pragma unroll
            for (int l = 0; l < ENACC; ++l) {
                uint32_t v[8];
                const uint32_t addr = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(l * EN + j0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                    : "r"(addr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // 2^{7 l} for the exact levels, 2^{35 - sh} for the shared one
                const float up = __int_as_float((127 + (l < ENACC - 1 ? 7 * l : 7 * l - sh)) << 23);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int x = __float2int_rn(__uint_as_float(v[u]) * up);   // |x| < 2^24 (2^18 for the shared one)
                    S[u] += l < ENACC - 1 ? ((long long)x << (7 * (ENACC - 1 - l) - sh)) : (long long)x;
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (BIG) {
                    R[g * 8 + u] += S[u];
                    if (last) st(m, j0 + u, i64_scaled(R[g * 8 + u], eA[m] + eB[j0 + u] - 49 + sh));
                } else {
                    st(m, j0 + u, i64_scaled(S[u], eA[m] + eB[j0 + u] - 49));
                }
            }
        }
    };
    uint32_t uses[2] = {0, 0};
    // operand registers of one chunk: A items (r, g) = tid, tid + 256 (rows
    // r = it % 128, eight K values g * 8 ..), B item (n, g) = tid; the next
    // chunk's loads are issued before the current chunk's MMAs
    double xa[2][8], xb[8];
    auto load_chunk = [&](int c) {
        if constexpr (!AIMG) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int it = tid + E_T * i, r = it & (EM - 1), k0 = c * EK + (it >> 7) * 8;
#pragma unroll
                for (int u = 0; u < 8; ++u) xa[i][u] = k0 + u < K ? fa(r, k0 + u) : 0.0;
            }
        }
        if constexpr (!BIMG) {
            const int n = tid & (EN - 1), k0 = c * EK + (tid >> 6) * 8;
#pragma unroll
            for (int u = 0; u < 8; ++u) xb[u] = k0 + u < K ? fb(k0 + u, n) : 0.0;
        }
    };
    // thread 0: the image slices of chunk c into stage c & 1 (free: its
    // previous MMAs complete), completing on s_full
    int img_issued = 0, img_waited = 0;
    auto issue_img = [&](int c) {
        unsigned char* sa = base + (c & 1) * E_STAGE;
        unsigned char* sb = sa + ENS * E_ATILE;
        const uint32_t fb_ = smem_u32(&s_full[c & 1]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb_), "r"(kImgBytes) : "memory");
#pragma unroll
        for (int p = 0; p < ENS; ++p) {
            if constexpr (AIMG)
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                 smem_u32(sa + p * E_ATILE)),
                             "l"(imgA + ((size_t)c * ENS + p) * img_stride), "r"(E_ATILE), "r"(fb_)
                             : "memory");
            if constexpr (BIMG)
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                 smem_u32(sb + p * E_BTILE)),
                             "l"(imgB + ((size_t)c * ENS + p) * img_stride_b), "r"(E_BTILE), "r"(fb_)
                             : "memory");
        }
        ++img_issued;
    };
    if (kImg && tid == 0) issue_img(0);
    load_chunk(0);
    for (int c = 0; c < nchk; ++c) {
        const int s = c & 1;
        unsigned char* st_a = base + s * E_STAGE;
        unsigned char* st_b = st_a + ENS * E_ATILE;
        if (c >= 2 && !mbar_wait(smem_u32(&s_bar[s]), (uses[s] - 1) & 1)) s_fail = 1;
        if constexpr (!AIMG) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int it = tid + E_T * i, r = it & (EM - 1);
                store_slices(st_a, E_ATILE, r, (it >> 7) * 8, xa[i], eA[r]);
            }
        }
        if constexpr (!BIMG) {
            const int n = tid & (EN - 1);
            store_slices(st_b, E_BTILE, n, (tid >> 6) * 8, xb, eB[n]);
        }
        if (c + 1 < nchk) load_chunk(c + 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s_fail) break;
        if (tid == 0) {
            bool landed = true;
            if constexpr (kImg) {
                landed = mbar_wait(smem_u32(&s_full[s]), (uint32_t)(c >> 1) & 1u);
                ++img_waited;
                if (!landed) s_fail = 1;   // no MMA on slices that did not land; the commit still arrives
            }
            if (landed) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(st_a), b0 = smem_u32(st_b);
            const bool first = (c % CH) == 0;   // the first chunk of an exact accumulation
#pragma unroll
            for (int ks = 0; ks < EK / 16; ++ks) {
                const uint32_t koff = ks * 256;
#pragma unroll
                for (int p = 1; p <= ENS; ++p) {
                    const uint64_t da = smem_desc(a0 + (p - 1) * E_ATILE + koff, 128, 512);
#pragma unroll
                    for (int q = 1; q <= ENS + 1 - p; ++q) {
                        const uint64_t db = smem_desc(b0 + (q - 1) * E_BTILE + koff, 128, 512);
                        const int l = p + q - 2 < ENACC - 1 ? p + q - 2 : ENACC - 1;
                        const uint32_t acc = (!first || ks > 0 || p > 1 || q > ENACC) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred pp;\n setp.ne.b32 pp, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n" ::"r"(tmem + (uint32_t)(l * EN)),
                            "l"(da), "l"(db), "r"(idesc), "r"(acc));
                    }
                }
            }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&s_bar[s]))
                         : "memory");
        }
        uses[s]++;
        if (kImg && tid == 0 && c + 1 < nchk && !s_fail) {
            // the next chunk's slices, once the MMAs of chunk c - 1 (its stage) are complete
            const int s1 = (c + 1) & 1;
            if (c >= 1 && !mbar_wait(smem_u32(&s_bar[s1]), (uses[s1] - 1) & 1)) s_fail = 1;
            else issue_img(c + 1);
        }
        if (BIG && (c + 1) % CH == 0 && c + 1 < nchk) {
            // drain this exact accumulation before the next one overwrites it
            if (!mbar_wait(smem_u32(&s_bar[s]), (uses[s] - 1) & 1)) s_fail = 1;
            __syncthreads();
            if (s_fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            drain(false);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }
    // image copies issued but not waited for (a failed tile breaks early)
    if (kImg && tid == 0)
        for (int c = img_waited; c < img_issued; ++c) mbar_wait(smem_u32(&s_full[c & 1]), (uint32_t)(c >> 1) & 1u);
    __syncthreads();
    if (!s_fail)
        for (int s = 0; s < 2; ++s)
            if (uses[s] > 0 && !mbar_wait(smem_u32(&s_bar[s]), (uses[s] - 1) & 1)) s_fail = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fail)
        drain(true);
    else if (tid == 0)
        atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

namespace {

// Row scale exponents of an Aop tile (rows m < M) and column exponents of a
// Bop tile: E = 1 + the largest entry exponent (0 for an all-zero line).
template <class F>
__device__ void line_exponents(int lines, int K, F f, int* out, int* scratch)
{
    // thread t: line t % lines, K range split over the threads of that line
    const int per = E_T / lines;
    const int li = threadIdx.x % lines, part = threadIdx.x / lines;
    int mx = -1100;
    if (part < per)
        for (int k0 = part; k0 < K; k0 += 8 * per) {
            // eight independent loads in flight per thread
            double x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = k0 + u * per < K ? f(li, k0 + u * per) : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) mx = max(mx, exp2_of(x[u]));
        }
    scratch[threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.x < lines) {
        int m = -1100;
        for (int p = 0; p < per; ++p) m = max(m, scratch[threadIdx.x + lines * p]);
        out[threadIdx.x] = m <= -1100 ? 0 : m + 1;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(E_T, 1) k_emu_gemm(int M, int N, int K, const double* __restrict__ A, int lda,
                                                     int transA, const double* __restrict__ B, int ldb,
                                                     double* __restrict__ C, int ldc, int* err)
{
    __shared__ int s_eA[EM], s_eB[EN], s_scr[E_T];
    const int m0 = blockIdx.x * EM, n0 = blockIdx.y * EN;
    auto fa = [&](int m, int k) -> double {
        const int mm = m0 + m;
        if (mm >= M || k >= K) return 0.0;
        return transA ? A[k + (size_t)lda * mm] : A[mm + (size_t)lda * k];
    };
    auto fb = [&](int k, int n) -> double {
        const int nn = n0 + n;
        return (nn < N && k < K) ? B[k + (size_t)ldb * nn] : 0.0;
    };
    line_exponents(EM, K, fa, s_eA, s_scr);
    line_exponents(EN, K, [&](int n, int k) { return fb(k, n); }, s_eB, s_scr);
    emu_tile<false>(K, fa, fb, s_eA, s_eB,
             [&](int m, int n, double v) {
                 if (m0 + m < M && n0 + n < N) C[(m0 + m) + (size_t)ldc * (n0 + n)] = v;
             },
             err);
}

// Line exponents of a whole matrix for the products with K > 256: out[i] =
// max over line i of (exponent + 2048), 0 for an all-zero line (out zeroed
// by the caller; atomicMax over K ranges).  by_row: line i = row i of the
// column-major X (X[i + ld k]); else column i (X[k + ld i]).
__global__ void k_emu_line_exps(int lines, int K, const double* __restrict__ X, int ld, int by_row, int* out)
{
    if (by_row) {
        const int i = blockIdx.x * blockDim.x + threadIdx.x, k0 = blockIdx.y * 64;
        if (i >= lines) return;
        int mx = -1100;
        for (int kk = k0; kk < min(K, k0 + 64); kk += 8) {
            double x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = kk + u < K ? X[i + (size_t)ld * (kk + u)] : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) mx = max(mx, exp2_of(x[u]));
        }
        if (mx > -1100) atomicMax(&out[i], mx + 2048);
    } else {
        const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
        if (i >= lines) return;
        const int k0 = blockIdx.y * 256;
        int mx = -1100;
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int kk = k0 + lane + 32 * u;
            x[u] = kk < K ? X[kk + (size_t)ld * i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) mx = max(mx, exp2_of(x[u]));
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && mx > -1100) atomicMax(&out[i], mx + 2048);
    }
}

// C = op(A) B (+ C when accumulate) for any K, FP64-accurate; tiles wholly
// above the diagonal are skipped when lower (the caller mirrors).
// With kchunk > 0 (split K): block z takes K values [z kchunk, (z+1) kchunk)
// and writes its M x N partial to C + z M N (ld M); the caller sums them.
template <bool IMG>
__global__ void __launch_bounds__(E_T, 1) k_emu_gemm_big(int M, int N, int K, const double* __restrict__ A, int lda,
                                                         int transA, const double* __restrict__ B, int ldb,
                                                         int accumulate, double* __restrict__ C, int ldc, int lower,
                                                         const int* __restrict__ xA, const int* __restrict__ xB,
                                                         int* err, int kchunk, const unsigned char* imgA,
                                                         const unsigned char* imgB, size_t strideA, size_t strideB)
{
    __shared__ int s_eA[EM], s_eB[EN];
    const int m0 = blockIdx.x * EM, n0 = blockIdx.y * EN;
    if (lower && m0 + EM - 1 < n0) return;
    int kb = 0;
    if (kchunk > 0) {   // this block's K range and partial
        kb = blockIdx.z * kchunk;
        K = min(K - kb, kchunk);
        C += (size_t)blockIdx.z * M * N;
        ldc = M;
        accumulate = 0;
    }
    for (int i = threadIdx.x; i < EM + EN; i += E_T) {
        const int v = i < EM ? (m0 + i < M ? xA[m0 + i] : 0) : (n0 + i - EM < N ? xB[n0 + i - EM] : 0);
        const int e = v == 0 ? 0 : v - 2048 + 1;
        if (i < EM) s_eA[i] = e;
        else s_eB[i - EM] = e;
    }
    __syncthreads();
    auto fa = [&](int m, int k) -> double {
        const int mm = m0 + m;
        if (mm >= M || k >= K) return 0.0;
        return transA ? A[kb + k + (size_t)lda * mm] : A[mm + (size_t)lda * (kb + k)];
    };
    auto fb = [&](int k, int n) -> double {
        const int nn = n0 + n;
        return (nn < N && k < K) ? B[kb + k + (size_t)ldb * nn] : 0.0;
    };
    auto stc = [&](int m, int n, double v) {
        if (m0 + m < M && n0 + n < N) {
            double* c = C + (m0 + m) + (size_t)ldc * (n0 + n);
            *c = accumulate ? *c + v : v;
        }
    };
    if constexpr (IMG)   // both operands' slices from the images (K chunks from kb, kb a multiple of 32)
        emu_tile<true, true, true>(K, fa, fb, s_eA, s_eB, stc, err,
                                   imgA + (size_t)(kb / EK) * ENS * strideA + (size_t)m0 * EK * 2,
                                   imgB + (size_t)(kb / EK) * ENS * strideB + (size_t)n0 * EK * 2, strideA, strideB);
    else
        emu_tile<true>(K, fa, fb, s_eA, s_eB, stc, err);
}

// The slices of `lines` lines of op(X) over K (line i: X[i + ld k] when
// trans = 0, X[k + ld i] when trans = 1), with the line scales of
// k_emu_line_exps (exponent + 2048, 0 for an all-zero line), into an image
// whose slice blocks hold R rows (R >= lines, a multiple of 64; padding rows
// zero): slice p of chunk c at img + (8 c + p) R 64 bytes, row r at
// tile_off(r, k - 32 c).  Block (c, g): rows 64 g .. 64 g + 63.
__global__ void __launch_bounds__(E_T) k_emu_slice_lines(int lines, int K, const double* __restrict__ X, int ld,
                                                         int trans, const int* __restrict__ xexp, int R,
                                                         unsigned char* __restrict__ img)
{
    const int c = blockIdx.x, r = blockIdx.y * 64 + (threadIdx.x & 63), g = threadIdx.x >> 6;
    const size_t sb = (size_t)R * EK * 2;
    const int k0 = c * EK + g * 8;
    double x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int kk = k0 + u;
        x[u] = (r < lines && kk < K) ? (trans ? X[kk + (size_t)ld * r] : X[r + (size_t)ld * kk]) : 0.0;
    }
    const int v = r < lines ? xexp[r] : 0;
    store_slices(img + (size_t)c * ENS * sb, (int)sb, r, g * 8, x, v == 0 ? 0 : v - 2048 + 1);
}

}  // namespace

cudaError_t launch_emu_gemm(int M, int N, int K, const double* A, int lda, int transA, const double* B, int ldb,
                            double* C, int ldc, int* err, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_emu_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, E_SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((M + EM - 1) / EM, (N + EN - 1) / EN);
    k_emu_gemm<<<grid, E_T, E_SMEM, s>>>(M, N, K, A, lda, transA, B, ldb, C, ldc, err);
    return cudaGetLastError();
}

size_t emu_gemm_img_bytes(int lines, int K)
{
    const size_t R = ((size_t)lines + EM - 1) / EM * EM;
    return ((size_t)K + EK - 1) / EK * ENS * R * EK * 2;
}

cudaError_t launch_emu_gemm_img(int M, int N, int K, const double* A, int lda, int transA, const double* B, int ldb,
                                int accumulate, double* C, int ldc, int lower, int* xA, int* xB,
                                unsigned char* imgA, unsigned char* imgB, int* err, cudaStream_t s)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_emu_gemm_big<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, E_SMEM);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(xA, 0, sizeof(int) * M, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(xB, 0, sizeof(int) * N, s)) != cudaSuccess)
        return e;
    if (transA)
        k_emu_line_exps<<<dim3((M + 7) / 8, (K + 255) / 256), 256, 0, s>>>(M, K, A, lda, 0, xA);
    else
        k_emu_line_exps<<<dim3((M + 255) / 256, (K + 63) / 64), 256, 0, s>>>(M, K, A, lda, 1, xA);
    k_emu_line_exps<<<dim3((N + 7) / 8, (K + 255) / 256), 256, 0, s>>>(N, K, B, ldb, 0, xB);
    const int RA = (M + EM - 1) / EM * EM, RB = (N + EM - 1) / EM * EM, nchk = (K + EK - 1) / EK;
    k_emu_slice_lines<<<dim3(nchk, RA / 64), E_T, 0, s>>>(M, K, A, lda, transA, xA, RA, imgA);
    k_emu_slice_lines<<<dim3(nchk, RB / 64), E_T, 0, s>>>(N, K, B, ldb, 1, xB, RB, imgB);
    dim3 grid((M + EM - 1) / EM, (N + EN - 1) / EN);
    k_emu_gemm_big<true><<<grid, E_T, E_SMEM, s>>>(M, N, K, A, lda, transA, B, ldb, accumulate, C, ldc, lower, xA,
                                                   xB, err, 0, imgA, imgB, (size_t)RA * EK * 2,
                                                   (size_t)RB * EK * 2);
    return cudaGetLastError();
}

cudaError_t launch_emu_gemm_big(int M, int N, int K, const double* A, int lda, int transA, const double* B, int ldb,
                                int accumulate, double* C, int ldc, int lower, int* xA, int* xB, int* err,
                                cudaStream_t s)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_emu_gemm_big<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, E_SMEM);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(xA, 0, sizeof(int) * M, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(xB, 0, sizeof(int) * N, s)) != cudaSuccess)
        return e;
    if (transA)   // rows of A^T: columns of A
        k_emu_line_exps<<<dim3((M + 7) / 8, (K + 255) / 256), 256, 0, s>>>(M, K, A, lda, 0, xA);
    else
        k_emu_line_exps<<<dim3((M + 255) / 256, (K + 63) / 64), 256, 0, s>>>(M, K, A, lda, 1, xA);
    k_emu_line_exps<<<dim3((N + 7) / 8, (K + 255) / 256), 256, 0, s>>>(N, K, B, ldb, 0, xB);
    dim3 grid((M + EM - 1) / EM, (N + EN - 1) / EN);
    k_emu_gemm_big<false><<<grid, E_T, E_SMEM, s>>>(M, N, K, A, lda, transA, B, ldb, accumulate, C, ldc, lower, xA,
                                                    xB, err, 0, nullptr, nullptr, 0, 0);
    return cudaGetLastError();
}

namespace {
// W(a, c) = sum_z part_z(c, a), fixed order: the transposed sum of the
// split-K partials (each M x N, ld M) into W (N x M, ld ldw).
__global__ void k_emu_sum_t(int M, int N, int nsplit, const double* __restrict__ part, double* __restrict__ W, int ldw)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)M * N) return;
    const int c = (int)(i % M), a = (int)(i / M);
    double v = 0.0;
    for (int z = 0; z < nsplit; ++z) v += part[(size_t)z * M * N + i];
    W[a + (size_t)ldw * c] = v;
}
}  // namespace

cudaError_t launch_emu_gemm_tsplit(int M, int N, int K, const double* A, int lda, int transA, const double* B, int ldb,
                                   double* W, int ldw, int kchunk, double* part, int* xA, int* xB, int* err,
                                   cudaStream_t s)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_emu_gemm_big<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, E_SMEM);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(xA, 0, sizeof(int) * M, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(xB, 0, sizeof(int) * N, s)) != cudaSuccess)
        return e;
    if (transA)
        k_emu_line_exps<<<dim3((M + 7) / 8, (K + 255) / 256), 256, 0, s>>>(M, K, A, lda, 0, xA);
    else
        k_emu_line_exps<<<dim3((M + 255) / 256, (K + 63) / 64), 256, 0, s>>>(M, K, A, lda, 1, xA);
    k_emu_line_exps<<<dim3((N + 7) / 8, (K + 255) / 256), 256, 0, s>>>(N, K, B, ldb, 0, xB);
    const int nsplit = (K + kchunk - 1) / kchunk;
    dim3 grid((M + EM - 1) / EM, (N + EN - 1) / EN, nsplit);
    k_emu_gemm_big<false><<<grid, E_T, E_SMEM, s>>>(M, N, K, A, lda, transA, B, ldb, 0, part, M, 0, xA, xB, err,
                                                    kchunk, nullptr, nullptr, 0, 0);
    const long long total = (long long)M * N;
    k_emu_sum_t<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(M, N, nsplit, part, W, ldw);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- emulated FP64 step update
namespace {

__device__ __forceinline__ int emap(int I, int J, int b, int x) { return x < b ? I * b + x : J * b + (x - b); }

__device__ __forceinline__ void eentry(const int2* pairs, int e, int& I, int& J)
{
    const int2 pr = pairs[e];
    I = pr.x < 0 ? -1 - pr.x : pr.x;
    J = pr.x < 0 ? -1 - pr.y : pr.y;
}

__device__ __forceinline__ void edecode_pb(int pb, int& e1, int& e2)
{
    int t = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)pb)) * 0.5f);
    while (t * (t - 1) / 2 > pb) --t;
    while ((t + 1) * t / 2 <= pb) ++t;
    e2 = t;
    e1 = pb - t * (t - 1) / 2;
}

// ---------------------------------------------------------------- V sliced once per step
// Rows of the image (the index n of V(kk, n)) are padded to a multiple of
// 128 so that the 128-row tiles of stage 2 and the 64-row tiles of stage 1
// are whole: per pair, nchk = ceil(k / 32) chunks x 8 slices x kr * 64
// bytes (kr = k rounded up to 128), slice p of chunk c holding element
// (n, kk) of V^T at tile_off(n, kk - 32 c).
__host__ __device__ __forceinline__ int emu_img_rows(int k) { return (k + EM - 1) / EM * EM; }
__host__ __device__ __forceinline__ size_t emu_img_slice_bytes(int k) { return (size_t)emu_img_rows(k) * EK * 2; }

// Column scales of V per pair: vexp[e][n] = 1 + the largest exponent in
// column n of V_e (0 for an all-zero or padding column) -- the scale
// line_exponents takes for the same column.  One warp per column.
__global__ void k_emu_vexp(const double* __restrict__ V, const int* __restrict__ rot, int k, int* __restrict__ vexp)
{
    const int kr = emu_img_rows(k);
    const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int e = blockIdx.y;
    if (col >= kr) return;
    int mx = -1100;
    if (col < k && rot[e] != 0) {
        const double* Vt = V + (size_t)e * 2 * k * k + (size_t)k * k;   // V^T(n, kk) at Vt[n + k kk]
        for (int kk = lane; kk < k; kk += 32) mx = max(mx, exp2_of(Vt[col + (size_t)k * kk]));
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) vexp[(size_t)e * kr + col] = mx <= -1100 ? 0 : mx + 1;
}

// The eight slices of V^T per pair and K chunk (pairs without rotation are
// skipped: their updates copy).  Block (c, e): items (n, g), eight K values
// kk = 32 c + 8 g .. + 7 of row n.
__global__ void __launch_bounds__(E_T) k_emu_slice_v(const double* __restrict__ V, const int* __restrict__ rot, int k,
                                                     const int* __restrict__ vexp, unsigned char* __restrict__ img)
{
    const int c = blockIdx.x, e = blockIdx.y, kr = emu_img_rows(k), nchk = (k + EK - 1) / EK;
    if (rot[e] == 0) return;
    const double* Vt = V + (size_t)e * 2 * k * k + (size_t)k * k;
    const size_t sb = emu_img_slice_bytes(k);
    unsigned char* dst = img + ((size_t)e * nchk + c) * ENS * sb;
    for (int it = threadIdx.x; it < kr * 4; it += E_T) {
        const int n = it % kr, g = it / kr, k0 = c * EK + g * 8;
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = (n < k && k0 + u < k) ? Vt[n + (size_t)k * (k0 + u)] : 0.0;
        store_slices(dst, (int)sb, n, g * 8, x, vexp[(size_t)e * kr + n]);
    }
}

// Row scales of the stage-1 A operands: out[e][i] = 1 + the largest exponent
// of X(i, P_e) over the 2b columns of pair e (0 when all are zero), for the
// rows i < rows of X (the working A, or Q).  Thread = row (coalesced).
__global__ void k_emu_rowexp(int rows, const double* __restrict__ X, int ld, const int2* __restrict__ pairs,
                             int b, int* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, e = blockIdx.y;
    if (i >= rows) return;
    int I, J;
    eentry(pairs, e, I, J);
    int mx = -1100;
    for (int x = 0; x < 2 * b; ++x) mx = max(mx, exp2_of(X[i + (size_t)ld * emap(I, J, b, x)]));
    out[(size_t)e * rows + i] = mx <= -1100 ? 0 : mx + 1;
}

// The slices of the stage-1 A operands, once per step.  mode 0: pair-block
// pb = (e1 < e2), rows = pair e1's 2b rows of A, K = pair e2's 2b columns,
// row scales atab[e2][row] (the table has `rows` = np rows); its image
// (nchk x 8 slices x kr x 64 bytes) at img + pb * that.  mode 1: pair e,
// rows = all `rows` = qrows rows of Q, K = pair e's columns, row scales
// qexp[e][row]; image nchk x 8 x qr x 64 bytes at img + e * that.  Block (c, row group of 64, item); blocks whose V is the
// identity (no rotation: the update copies) are skipped.
__global__ void __launch_bounds__(E_T) k_emu_slice_ops(int mode, const double* __restrict__ X, int ld, int rows,
                                                       const int2* __restrict__ pairs, const int* __restrict__ rot,
                                                       int b, int k, const int* __restrict__ tab, int R,
                                                       unsigned char* __restrict__ img)
{
    const int c = blockIdx.x, r = blockIdx.y * 64 + (threadIdx.x & 63), g = threadIdx.x >> 6, item = blockIdx.z;
    const int nchk = (k + EK - 1) / EK;
    int eK, I1 = 0, J1 = 0, I2, J2;
    if (mode == 0) {
        int e1, e2;
        edecode_pb(item, e1, e2);
        eentry(pairs, e1, I1, J1);
        eentry(pairs, e2, I2, J2);
        eK = e2;
    } else {
        eentry(pairs, item, I2, J2);
        eK = item;
    }
    if (rot[eK] == 0) return;
    const int nrow = mode == 0 ? k : rows;
    const int grow = r < nrow ? (mode == 0 ? emap(I1, J1, b, r) : r) : -1;
    const size_t sb = (size_t)R * EK * 2;
    const int k0 = c * EK + g * 8;
    double x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int kk = k0 + u;
        x[u] = (grow >= 0 && kk < k) ? X[grow + (size_t)ld * emap(I2, J2, b, kk)] : 0.0;
    }
    const int E = grow >= 0 ? tab[(size_t)eK * rows + grow] : 0;
    store_slices(img + ((size_t)item * nchk + c) * ENS * sb, (int)sb, r, g * 8, x, E);
}

// Stage 1.  Items [0, n_sand): tile (mt, nt) of T_pb = A_{P1P2} V2 (FP64,
// k x k per pair-block); items beyond: tile (rt, nt) of Q'(:,P) = Q(:,P) V_P.
// V^T (stored after V by the pivot kernel) gives the coalesced operand loads.
template <bool BAL>
__global__ void __launch_bounds__(E_T, 1) k_emu_upd1(EmuUpdArgs a, int n_sand)
{
    __shared__ int s_eA[EM], s_eB[EN], s_scr[E_T];
    const UpdateArgs& u = a.u;
    const int k = u.k, b = u.b, nmt = (k + EM - 1) / EM, nnt = (k + EN - 1) / EN;
    int item = blockIdx.x;
    if (item < n_sand) {
        const int pb = item / (nmt * nnt), rem = item % (nmt * nnt), mt = rem / nnt, nt = rem % nnt;
        int e1, e2, I1, J1, I2, J2;
        edecode_pb(pb, e1, e2);
        eentry(u.pairs, e1, I1, J1);
        eentry(u.pairs, e2, I2, J2);
        double* T = a.T + (size_t)pb * k * k;
        const int m0 = mt * EM, n0 = nt * EN;
        if (u.rot[e2] == 0) {
            for (int idx = threadIdx.x; idx < EM * EN; idx += E_T) {
                const int m = m0 + idx % EM, j = n0 + idx / EM;
                if (m < k && j < k) T[m + (size_t)k * j] = u.Ain[emap(I1, J1, b, m) + (size_t)u.lda * emap(I2, J2, b, j)];
            }
            return;
        }
        const double* V2t = u.V + (size_t)e2 * 2 * k * k + (size_t)k * k;
        // with a.balance: A_P1P2 V2 = (A_P1P2 2^-c)(2^c V2), c_kk ~ log2
        // sqrt|a_jj| of column kk's diagonal entry: balanced operands for
        // graded positive definite matrices (exact; for indefinite matrices
        // a small diagonal entry says nothing about its column, so off)
        __shared__ int s_cs[256];
        if constexpr (BAL) {
            for (int kk = threadIdx.x; kk < k; kk += E_T) {
                const int g = emap(I2, J2, b, kk);
                const int ed = exp2_of(u.Ain[g + (size_t)u.lda * g]);
                s_cs[kk] = ed <= -1100 ? 0 : (ed >> 1);
            }
            __syncthreads();
        }
        auto fa = [&](int m, int kk) -> double {
            if (!(m0 + m < k && kk < k)) return 0.0;
            const double x = u.Ain[emap(I1, J1, b, m0 + m) + (size_t)u.lda * emap(I2, J2, b, kk)];
            if constexpr (BAL) return pow2_shift(x, s_cs[kk]);
            return x;
        };
        auto fb = [&](int kk, int n) -> double {
            if (!(n0 + n < k && kk < k)) return 0.0;
            const double x = V2t[(n0 + n) + (size_t)k * kk];
            if constexpr (BAL) return pow2_shift(x, -s_cs[kk]);
            return x;
        };
        auto stT = [&](int m, int n, double v) {
            if (m0 + m < k && n0 + n < k) T[(m0 + m) + (size_t)k * (n0 + n)] = v;
        };
        if (!BAL && a.vimg && a.aimg) {   // both operands' slices from the step's images
            const int kr = emu_img_rows(k), nchk = (k + EK - 1) / EK;
            const size_t sb = emu_img_slice_bytes(k);
            for (int m = threadIdx.x; m < EM; m += E_T)
                s_eA[m] = m0 + m < k ? a.atab[(size_t)e2 * u.lda + emap(I1, J1, b, m0 + m)] : 0;
            for (int n = threadIdx.x; n < EN; n += E_T) s_eB[n] = a.vexp[(size_t)e2 * kr + n0 + n];
            __syncthreads();
            const unsigned char* ia = a.aimg + (size_t)pb * nchk * ENS * sb + (size_t)m0 * EK * 2;
            const unsigned char* im = a.vimg + (size_t)e2 * nchk * ENS * sb + (size_t)n0 * EK * 2;
            emu_tile<false, true, true>(k, fa, fb, s_eA, s_eB, stT, a.err, ia, im, sb, sb);
        } else if (!BAL && a.vimg) {   // V2's slices from the step's image
            const int kr = emu_img_rows(k), nchk = (k + EK - 1) / EK;
            for (int n = threadIdx.x; n < EN; n += E_T) s_eB[n] = a.vexp[(size_t)e2 * kr + n0 + n];
            __syncthreads();
            const unsigned char* im = a.vimg + (size_t)e2 * nchk * ENS * emu_img_slice_bytes(k) + (size_t)n0 * EK * 2;
            line_exponents(EM, k, fa, s_eA, s_scr);
            emu_tile<false, false, true>(k, fa, fb, s_eA, s_eB, stT, a.err, nullptr, im, emu_img_slice_bytes(k));
        } else {
            line_exponents(EM, k, fa, s_eA, s_scr);
            line_exponents(EN, k, [&](int n, int kk) { return fb(kk, n); }, s_eB, s_scr);
            emu_tile<false>(k, fa, fb, s_eA, s_eB, stT, a.err);
        }
        if (threadIdx.x == 0) {
            atomicAdd(&u.cnt->flops_update, 2ull * EM * EN * k);
            atomicAdd(&u.cnt->flops_lowp, 72ull * EM * EN * k);
        }
        return;
    }
    item -= n_sand;
    const int nrt = (u.qrows + EM - 1) / EM;
    const int e = item / (nrt * nnt), rem = item % (nrt * nnt), rt = rem / nnt, nt = rem % nnt;
    int I, J;
    eentry(u.pairs, e, I, J);
    const int r0 = rt * EM, n0 = nt * EN;
    if (u.rot[e] == 0) {
        for (int idx = threadIdx.x; idx < EM * EN; idx += E_T) {
            const int m = r0 + idx % EM, j = n0 + idx / EM;
            if (m < u.qrows && j < k) {
                const size_t o = m + (size_t)u.ldq * emap(I, J, b, j);
                u.Qout[o] = u.Qin[o];
            }
        }
        return;
    }
    const double* Vt = u.V + (size_t)e * 2 * k * k + (size_t)k * k;
    auto fa = [&](int m, int kk) -> double {
        return r0 + m < u.qrows && kk < k ? u.Qin[(r0 + m) + (size_t)u.ldq * emap(I, J, b, kk)] : 0.0;
    };
    auto fb = [&](int kk, int n) -> double { return n0 + n < k && kk < k ? Vt[(n0 + n) + (size_t)k * kk] : 0.0; };
    auto stQ = [&](int m, int n, double v) {
        if (r0 + m < u.qrows && n0 + n < k) u.Qout[(r0 + m) + (size_t)u.ldq * emap(I, J, b, n0 + n)] = v;
    };
    if (a.vimg && a.qimg) {   // Q(:, P)'s and V_P's slices from the step's images
        const int kr = emu_img_rows(k), nchk = (k + EK - 1) / EK;
        const size_t sb = emu_img_slice_bytes(k), sq = emu_img_slice_bytes(u.qrows);
        for (int m = threadIdx.x; m < EM; m += E_T) s_eA[m] = r0 + m < u.qrows ? a.qexp[(size_t)e * u.qrows + r0 + m] : 0;
        for (int n = threadIdx.x; n < EN; n += E_T) s_eB[n] = a.vexp[(size_t)e * kr + n0 + n];
        __syncthreads();
        const unsigned char* iq = a.qimg + (size_t)e * nchk * ENS * sq + (size_t)r0 * EK * 2;
        const unsigned char* im = a.vimg + (size_t)e * nchk * ENS * sb + (size_t)n0 * EK * 2;
        emu_tile<false, true, true>(k, fa, fb, s_eA, s_eB, stQ, a.err, iq, im, sq, sb);
    } else if (a.vimg) {   // V_P's slices from the step's image (the Q items never balance)
        const int kr = emu_img_rows(k), nchk = (k + EK - 1) / EK;
        for (int n = threadIdx.x; n < EN; n += E_T) s_eB[n] = a.vexp[(size_t)e * kr + n0 + n];
        __syncthreads();
        const unsigned char* im = a.vimg + (size_t)e * nchk * ENS * emu_img_slice_bytes(k) + (size_t)n0 * EK * 2;
        line_exponents(EM, k, fa, s_eA, s_scr);
        emu_tile<false, false, true>(k, fa, fb, s_eA, s_eB, stQ, a.err, nullptr, im, emu_img_slice_bytes(k));
    } else {
        line_exponents(EM, k, fa, s_eA, s_scr);
        line_exponents(EN, k, [&](int n, int kk) { return fb(kk, n); }, s_eB, s_scr);
        emu_tile<false>(k, fa, fb, s_eA, s_eB, stQ, a.err);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&u.cnt->flops_update, 2ull * EM * EN * k);
        atomicAdd(&u.cnt->flops_lowp, 72ull * EM * EN * k);
    }
}

// Stage 2: tile (mt, nt) of O_pb = V1^T T_pb, written to A' at (P1 rows, P2
// columns) and mirrored.
template <bool BAL>
__global__ void __launch_bounds__(E_T, 1) k_emu_upd2(EmuUpdArgs a)
{
    __shared__ int s_eA[EM], s_eB[EN], s_scr[E_T];
    const UpdateArgs& u = a.u;
    const int k = u.k, b = u.b, nmt = (k + EM - 1) / EM, nnt = (k + EN - 1) / EN;
    const int item = blockIdx.x;
    const int pb = item / (nmt * nnt), rem = item % (nmt * nnt), mt = rem / nnt, nt = rem % nnt;
    int e1, e2, I1, J1, I2, J2;
    edecode_pb(pb, e1, e2);
    eentry(u.pairs, e1, I1, J1);
    eentry(u.pairs, e2, I2, J2);
    const double* T = a.T + (size_t)pb * k * k;
    const int m0 = mt * EM, n0 = nt * EN;
    double* Ao = u.Aout;
    const size_t lda = (size_t)u.lda;
    auto put = [&](int m, int n, double v) {
        const int gi = emap(I1, J1, b, m), gj = emap(I2, J2, b, n);
        Ao[gi + lda * gj] = v;
        Ao[gj + lda * gi] = v;
    };
    if (u.rot[e1] == 0) {
        for (int idx = threadIdx.x; idx < EM * EN; idx += E_T) {
            const int m = m0 + idx % EM, j = n0 + idx / EM;
            if (m < k && j < k) put(m, j, T[m + (size_t)k * j]);
        }
        return;
    }
    const double* V1t = u.V + (size_t)e1 * 2 * k * k + (size_t)k * k;   // V1^T(m, kk) at V1t[m + k kk]
    // with a.balance: V1^T T = (V1^T 2^c)(2^-c T), c_kk from the diagonal of
    // row kk of P1
    __shared__ int s_cs[256];
    if constexpr (BAL) {
        for (int kk = threadIdx.x; kk < k; kk += E_T) {
            const int g = emap(I1, J1, b, kk);
            const int ed = exp2_of(u.Ain[g + lda * g]);
            s_cs[kk] = ed <= -1100 ? 0 : (ed >> 1);
        }
        __syncthreads();
    }
    auto fa = [&](int m, int kk) -> double {
        if (!(m0 + m < k && kk < k)) return 0.0;
        const double x = V1t[(m0 + m) + (size_t)k * kk];
        if constexpr (BAL) return pow2_shift(x, -s_cs[kk]);
        return x;
    };
    auto fb = [&](int kk, int n) -> double {
        if (!(n0 + n < k && kk < k)) return 0.0;
        const double x = T[kk + (size_t)k * (n0 + n)];
        if constexpr (BAL) return pow2_shift(x, s_cs[kk]);
        return x;
    };
    auto stO = [&](int m, int n, double v) {
        if (m0 + m < k && n0 + n < k) put(m0 + m, n0 + n, v);
    };
    if (!BAL && a.vimg) {   // V1^T's slices from the step's image (rows of V1^T = columns of V1)
        const int kr = emu_img_rows(k), nchk = (k + EK - 1) / EK;
        for (int m = threadIdx.x; m < EM; m += E_T) s_eA[m] = a.vexp[(size_t)e1 * kr + m0 + m];
        __syncthreads();
        line_exponents(EN, k, [&](int n, int kk) { return fb(kk, n); }, s_eB, s_scr);
        const unsigned char* im = a.vimg + (size_t)e1 * nchk * ENS * emu_img_slice_bytes(k) + (size_t)m0 * EK * 2;
        emu_tile<false, true, false>(k, fa, fb, s_eA, s_eB, stO, a.err, im, nullptr, emu_img_slice_bytes(k));
    } else {
        line_exponents(EM, k, fa, s_eA, s_scr);
        line_exponents(EN, k, [&](int n, int kk) { return fb(kk, n); }, s_eB, s_scr);
        emu_tile<false>(k, fa, fb, s_eA, s_eB, stO, a.err);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&u.cnt->flops_update, 2ull * EM * EN * k);
        atomicAdd(&u.cnt->flops_lowp, 72ull * EM * EN * k);
    }
}

// ---------------------------------------------------------------- one-sided step (Algorithm 6)
// Gram partials: item (pair e, row panel r, tile mt, nt) of
// part[e][r] = G(rows_r, P)^T G(rows_r, P) (k x k), K = the panel's rows
// (<= 512: two exact accumulations); tiles wholly above the diagonal are
// skipped (the pivot reads the lower triangle).
__global__ void __launch_bounds__(E_T, 1) k_emu_gram(EmuSvdArgs a, int nmt, int nnt)
{
    __shared__ int s_eA[EM], s_eB[EN], s_scr[E_T];
    const int k = a.k, b = a.b;
    int item = blockIdx.x;
    const int nt = item % nnt;
    item /= nnt;
    const int mt = item % nmt;
    item /= nmt;
    const int r = item % a.npanels, e = item / a.npanels;
    const int m0 = mt * EM, n0 = nt * EN;
    if (m0 + EM - 1 < n0) return;
    int I, J;
    eentry(a.pairs, e, I, J);
    const int r0 = r * a.panel_rows, K = min(a.panel_rows, a.m - r0);
    const double* G = a.Gin;
    const size_t ld = (size_t)a.ldg;
    double* out = a.part + ((size_t)e * a.npanels + r) * k * k;
    auto fa = [&](int mm, int kk) -> double {
        return m0 + mm < k && kk < K ? G[(r0 + kk) + ld * emap(I, J, b, m0 + mm)] : 0.0;
    };
    auto fb = [&](int kk, int nn) -> double {
        return n0 + nn < k && kk < K ? G[(r0 + kk) + ld * emap(I, J, b, n0 + nn)] : 0.0;
    };
    line_exponents(EM, K, fa, s_eA, s_scr);
    line_exponents(EN, K, [&](int nn, int kk) { return fb(kk, nn); }, s_eB, s_scr);
    emu_tile<true>(K, fa, fb, s_eA, s_eB,
                   [&](int mm, int nn, double v) {
                       if (m0 + mm < k && n0 + nn < k) out[(m0 + mm) + (size_t)k * (n0 + nn)] = v;
                   },
                   a.err);
    if (threadIdx.x == 0) {
        atomicAdd(&a.cnt->flops_update, 2ull * EM * EN * K);
        atomicAdd(&a.cnt->flops_lowp, 72ull * EM * EN * K);
    }
}

// Column update: items [0, n_g): tile (rt, nt) of G'(:, P) = G(:, P) V_P;
// beyond: the same for V.  V^T (stored after V) gives coalesced loads.
// The columns of G(:, P) can differ by many orders of magnitude (the
// singular values of the graded inputs span ten decades); a row scale taken
// across them would leave a small column with errors relative to the large
// ones.  So G(:, P) = (G(:, P) 2^-c) (2^c V_P): column kk of G is scaled by
// 2^-c_kk, c_kk from the step's Gram diagonal (~ its norm), and row kk of V_P
// by 2^c_kk (both exact), and the row / column scales of the product are
// taken on the balanced operands, as the FP64 rounding of the sum would.
__global__ void __launch_bounds__(E_T, 1) k_emu_cols(EmuSvdArgs a, int n_g)
{
    __shared__ int s_eA[EM], s_eB[EN], s_scr[E_T];
    __shared__ int s_cs[256];   // column shifts (k <= 256)
    const int k = a.k, b = a.b, nnt = (k + EN - 1) / EN;
    int item = blockIdx.x;
    const double* Min = a.Gin;
    double* Mout = a.Gout;
    size_t ld = (size_t)a.ldg;
    int rows = a.m;
    if (item >= n_g) {
        item -= n_g;
        Min = a.Vin;
        Mout = a.Vout;
        ld = (size_t)a.ldv;
        rows = a.vrows;
    }
    const int nrt = (rows + EM - 1) / EM;
    const int e = item / (nrt * nnt), rem = item % (nrt * nnt), rt = rem / nnt, nt = rem % nnt;
    int I, J;
    eentry(a.pairs, e, I, J);
    const int r0 = rt * EM, n0 = nt * EN;
    if (a.rot[e] == 0) {
        for (int idx = threadIdx.x; idx < EM * EN; idx += E_T) {
            const int mm = r0 + idx % EM, j = n0 + idx / EM;
            if (mm < rows && j < k) {
                const size_t o = mm + ld * emap(I, J, b, j);
                Mout[o] = Min[o];
            }
        }
        return;
    }
    const double* Vt = a.Vh + (size_t)e * 2 * k * k + (size_t)k * k;
    const bool gitem = blockIdx.x < (unsigned)n_g;
    for (int kk = threadIdx.x; kk < k; kk += E_T) {
        int c = 0;
        if (gitem) {
            double d = 0.0;   // ||G(:, kk)||^2, the Gram diagonal summed over the panels
            for (int r = 0; r < a.npanels; ++r) d += a.part[((size_t)e * a.npanels + r) * k * k + (size_t)kk * (k + 1)];
            const int ed = exp2_of(d);
            c = ed <= -1100 ? 0 : (ed >> 1);
        }
        s_cs[kk] = c;
    }
    __syncthreads();
    auto fa = [&](int mm, int kk) -> double {
        return r0 + mm < rows && kk < k ? pow2_shift(Min[(r0 + mm) + ld * emap(I, J, b, kk)], s_cs[kk]) : 0.0;
    };
    auto fb = [&](int kk, int nn) -> double {
        return n0 + nn < k && kk < k ? pow2_shift(Vt[(n0 + nn) + (size_t)k * kk], -s_cs[kk]) : 0.0;
    };
    line_exponents(EM, k, fa, s_eA, s_scr);
    line_exponents(EN, k, [&](int nn, int kk) { return fb(kk, nn); }, s_eB, s_scr);
    emu_tile<false>(k, fa, fb, s_eA, s_eB,
                    [&](int mm, int nn, double v) {
                        if (r0 + mm < rows && n0 + nn < k) Mout[(r0 + mm) + ld * emap(I, J, b, n0 + nn)] = v;
                    },
                    a.err);
    if (threadIdx.x == 0) {
        atomicAdd(&a.cnt->flops_update, 2ull * EM * EN * k);
        atomicAdd(&a.cnt->flops_lowp, 72ull * EM * EN * k);
    }
}

}  // namespace

size_t emu_update_tbuf_doubles(int npairs, int k) { return (size_t)(npairs * (npairs - 1) / 2) * k * k; }
size_t emu_update_vimg_bytes(int npairs, int k)
{
    return (size_t)npairs * ((k + EK - 1) / EK) * ENS * emu_img_slice_bytes(k);
}
size_t emu_update_vexp_ints(int npairs, int k) { return (size_t)npairs * emu_img_rows(k); }
size_t emu_update_aimg_bytes(int npairs, int k)
{
    return (size_t)(npairs * (npairs - 1) / 2) * ((k + EK - 1) / EK) * ENS * emu_img_slice_bytes(k);
}
size_t emu_update_qimg_bytes(int npairs, int k, int qrows)
{
    return (size_t)npairs * ((k + EK - 1) / EK) * ENS * emu_img_slice_bytes(qrows);
}

cudaError_t launch_emu_update(const EmuUpdArgs& a, cudaStream_t s)
{
    const UpdateArgs& u = a.u;
    const int nmt = (u.k + EM - 1) / EM, nnt = (u.k + EN - 1) / EN;
    if (a.vimg && u.npairs > 0) {   // V sliced once for the whole step
        const int kr = emu_img_rows(u.k);
        k_emu_vexp<<<dim3((kr + 7) / 8, u.npairs), 256, 0, s>>>(u.V, u.rot, u.k, a.vexp);
        k_emu_slice_v<<<dim3((u.k + EK - 1) / EK, u.npairs), E_T, 0, s>>>(u.V, u.rot, u.k, a.vexp, a.vimg);
        cudaError_t e0 = cudaGetLastError();
        if (e0 != cudaSuccess) return e0;
        const int nchk = (u.k + EK - 1) / EK;
        const int npb = u.npairs * (u.npairs - 1) / 2;
        if (a.aimg && !a.balance && npb > 0) {   // the pair-blocks of A, sliced once
            k_emu_rowexp<<<dim3((u.lda + 255) / 256, u.npairs), 256, 0, s>>>(u.lda, u.Ain, u.lda, u.pairs, u.b, a.atab);
            k_emu_slice_ops<<<dim3(nchk, emu_img_rows(u.k) / 64, npb), E_T, 0, s>>>(
                0, u.Ain, u.lda, u.lda, u.pairs, u.rot, u.b, u.k, a.atab, emu_img_rows(u.k), a.aimg);
        }
        if (a.qimg && u.Qin) {   // the column pairs of Q, sliced once
            k_emu_rowexp<<<dim3((u.qrows + 255) / 256, u.npairs), 256, 0, s>>>(u.qrows, u.Qin, u.ldq, u.pairs, u.b, a.qexp);
            k_emu_slice_ops<<<dim3(nchk, emu_img_rows(u.qrows) / 64, u.npairs), E_T, 0, s>>>(
                1, u.Qin, u.ldq, u.qrows, u.pairs, u.rot, u.b, u.k, a.qexp, emu_img_rows(u.qrows), a.qimg);
        }
        if ((e0 = cudaGetLastError()) != cudaSuccess) return e0;
    }
    const int npb = u.npairs * (u.npairs - 1) / 2;
    const int n_sand = npb * nmt * nnt;
    const int n_q = u.Qin ? u.npairs * ((u.qrows + EM - 1) / EM) * nnt : 0;
    auto u1 = a.balance ? k_emu_upd1<true> : k_emu_upd1<false>;
    auto u2 = a.balance ? k_emu_upd2<true> : k_emu_upd2<false>;
    cudaError_t e = cudaFuncSetAttribute(u1, cudaFuncAttributeMaxDynamicSharedMemorySize, E_SMEM);
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(u2, cudaFuncAttributeMaxDynamicSharedMemorySize, E_SMEM)) != cudaSuccess)
        return e;
    if (n_sand + n_q > 0) u1<<<n_sand + n_q, E_T, E_SMEM, s>>>(a, n_sand);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n_sand > 0) u2<<<n_sand, E_T, E_SMEM, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_emu_gram(const EmuSvdArgs& a, cudaStream_t s)
{
    const int nmt = (a.k + EM - 1) / EM, nnt = (a.k + EN - 1) / EN;
    const long long items = (long long)a.npairs * a.npanels * nmt * nnt;
    if (items <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_emu_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, E_SMEM);
    if (e != cudaSuccess) return e;
    k_emu_gram<<<(unsigned)items, E_T, E_SMEM, s>>>(a, nmt, nnt);
    return cudaGetLastError();
}

cudaError_t launch_emu_cols(const EmuSvdArgs& a, cudaStream_t s)
{
    const int nnt = (a.k + EN - 1) / EN;
    const int n_g = a.npairs * ((a.m + EM - 1) / EM) * nnt;
    const int n_v = a.Vin ? a.npairs * ((a.vrows + EM - 1) / EM) * nnt : 0;
    if (n_g + n_v == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_emu_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, E_SMEM);
    if (e != cudaSuccess) return e;
    k_emu_cols<<<n_g + n_v, E_T, E_SMEM, s>>>(a, n_g);
    return cudaGetLastError();
}

}  // namespace jac

// FP64-accurate product on the tensor cores (see the top of this file).
extern "C" int jacobi_f64emu_gemm(int M, int N, int K, const double* A, int lda, int transA, const double* B,
                                  int ldb, double* C, int ldc, void* stream)
{
    if (M < 0 || N < 0 || K < 0) return -1;
    if (K > (8192 << 7)) return JACOBI_ERR_UNSUPPORTED;
    if (!A || !B || !C) return -5;
    if ((!transA && lda < M) || (transA && lda < K) || ldb < K || ldc < M) return -5;
    if (M == 0 || N == 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (K == 0) {
        if (cudaMemset2DAsync(C, (size_t)ldc * 8, 0, (size_t)M * 8, N, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        return 0;
    }
    int* err = nullptr;
    const bool big = K > 256;
    if (cudaMallocAsync(&err, sizeof(int) * (1 + (big ? M + N : 0)), s) != cudaSuccess) return JACOBI_ERR_ALLOC;
    int h = 0, rc = 0;
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess ||
        (big ? jac::launch_emu_gemm_big(M, N, K, A, lda, transA, B, ldb, 0, C, ldc, 0, err + 1, err + 1 + M, err, s)
             : jac::launch_emu_gemm(M, N, K, A, lda, transA, B, ldb, C, ldc, err, s)) != cudaSuccess ||
        cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        rc = JACOBI_ERR_CUDA;
    cudaFreeAsync(err, s);
    cudaStreamSynchronize(s);
    if (rc == 0 && h) rc = JACOBI_ERR_TIMEOUT;
    return rc;
}
