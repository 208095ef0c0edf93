// k_fp64.cu -- FP64 kernels of the blocked Jacobi step on sm_103a.
//
// GB300's FP64 pipe issues about two DFMA per clock per SM (1.2 TFLOP/s for
// the GPU), so every kernel here is shaped to issue as few FP64 operations as
// possible; memory traffic is far below what HBM/L2 can move at that rate.
//
//   k_pivot      one CTA per pair: the 2b x 2b pivot of Algorithm 2 (line
//                "diagonalise the subproblem"), solved by parallel-ordered
//                scalar Jacobi (Algorithm 2 applied with b = 1) in FP64.  The
//                symmetric pivot lives in shared memory in packed lower form;
//                one round rotates every disjoint 2x2 "quad" from both sides
//                (J_i^T X J_j), a third fewer operations than separate row and
//                column passes.
//   k_update_evd the block-row and block-column updates of Algorithm 2 for all
//                pairs of a step, fused per pair-block: A'_{P1P2} =
//                V_{P1}^T A_{P1P2} V_{P2} is computed once and written with its
//                mirror (A stays exactly symmetric), plus Q'(:,P) = Q(:,P) V_P.
//                A and Q are double-buffered, so no tile is read after it has
//                been overwritten.
//   k_gram       split-K Gram blocks G(rows, P)^T G(rows, P) of the one-sided
//                method (Sec. 6), lower triangle only.
//   k_update_cols  G'(:,P) = G(:,P) V_P and V'(:,P) = V(:,P) V_P (Algorithm 6).
//   k_offnorm    Xi(A)^2 (Sec. 2.1) and ||A||_F^2 with a fixed-order two-level
//                reduction (deterministic), plus the relative measure.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"
#include "jacobi_core.cuh"
#include "qrcp.cuh"

namespace jac {

// Global row/column of local index x (0..2b-1) of the block pair (I, J).
__device__ __forceinline__ int pair_map(int I, int J, int b, int x)
{
    return x < b ? I * b + x : J * b + (x - b);
}

// Schedule entry e: the two blocks and whether the entry is frozen (blocks a
// step of Algorithm 3 leaves out; their transform is the identity).
__device__ __forceinline__ bool entry(const int2* pairs, int e, int& I, int& J)
{
    const int2 pr = pairs[e];
    const bool frozen = pr.x < 0;
    I = frozen ? -1 - pr.x : pr.x;
    J = frozen ? -1 - pr.y : pr.y;
    return frozen;
}

// ======================================================================== load
__global__ void k_load_sym(int n, int np, const double* __restrict__ A, int lda,
                           double* __restrict__ Aw, const double* __restrict__ Qin, int ldq,
                           double* __restrict__ Qw, int warm, DevCounters* cnt)
{
    const long long total = (long long)np * np;
    int bad = 0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int i = (int)(idx % np), j = (int)(idx / np);
        double v = 0.0;
        if (i < n && j < n) {
            v = i >= j ? A[i + (size_t)lda * j] : A[j + (size_t)lda * i];
            if (!isfinite(v)) bad = 1;
        }
        Aw[idx] = v;
        if (Qw) {
            double q = (i == j) ? 1.0 : 0.0;
            if (warm && i < n && j < n) q = Qin[i + (size_t)ldq * j];
            Qw[idx] = q;
        }
    }
    if (bad) atomicExch(&cnt->nonfinite, 1);
}

cudaError_t launch_load_sym(int n, int np, const double* A, int lda, double* Aw,
                            const double* Qin, int ldq, double* Qw, int warm, DevCounters* cnt,
                            cudaStream_t s)
{
    long long total = (long long)np * np;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_load_sym<<<blocks, 256, 0, s>>>(n, np, A, lda, Aw, Qin, ldq, Qw, warm, cnt);
    return cudaGetLastError();
}

__global__ void k_load_svd(int m, int n, int np, const double* __restrict__ G, int ldg,
                           double* __restrict__ Gw, double* __restrict__ Vw, DevCounters* cnt)
{
    const long long totg = (long long)m * np, totv = (long long)np * np;
    int bad = 0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < totg + totv;
         idx += (long long)gridDim.x * blockDim.x) {
        if (idx < totg) {
            int r = (int)(idx % m), j = (int)(idx / m);
            double v = j < n ? G[r + (size_t)ldg * j] : 0.0;
            if (!isfinite(v)) bad = 1;
            Gw[idx] = v;
        } else if (Vw) {
            long long t = idx - totg;
            int i = (int)(t % np), j = (int)(t / np);
            Vw[t] = (i == j) ? 1.0 : 0.0;
        }
    }
    if (bad) atomicExch(&cnt->nonfinite, 1);
}

cudaError_t launch_load_svd(int m, int n, int np, const double* G, int ldg, double* Gw,
                            double* Vw, DevCounters* cnt, cudaStream_t s)
{
    long long total = (long long)m * np + (long long)np * np;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_load_svd<<<blocks, 256, 0, s>>>(m, n, np, G, ldg, Gw, Vw, cnt);
    return cudaGetLastError();
}

// ======================================================================== off-norm
constexpr int RED_T = 256;

int reduce_blocks_for(int np)
{
    int g = np < 608 ? np : 608;  // 4 per SM at most
    return g < 1 ? 1 : g;
}

// Column j of the np x np matrix (leading dimension ld) is read by CTA
// j mod G, its rows strided over the CTA's threads; per-thread sums, a tree
// over the CTA, then one thread sums the CTA partials in index order.
template <typename TA>
__global__ void __launch_bounds__(RED_T) k_offnorm(int np, const TA* __restrict__ Aw, int ld,
                                                   double* partial, unsigned int* ticket,
                                                   double* result, int want_rel)
{
    __shared__ double s_off[RED_T], s_all[RED_T], s_rel[RED_T];
    __shared__ bool last;
    const int tid = threadIdx.x, G = gridDim.x;
    double off = 0.0, all = 0.0, rel = 0.0;
    for (int j = blockIdx.x; j < np; j += G) {
        const TA* col = Aw + (size_t)ld * j;
        const double ajj = fabs((double)col[j]);
        for (int i = tid; i < np; i += RED_T) {
            double v = (double)col[i];
            double v2 = v * v;
            all += v2;
            if (i != j) {
                off += v2;
                if (want_rel && v != 0.0) {
                    double d = fabs((double)Aw[(size_t)ld * i + i]) * ajj;
                    double r = d > 0.0 ? v2 / d : INFINITY;
                    rel = fmax(rel, r);
                }
            }
        }
    }
    s_off[tid] = off;
    s_all[tid] = all;
    s_rel[tid] = rel;
    __syncthreads();
    for (int w = RED_T / 2; w > 0; w >>= 1) {
        if (tid < w) {
            s_off[tid] += s_off[tid + w];
            s_all[tid] += s_all[tid + w];
            s_rel[tid] = fmax(s_rel[tid], s_rel[tid + w]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        partial[3 * blockIdx.x + 0] = s_off[0];
        partial[3 * blockIdx.x + 1] = s_all[0];
        partial[3 * blockIdx.x + 2] = s_rel[0];
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        last = (t == (unsigned int)G - 1);
    }
    __syncthreads();
    if (last && tid == 0) {
        __threadfence();
        double o = 0.0, a = 0.0, r = 0.0;
        for (int g = 0; g < G; ++g) {  // fixed order
            o += ((volatile double*)partial)[3 * g + 0];
            a += ((volatile double*)partial)[3 * g + 1];
            r = fmax(r, ((volatile double*)partial)[3 * g + 2]);
        }
        result[0] = o;
        result[1] = a;
        result[2] = sqrt(r);
        *ticket = 0u;
    }
}

cudaError_t launch_offnorm(int np, const double* Aw, double* partial, unsigned int* ticket,
                           double* result, bool want_rel, cudaStream_t s)
{
    return launch_offnorm_ld(np, Aw, np, partial, ticket, result, want_rel, s);
}

cudaError_t launch_offnorm_ld(int n, const double* A, int ld, double* partial, unsigned int* ticket,
                              double* result, bool want_rel, cudaStream_t s)
{
    k_offnorm<double><<<reduce_blocks_for(n), RED_T, 0, s>>>(n, A, ld, partial, ticket, result, want_rel);
    return cudaGetLastError();
}

cudaError_t launch_offnorm32(int np, const float* Aw, double* partial, unsigned int* ticket,
                             double* result, cudaStream_t s)
{
    k_offnorm<float><<<reduce_blocks_for(np), RED_T, 0, s>>>(np, Aw, np, partial, ticket, result, 0);
    return cudaGetLastError();
}

// ======================================================================== pivot
constexpr int PIV_T = 512;

__host__ __device__ static inline size_t tri_pad(int k) { return ((size_t)k * (k + 1) / 2 + 1) & ~(size_t)1; }

size_t pivot_gscratch_doubles(int k) { return k <= 128 ? 0 : tri_pad(k) + (size_t)k * k; }

static size_t pivot_smem_bytes(int k)
{
    const int half = k / 2, nq = half * (half - 1) / 2;
    size_t small = (size_t)4 * half * sizeof(double) + (size_t)k * sizeof(double) +
                   (size_t)3 * half * sizeof(int) + (size_t)nq * sizeof(unsigned) + 64;
    if (k <= 128) small += (tri_pad(k) + (size_t)k * k) * sizeof(double);
    return small;
}

template <bool V32> struct VType { using T = double; };
template <> struct VType<true> { using T = float; };

// V32: V accumulated in FP32 (in the first half of its k x k double region)
template <bool SMEM, bool V32>
__global__ void __launch_bounds__(PIV_T) k_pivot(PivotArgs a)
{
    using VT = typename VType<V32>::T;
    extern __shared__ __align__(16) double smem[];
    const int e = blockIdx.x, tid = threadIdx.x;
    const int k = a.k, b = a.b, half = k >> 1;
    int I, J;
    const bool frozen = entry(a.pairs, e, I, J);
    const size_t ntp = tri_pad(k);

    double *Ap, *tail;
    VT* V;
    if (SMEM) {
        Ap = smem;
        V = reinterpret_cast<VT*>(smem + ntp);
        tail = smem + ntp + (size_t)k * k;
    } else {
        Ap = a.gscratch + (size_t)e * (ntp + (size_t)k * k);
        V = reinterpret_cast<VT*>(Ap + ntp);
        tail = smem;
    }
    CoreSmem<double> cs;
    cs.tau = tail;
    cs.s = cs.tau + half;
    cs.t = cs.s + half;
    cs.apq = cs.t + half;
    cs.dlo = cs.apq + half;
    cs.p = (int*)(cs.dlo + k);
    cs.q = cs.p + half;
    cs.on = cs.q + half;
    unsigned* quad = (unsigned*)(cs.on + half);
    __shared__ int s_cnt;
    cs.cnt = &s_cnt;
    __shared__ double s_red[PIV_T / 32];
    __shared__ int s_dest[256];   // output slot of each eigenpair (k <= 256)
    __shared__ int s_pos[256];    // the pivot's non-padding positions, ascending

    // ---- pivot Ahat (lower triangle) and V = I
    if (a.gram == nullptr) {
        for (int idx = tid; idx < k * k; idx += PIV_T) {
            int ii = idx % k, jj = idx / k;
            if (ii >= jj) {
                const size_t g = pair_map(I, J, b, ii) + (size_t)a.ld * pair_map(I, J, b, jj);
                Ap[tri(ii) + jj] = a.Ain32 ? (double)a.Ain32[g] : a.Ain[g];
            }
        }
    } else {
        const double* g = a.gram + (size_t)e * a.npanels * k * k;
        for (int idx = tid; idx < k * k; idx += PIV_T) {
            int ii = idx % k, jj = idx / k;
            if (ii < jj) continue;
            double s = 0.0;
            for (int r = 0; r < a.npanels; ++r) s += g[(size_t)r * k * k + idx];  // fixed order
            Ap[tri(ii) + jj] = s;
        }
    }
    for (int idx = tid; idx < k * k; idx += PIV_T) V[idx] = (idx % k == idx / k) ? VT(1) : VT(0);
    for (int x = tid; x < k; x += PIV_T) cs.dlo[x] = 0.0;
    build_quad_table(quad, half);
    __syncthreads();

    // ---- one-sided stop statistic: max_{i != j} |a_ij| / sqrt(a_ii a_jj) before rotating
    if (a.relmax) {
        double mx = 0.0;
        if (!frozen)
        for (int idx = tid; idx < k * k; idx += PIV_T) {
            int ii = idx % k, jj = idx / k;
            if (ii <= jj) continue;
            double d = sqrt(Ap[tri(ii) + ii]) * sqrt(Ap[tri(jj) + jj]);
            if (d > 0.0) mx = fmax(mx, fabs(Ap[tri(ii) + jj]) / d);
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0) s_red[tid >> 5] = mx;
        __syncthreads();
        if (tid == 0) {
            double m = 0.0;
            for (int w = 0; w < PIV_T / 32; ++w) m = fmax(m, s_red[w]);
            a.relmax[e] = m;
        }
    }

    // ---- inner sweeps: round-robin over the k indices, k-1 rounds of k/2 rotations
    int sweeps = 0;
    const int total_rot =
        jacobi_solve<double, VT>(Ap, V, k, a.tol_rel, frozen ? 0 : a.max_sweeps, quad, cs, &sweeps);

    // ---- permutation Vhat <- Vhat P: eigenpair at position x moves to
    // s_dest[x]; with order == 1 the non-padding positions receive their
    // eigenvalues in descending order (ties by position); with order == 2 the
    // order QRCP picks on the leading rows of Vhat (Sec. 2.1); padding stays
    // put.
    __shared__ int s_nr, s_r1;
    if (tid == 0) {
        int nr = 0, r1 = 0;
        for (int x = 0; x < k; ++x)
            if (pair_map(I, J, b, x) < a.n_real) {
                r1 += x < b;
                s_pos[nr++] = x;
            }
        s_nr = nr;
        s_r1 = r1;
    }
    __syncthreads();
    if (a.order == 2 && total_rot > 0) {
        __shared__ int s_perm[256];
        __shared__ double s_cn[256], s_vh[128];
        const int nr = s_nr, r1 = s_r1;
        double* M = a.qrws + (size_t)e * b * k;
        for (int idx = tid; idx < r1 * nr; idx += PIV_T) {
            const int i = idx % r1, j = idx / r1;
            M[idx] = V[s_pos[i] + (size_t)k * s_pos[j]];
        }
        __syncthreads();
        qrcp_order(r1, nr, M, s_perm, s_cn, s_vh);
        for (int x = tid; x < k; x += PIV_T) s_dest[x] = x;
        __syncthreads();
        for (int t = tid; t < nr; t += PIV_T) s_dest[s_pos[s_perm[t]]] = s_pos[t];
        __syncthreads();
    } else {
    for (int x = tid; x < k; x += PIV_T) {
        int dest = x;
        if (a.order == 1 && total_rot > 0 && pair_map(I, J, b, x) < a.n_real) {
            const double dx = Ap[tri(x) + x];
            int r = 0;
            for (int y = 0; y < k; ++y) {
                if (y == x || pair_map(I, J, b, y) >= a.n_real) continue;
                const double dy = Ap[tri(y) + y];
                r += (dy > dx) || (dy == dx && y < x);
            }
            dest = s_pos[r];
        }
        s_dest[x] = dest;
    }
    __syncthreads();
    }

    // ---- outputs: V and V^T, D into the next A, counters
    double* Vo = a.V + (size_t)e * 2 * k * k;
    for (int idx = tid; idx < k * k; idx += PIV_T) {
        const int ii = idx % k, jj = idx / k;
        const double v = V[idx];                 // V(ii, jj) -> column s_dest[jj]
        Vo[ii + (size_t)k * s_dest[jj]] = v;
        Vo[(size_t)k * k + s_dest[jj] + (size_t)k * ii] = v;
    }
    if (a.Aout || a.Aout32) {
        for (int idx = tid; idx < k * k; idx += PIV_T) {
            const int ii = idx % k, jj = idx / k;
            const size_t g = pair_map(I, J, b, s_dest[ii]) + (size_t)a.ld * pair_map(I, J, b, s_dest[jj]);
            if (a.Aout32) a.Aout32[g] = (float)Ap[sidx(ii, jj)];
            else a.Aout[g] = Ap[sidx(ii, jj)];
        }
    }
    if (tid == 0) {
        a.rot[e] = total_rot;
        atomicAdd(&a.cnt->rotations, (unsigned long long)total_rot);
        atomicAdd(&a.cnt->inner_sweeps, (unsigned long long)sweeps);
        if (!frozen) atomicAdd(&a.cnt->pair_solves, 1ull);
        // per applied rotation: its row pair in k/2-1 quads (12 flops each, as
        // left and as right factor) and its column pair of V (6k flops, FP32
        // and not counted here when V is accumulated in FP32)
        atomicAdd(&a.cnt->flops_fp64, (unsigned long long)total_rot * (unsigned long long)((a.v32 ? 12 : 18) * k));
    }
}

cudaError_t launch_pivot(const PivotArgs& a, cudaStream_t s)
{
    if (a.npairs <= 0) return cudaSuccess;
    size_t smem = pivot_smem_bytes(a.k);
    void (*kern)(PivotArgs) = a.k <= 128 ? (a.v32 ? k_pivot<true, true> : k_pivot<true, false>)
                                         : (a.v32 ? k_pivot<false, true> : k_pivot<false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.npairs, PIV_T, smem, s>>>(a);
    return cudaGetLastError();
}

// ======================================================================== GEMM tiles
// C(M x 32) += Aop(M x K) Bop(K x 32) on 256 threads: thread (ty = tid % 32,
// tx = tid / 32) owns rows ty + 32 i (i < MR) and columns tx + 8 j (j < 4).
// K is streamed through shared memory in chunks of KC.
constexpr int UPD_T = 256, KC = 16, TN = 32, T_LD = TN + 1;

template <int MR>
struct Tile {
    double acc[MR][4];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    }
};

// As: [KC][AS_LD], Bs: [KC][T_LD] (or B directly from a shared buffer).
// fa(m, kk) loads Aop(m, kk); fb(kk, j) loads Bop(kk, j).  a_kfast / b_kfast
// choose which index runs fastest across threads while loading (coalescing).
template <int MR, bool A_KFAST, bool B_SMEM, bool B_KFAST, class FA, class FB>
__device__ __forceinline__ void gemm_tile(Tile<MR>& t, int M, int K, int mr, FA fa, FB fb,
                                          double* As, double* Bs, const double* Bsm)
{
    constexpr int AS_LD = 32 * MR + 1;
    const int tid = threadIdx.x, ty = tid & 31, tx = tid >> 5;
    for (int k0 = 0; k0 < K; k0 += KC) {
        const int kc = min(KC, K - k0);
        if (A_KFAST) {
            for (int idx = tid; idx < kc * M; idx += UPD_T) {
                const int m = idx / kc, kk = idx - m * kc;
                As[kk * AS_LD + m] = fa(m, k0 + kk);
            }
        } else {
            for (int idx = tid; idx < kc * M; idx += UPD_T) {
                const int kk = idx / M, m = idx - kk * M;
                As[kk * AS_LD + m] = fa(m, k0 + kk);
            }
        }
        if (!B_SMEM) {
            if (B_KFAST) {
                for (int idx = tid; idx < kc * TN; idx += UPD_T) {
                    const int j = idx / kc, kk = idx - j * kc;
                    Bs[kk * T_LD + j] = fb(k0 + kk, j);
                }
            } else {
                for (int idx = tid; idx < kc * TN; idx += UPD_T) {
                    const int kk = idx >> 5, j = idx & 31;
                    Bs[kk * T_LD + j] = fb(k0 + kk, j);
                }
            }
        }
        __syncthreads();
        const double* Bk = B_SMEM ? (Bsm + (size_t)k0 * T_LD) : Bs;
        for (int kk = 0; kk < kc; ++kk) {
            double bv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bk[kk * T_LD + tx + 8 * j];
#pragma unroll
            for (int i = 0; i < MR; ++i) {
                if (i < mr) {
                    const double av = As[kk * AS_LD + ty + 32 * i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) t.acc[i][j] = fma(av, bv[j], t.acc[i][j]);
                }
            }
        }
        __syncthreads();
    }
}

template <int MR>
static size_t update_smem_bytes()
{
    return ((size_t)KC * (32 * MR + 1) + (size_t)KC * T_LD + (size_t)(32 * MR) * T_LD) *
           sizeof(double);
}

// ======================================================================== EVD update
__device__ __forceinline__ void decode_pairblock(int pb, int& e1, int& e2)
{
    int t = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)pb)) * 0.5f);
    while (t * (t - 1) / 2 > pb) --t;
    while ((t + 1) * t / 2 <= pb) ++t;
    e2 = t;
    e1 = pb - t * (t - 1) / 2;
}

template <int MR>
__global__ void __launch_bounds__(UPD_T, 2) k_update_evd(UpdateArgs a, int n_sand, int nchunks)
{
    extern __shared__ __align__(16) double sm[];
    constexpr int AS_LD = 32 * MR + 1;
    double* As = sm;
    double* Bs = As + KC * AS_LD;
    double* Ts = Bs + KC * T_LD;  // [32*MR][T_LD]
    const int tid = threadIdx.x, ty = tid & 31, tx = tid >> 5;
    const int k = a.k, b = a.b;
    const int item = blockIdx.x;
    Tile<MR> t;

    if (item < n_sand) {
        // ---------------- A'_{P1P2} (:, chunk) = V1^T (A_{P1P2} V2(:, chunk))
        const int pbk = item / nchunks, c = item - pbk * nchunks;
        int e1, e2;
        decode_pairblock(pbk, e1, e2);
        int I1, J1, I2, J2;
        entry(a.pairs, e1, I1, J1);
        entry(a.pairs, e2, I2, J2);
        const int r1 = a.rot[e1], r2 = a.rot[e2];
        const int c0 = c * TN, kw = min(TN, k - c0);
        const int mr = (k + 31) >> 5;
        const double* Ain = a.Ain;
        const int lda = a.lda;
        const double* V2 = a.V + (size_t)e2 * 2 * k * k;          // V2, column-major
        const double* V1t = a.V + (size_t)e1 * 2 * k * k + (size_t)k * k;  // V1^T
        // stage 1: T = A_blk V2(:, chunk)  (or the plain chunk when V2 == I)
        if (r2) {
            t.zero();
            gemm_tile<MR, false, false, true>(
                t, k, k, mr,
                [&](int m, int kk) { return Ain[pair_map(I1, J1, b, m) + (size_t)lda * pair_map(I2, J2, b, kk)]; },
                [&](int kk, int j) { return j < kw ? V2[kk + (size_t)k * (c0 + j)] : 0.0; }, As, Bs,
                nullptr);
#pragma unroll
            for (int i = 0; i < MR; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i < mr) Ts[(ty + 32 * i) * T_LD + tx + 8 * j] = t.acc[i][j];
        } else {
            for (int idx = tid; idx < k * TN; idx += UPD_T) {
                const int j = idx / k, m = idx - j * k;
                Ts[m * T_LD + j] = j < kw ? Ain[pair_map(I1, J1, b, m) + (size_t)lda * pair_map(I2, J2, b, c0 + j)] : 0.0;
            }
        }
        __syncthreads();
        // stage 2: O = V1^T T
        if (r1) {
            t.zero();
            gemm_tile<MR, false, true, false>(
                t, k, k, mr, [&](int m, int kk) { return V1t[m + (size_t)k * kk]; },
                [&](int, int) { return 0.0; }, As, Bs, Ts);
#pragma unroll
            for (int i = 0; i < MR; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int m = ty + 32 * i, jj = tx + 8 * j;
                    if (i < mr && m < k && jj < kw) {
                        const int gi = pair_map(I1, J1, b, m), gj = pair_map(I2, J2, b, c0 + jj);
                        a.Aout[gi + (size_t)lda * gj] = t.acc[i][j];
                        a.Aout[gj + (size_t)lda * gi] = t.acc[i][j];
                    }
                }
        } else {
            for (int idx = tid; idx < k * TN; idx += UPD_T) {
                const int j = idx / k, m = idx - j * k;
                if (j < kw) {
                    const int gi = pair_map(I1, J1, b, m), gj = pair_map(I2, J2, b, c0 + j);
                    const double v = Ts[m * T_LD + j];
                    a.Aout[gi + (size_t)lda * gj] = v;
                    a.Aout[gj + (size_t)lda * gi] = v;
                }
            }
        }
        if (tid == 0) {
            const unsigned long long f = (unsigned long long)(r1 ? 2ull * k * k * kw : 0) +
                                         (unsigned long long)(r2 ? 2ull * k * k * kw : 0);
            atomicAdd(&a.cnt->flops_fp64, f);
            atomicAdd(&a.cnt->flops_update, f);
        }
    } else {
        // ---------------- Q'(rows, P chunk) = Q(rows, P) V_P(:, chunk)
        const int H = 32 * MR;
        const int nrt = (a.qrows + H - 1) / H;
        int rest = item - n_sand;
        const int c = rest % nchunks;
        rest /= nchunks;
        const int rt = rest % nrt, e = rest / nrt;
        int I, J;
        entry(a.pairs, e, I, J);
        const int r = a.rot[e];
        const int c0 = c * TN, kw = min(TN, k - c0), r0 = rt * H, M = min(H, a.qrows - r0);
        const int mr = (M + 31) >> 5;
        const double* Qin = a.Qin;
        const int ldq = a.ldq;
        const double* Vp = a.V + (size_t)e * 2 * k * k;
        if (r) {
            t.zero();
            gemm_tile<MR, false, false, true>(
                t, M, k, mr, [&](int m, int kk) { return Qin[(r0 + m) + (size_t)ldq * pair_map(I, J, b, kk)]; },
                [&](int kk, int j) { return j < kw ? Vp[kk + (size_t)k * (c0 + j)] : 0.0; }, As, Bs,
                nullptr);
#pragma unroll
            for (int i = 0; i < MR; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int m = ty + 32 * i, jj = tx + 8 * j;
                    if (i < mr && m < M && jj < kw)
                        a.Qout[(r0 + m) + (size_t)ldq * pair_map(I, J, b, c0 + jj)] = t.acc[i][j];
                }
            if (tid == 0) {
                atomicAdd(&a.cnt->flops_fp64, 2ull * M * k * kw);
                atomicAdd(&a.cnt->flops_update, 2ull * M * k * kw);
            }
        } else {
            for (int idx = tid; idx < M * kw; idx += UPD_T) {
                const int j = idx / M, m = idx - j * M;
                const size_t o = (r0 + m) + (size_t)ldq * pair_map(I, J, b, c0 + j);
                a.Qout[o] = Qin[o];
            }
        }
    }
}

template <int MR>
static cudaError_t launch_update_evd_mr(const UpdateArgs& a, cudaStream_t s)
{
    const int nchunks = (a.k + TN - 1) / TN;
    const int n_sand = a.npairs * (a.npairs - 1) / 2 * nchunks;
    const int H = 32 * MR;
    const int n_q = a.Qin ? a.npairs * ((a.qrows + H - 1) / H) * nchunks : 0;
    const int items = n_sand + n_q;
    if (items == 0) return cudaSuccess;
    const size_t smem = update_smem_bytes<MR>();
    cudaError_t e = cudaFuncSetAttribute(k_update_evd<MR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_update_evd<MR><<<items, UPD_T, smem, s>>>(a, n_sand, nchunks);
    return cudaGetLastError();
}

cudaError_t launch_update_evd(const UpdateArgs& a, cudaStream_t s)
{
    if (a.k <= 32) return launch_update_evd_mr<1>(a, s);
    if (a.k <= 64) return launch_update_evd_mr<2>(a, s);
    if (a.k <= 128) return launch_update_evd_mr<4>(a, s);
    return launch_update_evd_mr<8>(a, s);
}

// ======================================================================== one-sided column update
template <int MR>
__global__ void __launch_bounds__(UPD_T, 2) k_update_cols(ColUpdateArgs a, int n_g, int nchunks)
{
    extern __shared__ __align__(16) double sm[];
    constexpr int AS_LD = 32 * MR + 1;
    double* As = sm;
    double* Bs = As + KC * AS_LD;
    const int tid = threadIdx.x, ty = tid & 31, tx = tid >> 5;
    const int k = a.k, b = a.b, H = 32 * MR;
    int item = blockIdx.x;
    const double* Min;
    double* Mout;
    int ld, rows;
    if (item < n_g) {
        Min = a.Gin; Mout = a.Gout; ld = a.ldg; rows = a.m;
    } else {
        item -= n_g;
        Min = a.Vin; Mout = a.Vout; ld = a.ldv; rows = a.vrows;
    }
    const int nrt = (rows + H - 1) / H;
    const int c = item % nchunks;
    const int rest = item / nchunks;
    const int rt = rest % nrt, e = rest / nrt;
    int I, J;
    entry(a.pairs, e, I, J);
    const int r = a.rot[e];
    const int c0 = c * TN, kw = min(TN, k - c0), r0 = rt * H, M = min(H, rows - r0);
    const int mr = (M + 31) >> 5;
    const double* Vp = a.Vh + (size_t)e * 2 * k * k;
    if (r) {
        Tile<MR> t;
        t.zero();
        gemm_tile<MR, false, false, true>(
            t, M, k, mr, [&](int m, int kk) { return Min[(r0 + m) + (size_t)ld * pair_map(I, J, b, kk)]; },
            [&](int kk, int j) { return j < kw ? Vp[kk + (size_t)k * (c0 + j)] : 0.0; }, As, Bs, nullptr);
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int m = ty + 32 * i, jj = tx + 8 * j;
                if (i < mr && m < M && jj < kw)
                    Mout[(r0 + m) + (size_t)ld * pair_map(I, J, b, c0 + jj)] = t.acc[i][j];
            }
        if (tid == 0) {
            atomicAdd(&a.cnt->flops_fp64, 2ull * M * k * kw);
            atomicAdd(&a.cnt->flops_update, 2ull * M * k * kw);
        }
    } else {
        for (int idx = tid; idx < M * kw; idx += UPD_T) {
            const int j = idx / M, m = idx - j * M;
            const size_t o = (r0 + m) + (size_t)ld * pair_map(I, J, b, c0 + j);
            Mout[o] = Min[o];
        }
    }
}

template <int MR>
static cudaError_t launch_update_cols_mr(const ColUpdateArgs& a, cudaStream_t s)
{
    const int nchunks = (a.k + TN - 1) / TN, H = 32 * MR;
    const int n_g = a.npairs * ((a.m + H - 1) / H) * nchunks;
    const int n_v = a.Vin ? a.npairs * ((a.vrows + H - 1) / H) * nchunks : 0;
    if (n_g + n_v == 0) return cudaSuccess;
    const size_t smem = ((size_t)KC * (32 * MR + 1) + (size_t)KC * T_LD) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_update_cols<MR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_update_cols<MR><<<n_g + n_v, UPD_T, smem, s>>>(a, n_g, nchunks);
    return cudaGetLastError();
}

cudaError_t launch_update_cols(const ColUpdateArgs& a, cudaStream_t s)
{
    // tiles of 128 rows: the inner dimension is k, so a 128 x 32 tile costs 2*128*32*k
    return launch_update_cols_mr<4>(a, s);
}

// ======================================================================== Gram (split K over rows)
constexpr int GRAM_ROWS = 512;
int gram_panel_rows() { return GRAM_ROWS; }
int gram_panels_for(int m) { return (m + GRAM_ROWS - 1) / GRAM_ROWS; }

// Item (pair e, panel r, column chunk c): rows c0.. of the k x k Gram block
// (lower triangle only: rows >= c0), K = the panel's rows of G.
template <int MR>
__global__ void __launch_bounds__(UPD_T, 2) k_gram(const double* __restrict__ G, int ldg, int m,
                                                  const int2* __restrict__ pairs, int b, int k,
                                                  int npanels, int nchunks, double* __restrict__ part,
                                                  DevCounters* cnt)
{
    extern __shared__ __align__(16) double sm[];
    constexpr int AS_LD = 32 * MR + 1;
    double* As = sm;
    double* Bs = As + KC * AS_LD;
    const int tid = threadIdx.x, ty = tid & 31, tx = tid >> 5;
    const int item = blockIdx.x;
    const int c = item % nchunks;
    const int rest = item / nchunks;
    const int pr = rest % npanels, e = rest / npanels;
    int I, J;
    entry(pairs, e, I, J);
    const int c0 = c * TN, kw = min(TN, k - c0);
    const int row0 = c0;  // lower triangle: output rows >= first column of the chunk
    const int M = k - row0, mr = (M + 31) >> 5;
    const int g0 = pr * GRAM_ROWS, K = min(GRAM_ROWS, m - g0);
    Tile<MR> t;
    t.zero();
    gemm_tile<MR, true, false, true>(
        t, M, K, mr,
        [&](int mm, int kk) { return G[(g0 + kk) + (size_t)ldg * pair_map(I, J, b, row0 + mm)]; },
        [&](int kk, int j) { return j < kw ? G[(g0 + kk) + (size_t)ldg * pair_map(I, J, b, c0 + j)] : 0.0; },
        As, Bs, nullptr);
    double* out = part + ((size_t)e * npanels + pr) * k * k;
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int mm = ty + 32 * i, jj = tx + 8 * j;
            if (i < mr && mm < M && jj < kw) out[(row0 + mm) + (size_t)k * (c0 + jj)] = t.acc[i][j];
        }
    if (tid == 0) {
        atomicAdd(&cnt->flops_fp64, 2ull * M * K * kw);
        atomicAdd(&cnt->flops_update, 2ull * M * K * kw);
    }
}

cudaError_t launch_gram(const double* G, int ldg, int m, const int2* pairs, int npairs, int b,
                        int k, double* part, DevCounters* cnt, cudaStream_t s)
{
    const int nchunks = (k + TN - 1) / TN, npanels = gram_panels_for(m);
    const int items = npairs * npanels * nchunks;
    if (items == 0) return cudaSuccess;
#define JAC_GRAM(MR)                                                                               \
    do {                                                                                           \
        const size_t smem = ((size_t)KC * (32 * MR + 1) + (size_t)KC * T_LD) * sizeof(double);     \
        cudaError_t e = cudaFuncSetAttribute(k_gram<MR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                            \
        k_gram<MR><<<items, UPD_T, smem, s>>>(G, ldg, m, pairs, b, k, npanels, nchunks, part, cnt); \
    } while (0)
    if (k <= 32) JAC_GRAM(1);
    else if (k <= 64) JAC_GRAM(2);
    else if (k <= 128) JAC_GRAM(4);
    else JAC_GRAM(8);
#undef JAC_GRAM
    return cudaGetLastError();
}

// ======================================================================== general FP64 GEMM
// C (M x N) = alpha op(A) B + beta C, column-major; op(A) = A (M x K) or A^T
// (A stored K x M).  Tiles of 128 x 32 on 256 threads (the update kernels'
// register tiling).  With `lower`, tiles strictly above the diagonal are
// skipped (the caller mirrors a symmetric product afterwards).
template <bool TRANS>
__global__ void __launch_bounds__(UPD_T, 2) k_gemm64(int M, int N, int K, double alpha,
                                                     const double* __restrict__ A, int lda,
                                                     const double* __restrict__ B, int ldb, double beta,
                                                     double* __restrict__ C, int ldc, int lower)
{
    extern __shared__ __align__(16) double sm[];
    constexpr int MR = 4, AS_LD = 32 * MR + 1;
    double* As = sm;
    double* Bs = As + KC * AS_LD;
    const int tid = threadIdx.x, ty = tid & 31, tx = tid >> 5;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * TN;
    if (lower && n0 >= m0 + 128) return;
    const int Mt = min(128, M - m0), mr = (Mt + 31) >> 5;
    Tile<MR> t;
    t.zero();
    gemm_tile<MR, TRANS, false, true>(
        t, Mt, K, mr,
        [&](int m, int kk) { return TRANS ? A[kk + (size_t)lda * (m0 + m)] : A[(m0 + m) + (size_t)lda * kk]; },
        [&](int kk, int j) { return n0 + j < N ? B[kk + (size_t)ldb * (n0 + j)] : 0.0; }, As, Bs, nullptr);
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = ty + 32 * i, jj = tx + 8 * j;
            if (i < mr && m < Mt && n0 + jj < N) {
                double* c = C + (m0 + m) + (size_t)ldc * (n0 + jj);
                *c = beta == 0.0 ? alpha * t.acc[i][j] : fma(alpha, t.acc[i][j], beta * *c);
            }
        }
}

// C(i, j) <- C(j, i) for i < j (upper triangle from the lower), n x n.
__global__ void k_mirror_lower(int n, double* __restrict__ C, int ldc)
{
    __shared__ double t[32][33];
    const int bi = blockIdx.x, bj = blockIdx.y;  // tile rows bi, columns bj of the upper part
    if (bi > bj) return;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    // read the lower tile (rows bj*32.., cols bi*32..) coalesced, write it transposed
    for (int r = ty; r < 32; r += 8) {
        const int i = bj * 32 + tx, j = bi * 32 + r;
        t[r][tx] = (i < n && j < n) ? C[i + (size_t)ldc * j] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = bi * 32 + tx, j = bj * 32 + r;
        if (i < n && j < n && i < j) C[i + (size_t)ldc * j] = t[tx][r];
    }
}

cudaError_t launch_mirror_lower(int n, double* C, int ldc, cudaStream_t s)
{
    const int nb = (n + 31) / 32;
    k_mirror_lower<<<dim3(nb, nb), dim3(32, 8), 0, s>>>(n, C, ldc);
    return cudaGetLastError();
}

cudaError_t launch_gemm64(int M, int N, int K, double alpha, const double* A, int lda, int transA,
                          const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t s,
                          int lower)
{
    const size_t smem = ((size_t)KC * (32 * 4 + 1) + (size_t)KC * T_LD) * sizeof(double);
    dim3 grid((M + 127) / 128, (N + TN - 1) / TN);
    cudaError_t e;
    if (transA) {
        if ((e = cudaFuncSetAttribute(k_gemm64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
        k_gemm64<true><<<grid, UPD_T, smem, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower);
    } else {
        if ((e = cudaFuncSetAttribute(k_gemm64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
        k_gemm64<false><<<grid, UPD_T, smem, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower);
    }
    return cudaGetLastError();
}

// ======================================================================== finalisation
// Stable rank of key[i] among key[0..n): ascending (asc) or descending.
__global__ void k_rank(int n, const double* __restrict__ key, int stride, int asc,
                       int* __restrict__ rank)
{
    __shared__ double tile[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double ki = i < n ? key[(size_t)i * stride] : 0.0;
    int r = 0;
    for (int j0 = 0; j0 < n; j0 += 256) {
        const int j = j0 + threadIdx.x;
        tile[threadIdx.x] = j < n ? key[(size_t)j * stride] : 0.0;
        __syncthreads();
        const int lim = min(256, n - j0);
        for (int u = 0; u < lim; ++u) {
            const double kj = tile[u];
            const int jj = j0 + u;
            const bool before = asc ? (kj < ki || (kj == ki && jj < i)) : (kj > ki || (kj == ki && jj < i));
            r += before;
        }
        __syncthreads();
    }
    if (i < n) rank[i] = r;
}

__global__ void k_finalize_evd(int n, int np, const double* __restrict__ Aw,
                               const double* __restrict__ Qw, const int* __restrict__ rank,
                               double* __restrict__ w, double* __restrict__ Q, int ldq,
                               double* __restrict__ A, int lda)
{
    const long long total = (long long)n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % n), j = (int)(idx / n);
        if (Q) Q[i + (size_t)ldq * rank[j]] = Qw[i + (size_t)np * j];
        if (A) A[rank[i] + (size_t)lda * rank[j]] = Aw[i + (size_t)np * j];
        if (i == 0) w[rank[j]] = Aw[j + (size_t)np * j];
    }
}

cudaError_t launch_finalize_evd(int n, int np, const double* Aw, const double* Qw, double* w,
                                double* Q, int ldq, double* A, int lda, int* rank_ws,
                                cudaStream_t s)
{
    k_rank<<<(n + 255) / 256, 256, 0, s>>>(n, Aw, np + 1, 1, rank_ws);
    long long total = (long long)n * n;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_finalize_evd<<<blocks, 256, 0, s>>>(n, np, Aw, Qw, rank_ws, w, Q, ldq, A, lda);
    return cudaGetLastError();
}

__global__ void k_colnorm(int m, const double* __restrict__ Gw, int ld, double* __restrict__ norms)
{
    __shared__ double red[256];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int r = threadIdx.x; r < m; r += 256) {
        const double v = Gw[r + (size_t)ld * j];
        s = fma(v, v, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) norms[j] = sqrt(red[0]);
}

__global__ void k_finalize_svd(int m, int n, const double* __restrict__ Gw, int ldgw,
                               const double* __restrict__ Vw, int ldvw,
                               const double* __restrict__ norms, const int* __restrict__ rank,
                               double* __restrict__ U, int ldu, double* __restrict__ sigma,
                               double* __restrict__ V, int ldv)
{
    const long long totu = (long long)m * n, totv = V ? (long long)n * n : 0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < totu + totv;
         idx += (long long)gridDim.x * blockDim.x) {
        if (idx < totu) {
            const int r = (int)(idx % m), j = (int)(idx / m);
            const double nj = norms[j];
            U[r + (size_t)ldu * rank[j]] = nj > 0.0 ? Gw[r + (size_t)ldgw * j] / nj : 0.0;
            if (r == 0) sigma[rank[j]] = nj;
        } else {
            const long long t = idx - totu;
            const int r = (int)(t % n), j = (int)(t / n);
            V[r + (size_t)ldv * rank[j]] = Vw[r + (size_t)ldvw * j];
        }
    }
}

cudaError_t launch_finalize_svd(int m, int n, const double* Gw, int ldgw, const double* Vw,
                                int ldvw, double* U, int ldu, double* sigma, double* V, int ldv,
                                double* norms_ws, int* rank_ws, cudaStream_t s)
{
    k_colnorm<<<n, 256, 0, s>>>(m, Gw, ldgw, norms_ws);
    k_rank<<<(n + 255) / 256, 256, 0, s>>>(n, norms_ws, 1, 0, rank_ws);
    long long total = (long long)m * n + (V ? (long long)n * n : 0);
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_finalize_svd<<<blocks, 256, 0, s>>>(m, n, Gw, ldgw, Vw, ldvw, norms_ws, rank_ws, U, ldu,
                                          sigma, V, ldv);
    return cudaGetLastError();
}

__global__ void k_max_into(const double* __restrict__ v, int n, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double m = *out;
        for (int i = 0; i < n; ++i) m = fmax(m, v[i]);
        *out = m;
    }
}

cudaError_t launch_max_into(const double* relmax, int npairs, double* out, cudaStream_t s)
{
    k_max_into<<<1, 32, 0, s>>>(relmax, npairs, out);
    return cudaGetLastError();
}

// ======================================================================== rotation diagnostic
__global__ void k_rotation_params(int count, const double* __restrict__ app, const double* __restrict__ aqq,
                                  const double* __restrict__ apq, double tol, double* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double p = app[i], q = aqq[i], x = apq[i];
    double* o = out + (size_t)8 * i;
    double s = 0.0, t = 0.0, tau = 0.0;
    const bool on = rotation_wanted(p, q, x, tol);
    if (x != 0.0) schur2(p, q, x, s, t, tau);
    o[0] = t;
    o[1] = s;
    o[2] = tau;
    o[3] = on ? 1.0 : 0.0;
    s = t = tau = 0.0;
    const bool on_ref = x != 0.0 && fabs(x) > rn_mul(rn_mul(tol, rn_sqrt(fabs(p))), rn_sqrt(fabs(q)));
    if (x != 0.0) schur2_ref(p, q, x, s, t, tau);
    o[4] = t;
    o[5] = s;
    o[6] = tau;
    o[7] = on_ref ? 1.0 : 0.0;
}

cudaError_t launch_rotation_params(int count, const double* app, const double* aqq, const double* apq, double tol,
                                   double* out, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_rotation_params<<<(count + 255) / 256, 256, 0, s>>>(count, app, aqq, apq, tol, out);
    return cudaGetLastError();
}

}  // namespace jac
