// k_batched_blocked.cu -- the batched EVD for matrices above the
// shared-memory size, by the blocked method itself: one CTA per matrix
// (persistent, longest first from a queue), block size 16 (2b = 32), the
// round-robin schedule of Algorithm 2, one inner sweep per pivot solve, and
// the symmetric pair-block updates of the single-matrix path.
//
// Per step of a sweep, inside the CTA:
//   1. pivot solves, one warp per pair: the 32 x 32 pivot (lower triangle in
//      shared memory) is swept once by the scalar parallel-ordered Jacobi of
//      the pivot kernels (round-robin over its 32 indices, rotations in
//      Rutishauser's form, diagonal carried as hi + lo), its eigenpairs
//      sorted by descending eigenvalue over the non-padding positions, D
//      written back into the working A and V kept in shared memory;
//   2. updates, one warp per item: A'_{P1P2} = V1^T A_{P1P2} V2 for every
//      pair-block whose pivots rotated (written with its mirror, in place:
//      every item owns its blocks), and Q'(rows, P) = Q(rows, P) V_P in
//      32-row chunks.
// A sweep in which no pivot rotates ends the solve (every index pair meets in
// some pivot of a sweep, so this is the scalar method's stop test).  The
// working A and Q (np x np, np = the order rounded up to a multiple of 32,
// zero padding that is never rotated) live in a per-CTA slot of global
// memory; the blocks a warp works on are staged through shared memory.
#include <cuda_runtime.h>

#include "batched.h"
#include "cluster_common.cuh"
#include "jacobi_core.cuh"

namespace jac {

namespace {

constexpr int BB = 16;            // block size
constexpr int BK = 32;            // pivot order 2b
constexpr int BLD = 33;           // padded leading dimension of 32 x 32 tiles in shared memory
constexpr int BMAXP = kBatchedMaxK / BK;   // pairs per step at most (16)

// Leading dimension of the staging tiles and of the kept V's: FP32 uses 36
// (16-byte rows for the vectorised, register-blocked 32 x 32 products), FP64
// 33 (conflict-free scalar access).
template <typename T>
constexpr int sld() { return sizeof(T) == 4 ? 36 : BLD; }

template <typename T>
struct BlkWarp {                  // per-warp scratch
    alignas(16) T tile[BK * sld<T>()];   // pivot (lower triangle, ld BLD) / staging of a 32 x 32 block
    T dlo[BK];
    T rs[BK / 2], rtau[BK / 2], rt[BK / 2], rapq[BK / 2];
    int rp[BK / 2], rq[BK / 2], ron[BK / 2];
    int dest[BK];
};

template <typename T>
constexpr int blk_threads() { return sizeof(T) == 4 ? 512 : 256; }

// FP32: acc(i, j) += sum_k A(8 ty + i, k) B(k, 4 tx + j), ty = lane / 8,
// tx = lane % 8, for 32 x 32 x 32 operands in shared memory: A column-major
// (A(m, k) at A[m + 36 k]), B row-major (B(k, n) at B[n + 36 k]); two 16-byte
// loads of A and one of B feed 32 FMAs.
__device__ __forceinline__ void mm32(const float* A, const float* B, float (&acc)[8][4], int lane)
{
    const int ty = lane >> 3, tx = lane & 7;
#pragma unroll 4
    for (int k = 0; k < BK; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(A + 8 * ty + 36 * k);
        const float4 a1 = *reinterpret_cast<const float4*>(A + 8 * ty + 4 + 36 * k);
        const float4 b = *reinterpret_cast<const float4*>(B + 4 * tx + 36 * k);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
}

__device__ __forceinline__ int bmap(int I, int J, int x) { return x < BB ? I * BB + x : J * BB + (x - BB); }

// round-robin pair of position e in step s of N blocks (N even)
__device__ __forceinline__ void rr_pair(int N, int s, int e, int& I, int& J)
{
    const int x = e == 0 ? 0 : 1 + (e - 1 + s) % (N - 1);
    const int y = 1 + (N - 1 - e - 1 + s) % (N - 1);
    I = x < y ? x : y;
    J = x < y ? y : x;
}

// One inner sweep of the 32 x 32 pivot in w.tile (lower triangle, ld BLD)
// by one warp; V (ld BLD) accumulates.  Returns the rotations applied.
template <typename T>
__device__ int warp_pivot(BlkWarp<T>& w, T* V, T tol, int lane)
{
    T* P = w.tile;
    int total = 0;
    for (int r = 0; r < BK - 1; ++r) {
        if (lane < BK / 2) {
            const int pa = lane, pb = BK - 1 - lane;
            const int ia = pa == 0 ? 0 : 1 + (pa - 1 + r) % (BK - 1);
            const int ib = 1 + (pb - 1 + r) % (BK - 1);
            const int p = ia < ib ? ia : ib, q = ia < ib ? ib : ia;
            const T app = P[p * BLD + p], aqq = P[q * BLD + q], apq = P[q * BLD + p];
            const bool on = rotation_wanted(app, aqq, apq, tol);
            w.rp[lane] = p;
            w.rq[lane] = q;
            w.ron[lane] = on;
            if (on) {
                T s, t, tau;
                schur2(app, aqq, apq, s, t, tau);
                w.rs[lane] = s;
                w.rt[lane] = t;
                w.rtau[lane] = tau;
                w.rapq[lane] = apq;
            }
        }
        __syncwarp();
        const unsigned on_mask = __ballot_sync(0xffffffffu, lane < BK / 2 && w.ron[lane]);
        total += __popc(on_mask);
        if (on_mask) {
            // quads (e1 < e2): 120 of them, about 4 per lane
            for (int qi = lane; qi < (BK / 2) * (BK / 2 - 1) / 2; qi += 32) {
                int e1, e2;
                quad_decode(qi, e1, e2);
                const int on1 = w.ron[e1], on2 = w.ron[e2];
                if (!(on1 | on2)) continue;
                const int p1 = w.rp[e1], q1 = w.rq[e1], p2 = w.rp[e2], q2 = w.rq[e2];
                auto at = [&](int i, int j) -> T& { return i >= j ? P[i * BLD + j] : P[j * BLD + i]; };
                T x00 = at(p1, p2), x01 = at(p1, q2), x10 = at(q1, p2), x11 = at(q1, q2);
                if (on1) {
                    rot2(w.rs[e1], w.rtau[e1], x00, x10);
                    rot2(w.rs[e1], w.rtau[e1], x01, x11);
                }
                if (on2) {
                    rot2(w.rs[e2], w.rtau[e2], x00, x01);
                    rot2(w.rs[e2], w.rtau[e2], x10, x11);
                }
                at(p1, p2) = x00;
                at(p1, q2) = x01;
                at(q1, p2) = x10;
                at(q1, q2) = x11;
            }
            // the rotations' own 2 x 2 blocks: exact diagonal, zeroed a_pq
            if (lane < BK / 2 && w.ron[lane]) {
                const int p = w.rp[lane], q = w.rq[lane];
                T hp = P[p * BLD + p], hq = P[q * BLD + q];
                dd_add_prod(hp, w.dlo[p], w.rt[lane], w.rapq[lane], T(-1));
                dd_add_prod(hq, w.dlo[q], w.rt[lane], w.rapq[lane], T(1));
                P[p * BLD + p] = hp;
                P[q * BLD + q] = hq;
                P[q * BLD + p] = T(0);
            }
            // V <- V J: lane = row
            for (int e = 0; e < BK / 2; ++e) {
                if (!((on_mask >> e) & 1u)) continue;
                const int p = w.rp[e], q = w.rq[e];
                T vp = V[lane + BLD * p], vq = V[lane + BLD * q];
                rot2(w.rs[e], w.rtau[e], vp, vq);
                V[lane + BLD * p] = vp;
                V[lane + BLD * q] = vq;
            }
        }
        __syncwarp();
    }
    return total;
}

template <typename T>
__global__ void __launch_bounds__(blk_threads<T>()) k_batched_evd_blocked(BatchedEvdArgs<T> a, const int* list,
                                                                        int count, unsigned* queue, T* slots,
                                                                        size_t slot_elems)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    constexpr int VLD = sld<T>();
    T* Vs = (T*)bsm;                                          // [BMAXP][BK * VLD] pivot V's of the step
    BlkWarp<T>* warps = (BlkWarp<T>*)(Vs + (size_t)BMAXP * BK * VLD);
    __shared__ int s_item, s_rot, s_prot[BMAXP];
    __shared__ unsigned long long s_flops;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    BlkWarp<T>& w = warps[wid];
    T* Aw = slots + (size_t)blockIdx.x * slot_elems;

    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= count) break;
        const int mat = list[item];
        const int n = a.n[mat];
        const int np = (n + BK - 1) / BK * BK, N = np / BB, npairs = N / 2;
        T* Qw = Aw + (size_t)np * np;
        const bool vec = a.Q != nullptr;
        const T* A = a.A[mat];
        const size_t lda = (size_t)a.lda[mat];
        // ---- load: mirrored lower triangle, zero padding; Q = I
        int bad = 0;
        for (size_t idx = tid; idx < (size_t)np * np; idx += blockDim.x) {
            const int i = (int)(idx % np), j = (int)(idx / np);
            T v = T(0);
            if (i < n && j < n) {
                v = i >= j ? A[i + lda * j] : A[j + lda * i];
                if (!isfinite(v)) bad = 1;
            }
            Aw[idx] = v;
            if (vec) Qw[idx] = i == j ? T(1) : T(0);
        }
        if (tid == 0) {
            s_rot = 0;
            s_flops = 0;
        }
        bad = __syncthreads_or(bad);
        int sweeps = 0, last = 1;
        const int max_sweeps = bad ? 0 : a.max_sweeps;
        for (int sw = 0; sw < max_sweeps; ++sw) {
            for (int s = 0; s < N - 1; ++s) {
                // ---- 1. pivot solves, one warp per pair
                for (int e = wid; e < npairs; e += nw) {
                    int I, J;
                    rr_pair(N, s, e, I, J);
                    T* V = Vs + (size_t)e * BK * VLD;   // accumulated column-major, ld BLD
                    for (int c = 0; c < BK; ++c) {
                        // lane = row: the lower triangle of the pivot, and V = I
                        if (lane >= c) w.tile[lane * BLD + c] = Aw[bmap(I, J, lane) + (size_t)np * bmap(I, J, c)];
                        V[lane + BLD * c] = lane == c ? T(1) : T(0);
                    }
                    w.dlo[lane] = T(0);
                    __syncwarp();
                    const int rot = warp_pivot(w, V, a.tol, lane);
                    // eigenpairs by descending eigenvalue over the real positions
                    const T dx = w.tile[lane * BLD + lane] + w.dlo[lane];
                    w.tile[lane * BLD + lane] = dx;
                    __syncwarp();
                    const bool real = bmap(I, J, lane) < n;
                    const unsigned realm = __ballot_sync(0xffffffffu, real);
                    int dest = lane;
                    if (rot > 0 && real) {
                        int rk = 0;
                        for (int y = 0; y < BK; ++y) {
                            if (y == lane || !((realm >> y) & 1u)) continue;
                            const T dy = w.tile[y * BLD + y];
                            rk += (dy > dx) || (dy == dx && y < lane);
                        }
                        // the rk-th real position
                        unsigned m = realm;
                        for (int t = 0; t < rk; ++t) m &= m - 1;
                        dest = __ffs(m) - 1;
                    }
                    w.dest[lane] = dest;
                    __syncwarp();
                    // D into the working A (full 32 x 32 block), V permuted in place
                    for (int c = 0; c < BK; ++c) {
                        const int i = lane, j = c;
                        const T v = i >= j ? w.tile[i * BLD + j] : w.tile[j * BLD + i];
                        Aw[bmap(I, J, w.dest[i]) + (size_t)np * bmap(I, J, w.dest[j])] = v;
                    }
                    if (rot > 0) {
                        // V <- V P; FP32 keeps it row-major (ld 36) for the products
                        T col[BK];
#pragma unroll
                        for (int c = 0; c < BK; ++c) col[c] = V[lane + BLD * c];
                        __syncwarp();
                        if constexpr (sizeof(T) == 4) {
#pragma unroll
                            for (int c = 0; c < BK; ++c) V[w.dest[c] + VLD * lane] = col[c];
                        } else {
#pragma unroll
                            for (int c = 0; c < BK; ++c) V[lane + BLD * w.dest[c]] = col[c];
                        }
                    }
                    if (lane == 0) {
                        s_prot[e] = rot;
                        if (rot) {
                            atomicAdd(&s_rot, rot);
                            // per applied rotation: its quads in the pivot (both sides) and a V column pair
                            atomicAdd(&s_flops, (unsigned long long)rot * 12ull * BK);
                        }
                    }
                    __syncwarp();
                }
                __syncthreads();
                // ---- 2. updates, one warp per item
                const int npb = npairs * (npairs - 1) / 2;
                const int nq = vec ? npairs * (np / BK) : 0;
                for (int it = wid; it < npb + nq; it += nw) {
                    T* S = w.tile;
                    if (it < npb) {
                        int e1, e2;
                        quad_decode(it, e1, e2);
                        const int r1 = s_prot[e1], r2 = s_prot[e2];
                        if (!(r1 | r2)) continue;            // V1 = V2 = I: unchanged
                        int I1, J1, I2, J2;
                        rr_pair(N, s, e1, I1, J1);
                        rr_pair(N, s, e2, I2, J2);
                        const T* V1 = Vs + (size_t)e1 * BK * VLD;
                        const T* V2 = Vs + (size_t)e2 * BK * VLD;
                        const size_t row = bmap(I1, J1, lane);
                        for (int c = 0; c < BK; ++c) S[lane + VLD * c] = Aw[row + (size_t)np * bmap(I2, J2, c)];
                        __syncwarp();
                        if constexpr (sizeof(T) == 4) {
                            const int ty = lane >> 3, tx = lane & 7;
                            float acc[8][4];
#pragma unroll
                            for (int i = 0; i < 8; ++i)
#pragma unroll
                                for (int j = 0; j < 4; ++j) acc[i][j] = r2 ? 0.f : S[(8 * ty + i) + VLD * (4 * tx + j)];
                            if (r2) mm32(S, V2, acc, lane);                    // T = A_blk V2
                            __syncwarp();
                            if (r1) {
                                // T row-major into S, then O = V1^T T (V1 row-major = V1^T column-major)
#pragma unroll
                                for (int i = 0; i < 8; ++i)
                                    *reinterpret_cast<float4*>(S + 4 * tx + VLD * (8 * ty + i)) =
                                        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                                __syncwarp();
#pragma unroll
                                for (int i = 0; i < 8; ++i)
#pragma unroll
                                    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
                                mm32(V1, S, acc, lane);
                                __syncwarp();
                            }
                            // O column-major (ld BLD) for the coalesced write-back
#pragma unroll
                            for (int i = 0; i < 8; ++i)
#pragma unroll
                                for (int j = 0; j < 4; ++j) S[(8 * ty + i) + BLD * (4 * tx + j)] = acc[i][j];
                            __syncwarp();
                        } else {
                            // lane j: T(:, j) = A_blk V2(:, j), then O(:, j) = V1^T T(:, j)
                            T t[BK];
#pragma unroll
                            for (int l = 0; l < BK; ++l) t[l] = T(0);
                            if (r2) {
                                for (int c = 0; c < BK; ++c) {
                                    const T v = V2[c + BLD * lane];
#pragma unroll
                                    for (int l = 0; l < BK; ++l) t[l] = fma(S[l + BLD * c], v, t[l]);
                                }
                            } else {
#pragma unroll
                                for (int l = 0; l < BK; ++l) t[l] = S[l + BLD * lane];
                            }
                            __syncwarp();
                            if (r1) {
                                for (int i = 0; i < BK; ++i) {
                                    T o = T(0);
#pragma unroll
                                    for (int l = 0; l < BK; ++l) o = fma(V1[l + BLD * i], t[l], o);
                                    S[i + BLD * lane] = o;
                                }
                            } else {
#pragma unroll
                                for (int i = 0; i < BK; ++i) S[i + BLD * lane] = t[i];
                            }
                            __syncwarp();
                        }
                        // O(lane, c) to (P1 row lane, P2 column c); the mirror
                        // O(r, lane) to (P2 row lane, P1 column r)
                        for (int c = 0; c < BK; ++c) Aw[row + (size_t)np * bmap(I2, J2, c)] = S[lane + BLD * c];
                        for (int r = 0; r < BK; ++r) Aw[bmap(I2, J2, lane) + (size_t)np * bmap(I1, J1, r)] = S[r + BLD * lane];
                        if (lane == 0) atomicAdd(&s_flops, (unsigned long long)((r1 ? 2 : 0) + (r2 ? 2 : 0)) * BK * BK * BK);
                        __syncwarp();
                    } else {
                        const int qi = it - npb, e = qi / (np / BK), r0 = (qi % (np / BK)) * BK;
                        if (!s_prot[e]) continue;                  // V = I
                        int I, J;
                        rr_pair(N, s, e, I, J);
                        const T* V = Vs + (size_t)e * BK * VLD;
                        for (int c = 0; c < BK; ++c) S[lane + VLD * c] = Qw[(r0 + lane) + (size_t)np * bmap(I, J, c)];
                        __syncwarp();
                        if constexpr (sizeof(T) == 4) {
                            const int ty = lane >> 3, tx = lane & 7;
                            float acc[8][4];
#pragma unroll
                            for (int i = 0; i < 8; ++i)
#pragma unroll
                                for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
                            mm32(S, V, acc, lane);
                            __syncwarp();
#pragma unroll
                            for (int i = 0; i < 8; ++i)
#pragma unroll
                                for (int j = 0; j < 4; ++j) S[(8 * ty + i) + BLD * (4 * tx + j)] = acc[i][j];
                        } else {
                            T o[BK];
#pragma unroll
                            for (int r = 0; r < BK; ++r) o[r] = T(0);
                            for (int c = 0; c < BK; ++c) {
                                const T v = V[c + BLD * lane];
#pragma unroll
                                for (int r = 0; r < BK; ++r) o[r] = fma(S[r + BLD * c], v, o[r]);
                            }
                            __syncwarp();
#pragma unroll
                            for (int r = 0; r < BK; ++r) S[r + BLD * lane] = o[r];
                        }
                        __syncwarp();
                        for (int c = 0; c < BK; ++c) Qw[(r0 + lane) + (size_t)np * bmap(I, J, c)] = S[lane + BLD * c];
                        if (lane == 0) atomicAdd(&s_flops, 2ull * BK * BK * BK);
                        __syncwarp();
                    }
                }
                __syncthreads();
            }
            sweeps = sw + 1;
            last = s_rot;
            __syncthreads();
            if (tid == 0) s_rot = 0;
            __syncthreads();
            if (last == 0) break;
        }
        // ---- eigenvalues ascending (stable), Q's columns with them
        int* rank = (int*)Vs;   // the step's V's are no longer needed
        T* wout = a.w[mat];
        for (int x = tid; x < n; x += blockDim.x) {
            const T dx = Aw[x + (size_t)np * x];
            int r = 0;
            for (int y = 0; y < n; ++y) {
                const T dy = Aw[y + (size_t)np * y];
                r += (dy < dx) || (dy == dx && y < x);
            }
            wout[r] = dx;
            rank[x] = r;
        }
        __syncthreads();
        if (vec) {
            T* Q = a.Q[mat];
            const size_t ldq = (size_t)a.ldq[mat];
            for (size_t idx = tid; idx < (size_t)n * n; idx += blockDim.x) {
                const int i = (int)(idx % n), j = (int)(idx / n);
                Q[i + ldq * rank[j]] = Qw[i + (size_t)np * j];
            }
        }
        if (tid == 0) {
            const bool converged = !bad && last == 0;
            a.info[mat] = bad ? -100 : (converged ? 0 : sweeps);
            atomicAdd(&a.cnt->inner_sweeps, (unsigned long long)sweeps);
            atomicAdd(&a.cnt->pair_solves, 1ull);
            if (sizeof(T) == 8) atomicAdd(&a.cnt->flops_fp64, s_flops);
            else atomicAdd(&a.cnt->flops_fp32, s_flops);
        }
        __syncthreads();
    }
}

}  // namespace

template <typename T>
size_t batched_blocked_smem()
{
    return (size_t)BMAXP * BK * sld<T>() * sizeof(T) + (size_t)(blk_threads<T>() / 32) * sizeof(BlkWarp<T>);
}

template <typename T>
int batched_blocked_ctas_per_sm()
{
    const size_t smem = batched_blocked_smem<T>();
    if (cudaFuncSetAttribute(k_batched_evd_blocked<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched_evd_blocked<T>, blk_threads<T>(), smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

template <typename T>
size_t batched_blocked_slot_elems(int nmax)
{
    const size_t np = (size_t)(nmax + BK - 1) / BK * BK;
    return 2 * np * np;
}

template <typename T>
cudaError_t launch_batched_evd_blocked(const BatchedEvdArgs<T>& a, const int* list, int count, unsigned* queue,
                                       T* slots, size_t slot_elems, int grid, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = batched_blocked_smem<T>();
    cudaError_t e = cudaFuncSetAttribute(k_batched_evd_blocked<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(queue, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    k_batched_evd_blocked<T><<<grid, blk_threads<T>(), smem, s>>>(a, list, count, queue, slots, slot_elems);
    return cudaGetLastError();
}

template size_t batched_blocked_smem<float>();
template size_t batched_blocked_smem<double>();
template int batched_blocked_ctas_per_sm<float>();
template int batched_blocked_ctas_per_sm<double>();
template size_t batched_blocked_slot_elems<float>(int);
template size_t batched_blocked_slot_elems<double>(int);
template cudaError_t launch_batched_evd_blocked<float>(const BatchedEvdArgs<float>&, const int*, int, unsigned*, float*,
                                                       size_t, int, cudaStream_t);
template cudaError_t launch_batched_evd_blocked<double>(const BatchedEvdArgs<double>&, const int*, int, unsigned*,
                                                        double*, size_t, int, cudaStream_t);

}  // namespace jac
