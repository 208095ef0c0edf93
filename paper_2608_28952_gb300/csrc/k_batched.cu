// k_batched.cu -- batched forms: thousands of independent small matrices in
// one persistent launch.
//
// k_batched_evd<T>: a persistent grid pops matrices from an atomic queue in
// longest-first order (sizes sorted descending on the host, so the long
// solves start first and the short ones fill the tail).  One CTA solves one
// matrix with the scalar parallel-ordered Jacobi of jacobi_core.cuh (the
// blocked method with a single pair, 2b = n): the packed matrix and its V
// live in shared memory when they fit, else in the CTA's slot of a global
// scratch area (L2-resident for the matrix being solved).  Eigenvalues are
// sorted ascending with Q's columns.
//
// k_batched_svd<T>: one-sided Jacobi (Algorithm 6) with one column-block pair
// covering all n columns: each sweep forms the n x n Gram block from G,
// solves it with the same core, sorts its eigenpairs descending and rotates
// G's columns (G <- G Vhat) and the accumulated V.  Stops when the Gram's
// largest normalised off-diagonal is <= tol_eff or no rotation is applied;
// finalises sigma = column norms, U = G Sigma^+.
#include <cuda_runtime.h>

#include "batched.h"
#include "batched_svd.h"
#include "jacobi_core.cuh"

namespace jac {

__host__ __device__ size_t batched_tri_pad(int k) { return ((size_t)k * (k + 1) / 2 + 1) & ~(size_t)1; }

template <typename T>
__host__ __device__ static size_t core_bytes(int kmax)
{
    const int half = kmax / 2;
    return (size_t)4 * half * sizeof(T) + (size_t)kmax * sizeof(T) + (size_t)3 * half * sizeof(int) + 64;
}

template <typename T>
__device__ __forceinline__ CoreSmem<T> carve_core(unsigned char* base, int kmax)
{
    const int half = kmax / 2;
    CoreSmem<T> cs;
    cs.tau = (T*)base;
    cs.s = cs.tau + half;
    cs.t = cs.s + half;
    cs.apq = cs.t + half;
    cs.dlo = cs.apq + half;
    cs.p = (int*)(cs.dlo + kmax);
    cs.q = cs.p + half;
    cs.on = cs.q + half;
    return cs;
}

// ================================================================ EVD
template <typename T>
__global__ void k_batched_evd(BatchedEvdArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ int s_item, s_cnt, s_bad;
    __shared__ int s_dest[kBatchedMaxK];
    CoreSmem<T> cs = carve_core<T>(bsm, kBatchedMaxK);
    cs.cnt = &s_cnt;
    T* smat = (T*)(bsm + core_bytes<T>(kBatchedMaxK));
    const int tid = threadIdx.x, nt = blockDim.x;

    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= a.batch) break;
        const int mat = a.order[item];
        const int n = a.n[mat], k = n + (n & 1);
        const bool vec = a.Q != nullptr;
        const size_t ntp = batched_tri_pad(k);
        T* Ap;
        if (k <= a.smem_kmax) {
            Ap = smat;
        } else {
            Ap = a.gscratch + (size_t)blockIdx.x * a.slot_elems;
        }
        T* V = vec ? Ap + ntp : nullptr;
        const T* A = a.A[mat];
        const int lda = a.lda[mat];
        if (tid == 0) s_bad = 0;
        __syncthreads();
        int bad = 0;
        for (int idx = tid; idx < k * k; idx += nt) {
            const int ii = idx % k, jj = idx / k;
            if (ii >= jj) {
                T v = T(0);
                if (ii < n) {
                    v = A[ii + (size_t)lda * jj];
                    if (!isfinite(v)) bad = 1;
                }
                Ap[tri(ii) + jj] = v;
            }
            if (V) V[idx] = (ii == jj) ? T(1) : T(0);
        }
        for (int x = tid; x < k; x += nt) cs.dlo[x] = T(0);
        if (bad) atomicExch(&s_bad, 1);
        __syncthreads();
        const bool nonfinite = s_bad != 0;
        int sweeps = 0, rot = 0;
        if (!nonfinite) rot = jacobi_solve<T>(Ap, V, k, a.tol, a.max_sweeps, a.qtab, cs, &sweeps);
        const bool converged = !nonfinite && s_cnt == 0;
        // ascending, stable rank among the n real positions (position n is padding)
        for (int x = tid; x < n; x += nt) {
            const T dx = Ap[tri(x) + x];
            int r = 0;
            for (int y = 0; y < n; ++y) {
                const T dy = Ap[tri(y) + y];
                r += (dy < dx) || (dy == dx && y < x);
            }
            s_dest[x] = r;
        }
        __syncthreads();
        T* w = a.w[mat];
        for (int x = tid; x < n; x += nt) w[s_dest[x]] = Ap[tri(x) + x];
        if (vec) {
            T* Q = a.Q[mat];
            const int ldq = a.ldq[mat];
            for (int idx = tid; idx < n * n; idx += nt) {
                const int i = idx % n, j = idx / n;
                Q[i + (size_t)ldq * s_dest[j]] = V[i + (size_t)k * j];
            }
        }
        if (tid == 0) {
            a.info[mat] = nonfinite ? -100 : (converged ? 0 : sweeps);
            atomicAdd(&a.cnt->rotations, (unsigned long long)rot);
            atomicAdd(&a.cnt->inner_sweeps, (unsigned long long)sweeps);
            atomicAdd(&a.cnt->pair_solves, 1ull);
            // per applied rotation: (k/2 - 1) quads (two 2x2 products) and a column pair of V
            const unsigned long long f = (unsigned long long)rot * (unsigned long long)(6 * k + (vec ? 6 * k : 0));
            if (sizeof(T) == 8) atomicAdd(&a.cnt->flops_fp64, f);
            else atomicAdd(&a.cnt->flops_fp32, f);
        }
        __syncthreads();
    }
}

// ================================================================ one-sided SVD
template <typename T>
__global__ void k_batched_svd(BatchedSvdArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ int s_item, s_cnt, s_bad;
    __shared__ T s_red[32];
    __shared__ int s_dest[kBatchedMaxK];
    CoreSmem<T> cs = carve_core<T>(bsm, kBatchedMaxK);
    cs.cnt = &s_cnt;
    const int tid = threadIdx.x, nt = blockDim.x;

    for (;;) {
        if (tid == 0) {  // the flag is cleared before the barrier that publishes the item
            s_item = (int)atomicAdd(a.queue, 1u);
            s_bad = 0;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= a.batch) break;
        const int mat = a.order[item];
        const int m = a.m[mat], n = a.n[mat], k = n + (n & 1);
        const size_t ntp = batched_tri_pad(k);
        T* Ap = (T*)(bsm + core_bytes<T>(kBatchedMaxK));       // packed Gram
        T* Vh = Ap + ntp;                                         // k x k pivot eigenvectors
        T* Vacc = Vh + (size_t)k * k;                             // accumulated V (k x k)
        T* rowbuf = Vacc + (size_t)k * k;                         // nt x (k+1) staging
        T* G = a.G[mat];
        const int ldg = a.ldg[mat];
        for (int idx = tid; idx < k * k; idx += nt) Vacc[idx] = (idx % k == idx / k) ? T(1) : T(0);
        int bad = 0;
        for (int idx = tid; idx < m * n; idx += nt) {
            if (!isfinite(G[(idx % m) + (size_t)ldg * (idx / m)])) bad = 1;
        }
        if (bad) atomicExch(&s_bad, 1);
        __syncthreads();
        const bool nonfinite = s_bad != 0;
        int sweeps = 0, rot_total = 0;
        bool converged = false;
        for (int sw = 0; !nonfinite && sw < a.max_sweeps; ++sw) {
            // Gram block (lower triangle), padding column k-1 (n odd) is zero
            for (int idx = tid; idx < (int)ntp; idx += nt) Ap[idx] = T(0);
            __syncthreads();
            for (int e = tid; e < k * (k + 1) / 2; e += nt) {
                // decode packed index e -> (ii >= jj)
                int ii = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
                while (tri(ii + 1) <= e) ++ii;
                while (tri(ii) > e) --ii;
                const int jj = e - tri(ii);
                if (ii >= n) continue;
                const T* gi = G + (size_t)ldg * ii;
                const T* gj = G + (size_t)ldg * jj;
                T acc = T(0);
                for (int r = 0; r < m; ++r) acc = fma(gi[r], gj[r], acc);
                Ap[e] = acc;
            }
            __syncthreads();
            // stop statistic: largest normalised off-diagonal before rotating
            T mx = T(0);
            for (int e = tid; e < k * (k + 1) / 2; e += nt) {
                int ii = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
                while (tri(ii + 1) <= e) ++ii;
                while (tri(ii) > e) --ii;
                const int jj = e - tri(ii);
                if (ii == jj) continue;
                const T d = sqrt(Ap[tri(ii) + ii]) * sqrt(Ap[tri(jj) + jj]);
                if (d > T(0)) mx = fmax(mx, fabs(Ap[e]) / d);
            }
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if ((tid & 31) == 0) s_red[tid >> 5] = mx;
            for (int idx = tid; idx < k * k; idx += nt) Vh[idx] = (idx % k == idx / k) ? T(1) : T(0);
            for (int x = tid; x < k; x += nt) cs.dlo[x] = T(0);
            __syncthreads();
            T smax = T(0);
            for (int w = 0; w < (nt + 31) / 32; ++w) smax = fmax(smax, s_red[w]);
            sweeps = sw + 1;
            if (smax <= a.tol) {
                converged = true;
                break;
            }
            int isw = 0;
            const int rot = jacobi_solve<T>(Ap, Vh, k, a.tol, a.inner_max_sweeps, a.qtab, cs, &isw);
            rot_total += rot;
            if (rot == 0) {
                converged = true;
                break;
            }
            // permutation: eigenpairs by descending eigenvalue over the n real positions
            for (int x = tid; x < k; x += nt) {
                int dest = x;
                if (x < n) {
                    const T dx = Ap[tri(x) + x];
                    int r = 0;
                    for (int y = 0; y < n; ++y) {
                        const T dy = Ap[tri(y) + y];
                        r += (dy > dx) || (dy == dx && y < x);
                    }
                    dest = r;
                }
                s_dest[x] = dest;
            }
            __syncthreads();
            // G(:, 0:n) <- G(:, 0:n) Vhat P, one row per thread through a staging row
            T* row = rowbuf + (size_t)tid * (k + 1);
            for (int r0 = 0; r0 < m; r0 += nt) {
                const int r = r0 + tid;
                if (r < m) {
                    for (int j = 0; j < n; ++j) row[j] = G[r + (size_t)ldg * j];
                    for (int j = 0; j < n; ++j) {
                        const int src = j;  // output column s_dest[src] gets G Vhat(:, src)
                        T acc = T(0);
                        for (int l = 0; l < n; ++l) acc = fma(row[l], Vh[l + (size_t)k * src], acc);
                        G[r + (size_t)ldg * s_dest[src]] = acc;
                    }
                }
            }
            // Vacc <- Vacc Vhat P (k x k, in shared memory)
            __syncthreads();
            for (int rr = tid; rr < n; rr += nt) {
                T* vr = rowbuf + (size_t)tid * (k + 1);
                for (int j = 0; j < n; ++j) vr[j] = Vacc[rr + (size_t)k * j];
                for (int j = 0; j < n; ++j) {
                    T acc = T(0);
                    for (int l = 0; l < n; ++l) acc = fma(vr[l], Vh[l + (size_t)k * j], acc);
                    Vacc[rr + (size_t)k * s_dest[j]] = acc;
                }
            }
            __syncthreads();
        }
        // finalise: sigma_j = ||G(:, j)||, U = G Sigma^+, descending (stable)
        T* sig = a.sigma[mat];
        T* nrm = Ap;  // reuse
        for (int j = tid; j < n; j += nt) {
            T s = T(0);
            for (int r = 0; r < m; ++r) s = fma(G[r + (size_t)ldg * j], G[r + (size_t)ldg * j], s);
            nrm[j] = sqrt(s);
        }
        __syncthreads();
        for (int x = tid; x < n; x += nt) {
            const T dx = nrm[x];
            int r = 0;
            for (int y = 0; y < n; ++y) r += (nrm[y] > dx) || (nrm[y] == dx && y < x);
            s_dest[x] = r;
        }
        __syncthreads();
        for (int x = tid; x < n; x += nt) sig[s_dest[x]] = nrm[x];
        // permute/scale U in place through the staging rows, V from Vacc
        T* row = rowbuf + (size_t)tid * (k + 1);
        for (int r0 = 0; r0 < m; r0 += nt) {
            const int r = r0 + tid;
            if (r < m) {
                for (int j = 0; j < n; ++j) row[j] = G[r + (size_t)ldg * j];
                for (int j = 0; j < n; ++j)
                    G[r + (size_t)ldg * s_dest[j]] = nrm[j] > T(0) ? row[j] / nrm[j] : T(0);
            }
        }
        if (a.V) {
            T* V = a.V[mat];
            const int ldv = a.ldv[mat];
            for (int idx = tid; idx < n * n; idx += nt) {
                const int i = idx % n, j = idx / n;
                V[i + (size_t)ldv * s_dest[j]] = Vacc[i + (size_t)k * j];
            }
        }
        if (tid == 0) {
            a.info[mat] = nonfinite ? -100 : (converged ? 0 : sweeps);
            atomicAdd(&a.cnt->rotations, (unsigned long long)rot_total);
            atomicAdd(&a.cnt->pair_solves, (unsigned long long)sweeps);
            const unsigned long long f = (unsigned long long)sweeps * (unsigned long long)(3ull * m * n * n);
            if (sizeof(T) == 8) atomicAdd(&a.cnt->flops_fp64, f);
            else atomicAdd(&a.cnt->flops_fp32, f);
        }
        __syncthreads();
    }
}

// ================================================================ launchers
template <typename T>
size_t batched_evd_smem(int smem_kmax, bool vec)
{
    size_t mat = smem_kmax > 0
                     ? (batched_tri_pad(smem_kmax) + (vec ? (size_t)smem_kmax * smem_kmax : 0)) * sizeof(T)
                     : 0;
    return core_bytes<T>(kBatchedMaxK) + mat;
}

template <typename T>
size_t batched_svd_smem(int kmax, int threads)
{
    return core_bytes<T>(kBatchedMaxK) +
           (batched_tri_pad(kmax) + 2 * (size_t)kmax * kmax + (size_t)threads * (kmax + 1)) * sizeof(T);
}

template <typename T>
cudaError_t launch_batched_evd(const BatchedEvdArgs<T>& a, int grid, int threads, cudaStream_t s)
{
    const size_t smem = batched_evd_smem<T>(a.smem_kmax, a.Q != nullptr);
    cudaError_t e = cudaFuncSetAttribute(k_batched_evd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_batched_evd<T><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batched_svd(const BatchedSvdArgs<T>& a, int kmax, int grid, int threads,
                               cudaStream_t s)
{
    const size_t smem = batched_svd_smem<T>(kmax, threads);
    cudaError_t e = cudaFuncSetAttribute(k_batched_svd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_batched_svd<T><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
int batched_evd_occupancy(int threads, int smem_kmax, bool vec)
{
    const size_t smem = batched_evd_smem<T>(smem_kmax, vec);
    if (cudaFuncSetAttribute(k_batched_evd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched_evd<T>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

template <typename T>
int batched_svd_occupancy(int threads, int kmax)
{
    const size_t smem = batched_svd_smem<T>(kmax, threads);
    if (cudaFuncSetAttribute(k_batched_svd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched_svd<T>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

template int batched_evd_occupancy<float>(int, int, bool);
template int batched_evd_occupancy<double>(int, int, bool);
template int batched_svd_occupancy<float>(int, int);
template int batched_svd_occupancy<double>(int, int);

__global__ void k_quad_table(unsigned* qtab, int h) { build_quad_table(qtab, h); }

cudaError_t launch_quad_table(unsigned* qtab, int h, cudaStream_t s)
{
    k_quad_table<<<1, 256, 0, s>>>(qtab, h);
    return cudaGetLastError();
}

template size_t batched_evd_smem<float>(int, bool);
template size_t batched_evd_smem<double>(int, bool);
template size_t batched_svd_smem<float>(int, int);
template size_t batched_svd_smem<double>(int, int);
template cudaError_t launch_batched_evd<float>(const BatchedEvdArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_batched_evd<double>(const BatchedEvdArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_batched_svd<float>(const BatchedSvdArgs<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_batched_svd<double>(const BatchedSvdArgs<double>&, int, int, int, cudaStream_t);

// ================================================================ one-sided SVD, row-tiled
// X(0:rows, 0:n) <- X(0:rows, 0:n) Vhat(0:n, 0:n) with output column j stored
// at dest[j].  Rows are staged kSvdTileRows at a time (column-major in
// `tile`); lane l of warp w forms rows l and l + 32 of the tile against the
// columns j = jc + w + nw y, y < 8, so the Vhat reads of a warp are
// broadcasts.  Each output is the FMA chain over l = 0..n-1 in order.
// X may be global (G) or shared (the accumulated V); no tile's rows are read
// after they are written.  All threads call; blockDim.x is a multiple of 32.
template <typename T>
__device__ void svd_rotate_rows(T* X, size_t ldx, int rows, int n, int k, const T* Vh, const int* dest, T* tile)
{
    constexpr int CT = 8;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, w = tid >> 5, nw = nt >> 5;
    for (int r0 = 0; r0 < rows; r0 += kSvdTileRows) {
        const int tr = min(kSvdTileRows, rows - r0);
        for (int idx = tid; idx < tr * n; idx += nt) {
            const int rr = idx % tr, c = idx / tr;
            tile[c * kSvdTileLd + rr] = X[(size_t)(r0 + rr) + ldx * c];
        }
        __syncthreads();
        for (int jc = 0; jc < n; jc += nw * CT) {
            T acc0[CT], acc1[CT];
#pragma unroll
            for (int y = 0; y < CT; ++y) acc0[y] = acc1[y] = T(0);
            for (int l = 0; l < n; ++l) {
                const T a0 = lane < tr ? tile[l * kSvdTileLd + lane] : T(0);
                const T a1 = lane + 32 < tr ? tile[l * kSvdTileLd + lane + 32] : T(0);
#pragma unroll
                for (int y = 0; y < CT; ++y) {
                    const int j = jc + w + nw * y;
                    const T b = j < n ? Vh[l + (size_t)k * j] : T(0);
                    acc0[y] = fma(a0, b, acc0[y]);
                    acc1[y] = fma(a1, b, acc1[y]);
                }
            }
#pragma unroll
            for (int y = 0; y < CT; ++y) {
                const int j = jc + w + nw * y;
                if (j >= n) continue;
                const size_t col = ldx * (size_t)dest[j];
                if (lane < tr) X[(size_t)(r0 + lane) + col] = acc0[y];
                if (lane + 32 < tr) X[(size_t)(r0 + lane + 32) + col] = acc1[y];
            }
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void k_batched_svd_tiled(BatchedSvdArgs<T> a, int kq)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ int s_item, s_cnt, s_bad;
    __shared__ T s_red[32];
    __shared__ int s_dest[kBatchedMaxK];
    CoreSmem<T> cs = carve_core<T>(bsm, kBatchedMaxK);
    cs.cnt = &s_cnt;
    const int tid = threadIdx.x, nt = blockDim.x;
    // layout after the core: packed Gram, Vhat, accumulated V (sized for the
    // plan's largest order kq - 3 <= kmax <= kq), then the row tile
    T* Ap = (T*)(bsm + core_bytes<T>(kBatchedMaxK));
    T* Vh = Ap + batched_tri_pad(kq);
    T* Vacc = Vh + (size_t)kq * kq;
    T* tile = Vacc + (size_t)kq * kq;                               // kSvdTileLd x kq

    for (;;) {
        if (tid == 0) {  // the flag is cleared before the barrier that publishes the item
            s_item = (int)atomicAdd(a.queue, 1u);
            s_bad = 0;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= a.batch) break;
        const int mat = a.order[item];
        const int m = a.m[mat], n = a.n[mat], k = n + (n & 1);
        const int nb4 = (n + 3) >> 2, nbl = nb4 * (nb4 + 1) / 2;   // 4 x 4 Gram blocks, lower
        const size_t ntp = batched_tri_pad(k);
        T* G = a.G[mat];
        const size_t ldg = (size_t)a.ldg[mat];
        for (int idx = tid; idx < k * k; idx += nt) Vacc[idx] = (idx % k == idx / k) ? T(1) : T(0);
        int bad = 0;
        for (int idx = tid; idx < m * n; idx += nt) {
            if (!isfinite(G[(size_t)(idx % m) + ldg * (idx / m)])) bad = 1;
        }
        if (bad) atomicExch(&s_bad, 1);
        __syncthreads();
        const bool nonfinite = s_bad != 0;
        int sweeps = 0, rot_total = 0;
        bool converged = false;
        for (int sw = 0; !nonfinite && sw < a.max_sweeps; ++sw) {
            // Gram (lower triangle): thread b0 + tid owns 4 x 4 block (bi, bj),
            // bi >= bj; columns n .. 4 nb4 - 1 of the tile are zero
            for (int idx = tid; idx < (int)ntp; idx += nt) Ap[idx] = T(0);
            for (int b0 = 0; b0 < nbl; b0 += nt) {
                const int bl = b0 + tid;
                const bool own = bl < nbl;
                int bi = 0, bj = 0;
                if (own) {
                    bi = (int)((sqrtf(8.0f * (float)bl + 1.0f) - 1.0f) * 0.5f);
                    while (tri(bi + 1) <= bl) ++bi;
                    while (tri(bi) > bl) --bi;
                    bj = bl - tri(bi);
                }
                T acc[4][4];
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] = T(0);
                for (int r0 = 0; r0 < m; r0 += kSvdTileRows) {
                    const int tr = min(kSvdTileRows, m - r0);
                    for (int idx = tid; idx < tr * 4 * nb4; idx += nt) {
                        const int rr = idx % tr, c = idx / tr;
                        tile[c * kSvdTileLd + rr] = c < n ? G[(size_t)(r0 + rr) + ldg * c] : T(0);
                    }
                    __syncthreads();
                    if (own) {
                        const T* ti = tile + 4 * bi * kSvdTileLd;
                        const T* tj = tile + 4 * bj * kSvdTileLd;
                        for (int r = 0; r < tr; ++r) {
                            T ai[4], aj[4];
#pragma unroll
                            for (int x = 0; x < 4; ++x) {
                                ai[x] = ti[x * kSvdTileLd + r];
                                aj[x] = tj[x * kSvdTileLd + r];
                            }
#pragma unroll
                            for (int x = 0; x < 4; ++x)
#pragma unroll
                                for (int y = 0; y < 4; ++y) acc[x][y] = fma(ai[x], aj[y], acc[x][y]);
                        }
                    }
                    __syncthreads();
                }
                if (own) {
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) {
                            const int i = 4 * bi + x, j = 4 * bj + y;
                            if (i < n && j <= i) Ap[tri(i) + j] = acc[x][y];
                        }
                }
            }
            __syncthreads();
            // stop statistic: largest normalised off-diagonal before rotating
            T mx = T(0);
            for (int e = tid; e < k * (k + 1) / 2; e += nt) {
                int ii = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
                while (tri(ii + 1) <= e) ++ii;
                while (tri(ii) > e) --ii;
                const int jj = e - tri(ii);
                if (ii == jj) continue;
                const T d = sqrt(Ap[tri(ii) + ii]) * sqrt(Ap[tri(jj) + jj]);
                if (d > T(0)) mx = fmax(mx, fabs(Ap[e]) / d);
            }
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if ((tid & 31) == 0) s_red[tid >> 5] = mx;
            for (int idx = tid; idx < k * k; idx += nt) Vh[idx] = (idx % k == idx / k) ? T(1) : T(0);
            for (int x = tid; x < k; x += nt) cs.dlo[x] = T(0);
            __syncthreads();
            T smax = T(0);
            for (int w = 0; w < (nt + 31) / 32; ++w) smax = fmax(smax, s_red[w]);
            sweeps = sw + 1;
            if (smax <= a.tol) {
                converged = true;
                break;
            }
            int isw = 0;
            const int rot = jacobi_solve<T>(Ap, Vh, k, a.tol, a.inner_max_sweeps, a.qtab, cs, &isw);
            rot_total += rot;
            if (rot == 0) {
                converged = true;
                break;
            }
            // permutation: eigenpairs by descending eigenvalue over the n real positions
            for (int x = tid; x < k; x += nt) {
                int dest = x;
                if (x < n) {
                    const T dx = Ap[tri(x) + x];
                    int r = 0;
                    for (int y = 0; y < n; ++y) {
                        const T dy = Ap[tri(y) + y];
                        r += (dy > dx) || (dy == dx && y < x);
                    }
                    dest = r;
                }
                s_dest[x] = dest;
            }
            __syncthreads();
            svd_rotate_rows<T>(G, ldg, m, n, k, Vh, s_dest, tile);
            svd_rotate_rows<T>(Vacc, (size_t)k, n, n, k, Vh, s_dest, tile);
        }
        // finalise: sigma_j = ||G(:, j)|| (FMA chain over the rows in order),
        // U = G Sigma^+, descending (stable)
        T* sig = a.sigma[mat];
        T* nrm = Ap;  // reuse
        for (int j = tid; j < n; j += nt) nrm[j] = T(0);
        __syncthreads();
        for (int r0 = 0; r0 < m; r0 += kSvdTileRows) {
            const int tr = min(kSvdTileRows, m - r0);
            for (int idx = tid; idx < tr * n; idx += nt) {
                const int rr = idx % tr, c = idx / tr;
                tile[c * kSvdTileLd + rr] = G[(size_t)(r0 + rr) + ldg * c];
            }
            __syncthreads();
            for (int j = tid; j < n; j += nt) {
                T s = nrm[j];
                for (int rr = 0; rr < tr; ++rr) s = fma(tile[j * kSvdTileLd + rr], tile[j * kSvdTileLd + rr], s);
                nrm[j] = s;
            }
            __syncthreads();
        }
        for (int j = tid; j < n; j += nt) nrm[j] = sqrt(nrm[j]);
        __syncthreads();
        for (int x = tid; x < n; x += nt) {
            const T dx = nrm[x];
            int r = 0;
            for (int y = 0; y < n; ++y) r += (nrm[y] > dx) || (nrm[y] == dx && y < x);
            s_dest[x] = r;
        }
        __syncthreads();
        for (int x = tid; x < n; x += nt) sig[s_dest[x]] = nrm[x];
        // permute / scale U in place, one staged row tile at a time; V from Vacc
        for (int r0 = 0; r0 < m; r0 += kSvdTileRows) {
            const int tr = min(kSvdTileRows, m - r0);
            for (int idx = tid; idx < tr * n; idx += nt) {
                const int rr = idx % tr, c = idx / tr;
                tile[c * kSvdTileLd + rr] = G[(size_t)(r0 + rr) + ldg * c];
            }
            __syncthreads();
            for (int idx = tid; idx < tr * n; idx += nt) {
                const int rr = idx % tr, j = idx / tr;
                G[(size_t)(r0 + rr) + ldg * s_dest[j]] = nrm[j] > T(0) ? tile[j * kSvdTileLd + rr] / nrm[j] : T(0);
            }
            __syncthreads();
        }
        if (a.V) {
            T* V = a.V[mat];
            const int ldv = a.ldv[mat];
            for (int idx = tid; idx < n * n; idx += nt) {
                const int i = idx % n, j = idx / n;
                V[i + (size_t)ldv * s_dest[j]] = Vacc[i + (size_t)k * j];
            }
        }
        if (tid == 0) {
            a.info[mat] = nonfinite ? -100 : (converged ? 0 : sweeps);
            atomicAdd(&a.cnt->rotations, (unsigned long long)rot_total);
            atomicAdd(&a.cnt->pair_solves, (unsigned long long)sweeps);
            const unsigned long long f = (unsigned long long)sweeps * (unsigned long long)(3ull * m * n * n);
            if (sizeof(T) == 8) atomicAdd(&a.cnt->flops_fp64, f);
            else atomicAdd(&a.cnt->flops_fp32, f);
        }
        __syncthreads();
    }
}

// tile columns: the plan's largest order rounded up to the 4 x 4 Gram blocks
static int svd_tile_cols(int kmax) { return (kmax + 3) / 4 * 4; }

template <typename T>
size_t batched_svd_tiled_smem(int kmax)
{
    const int kq = svd_tile_cols(kmax);
    return core_bytes<T>(kBatchedMaxK) +
           (batched_tri_pad(kq) + 2 * (size_t)kq * kq + (size_t)kSvdTileLd * kq) * sizeof(T);
}

template <typename T>
int batched_svd_tiled_occupancy(int threads, int kmax)
{
    const size_t smem = batched_svd_tiled_smem<T>(kmax);
    if (cudaFuncSetAttribute(k_batched_svd_tiled<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched_svd_tiled<T>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

template <typename T>
cudaError_t launch_batched_svd_tiled(const BatchedSvdArgs<T>& a, int kmax, int grid, int threads, cudaStream_t s)
{
    if (threads % 32 != 0 || threads < 32 || threads > 1024) return cudaErrorInvalidValue;
    const size_t smem = batched_svd_tiled_smem<T>(kmax);
    cudaError_t e = cudaFuncSetAttribute(k_batched_svd_tiled<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_batched_svd_tiled<T><<<grid, threads, smem, s>>>(a, svd_tile_cols(kmax));
    return cudaGetLastError();
}

template size_t batched_svd_tiled_smem<float>(int);
template size_t batched_svd_tiled_smem<double>(int);
template int batched_svd_tiled_occupancy<float>(int, int);
template int batched_svd_tiled_occupancy<double>(int, int);
template cudaError_t launch_batched_svd_tiled<float>(const BatchedSvdArgs<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_batched_svd_tiled<double>(const BatchedSvdArgs<double>&, int, int, int, cudaStream_t);

}  // namespace jac
