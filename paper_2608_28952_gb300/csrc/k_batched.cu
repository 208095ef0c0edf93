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
        if (tid == 0) s_item = (int)atomicAdd(a.queue, 1u);
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
        if (tid == 0) s_bad = 0;
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

}  // namespace jac
