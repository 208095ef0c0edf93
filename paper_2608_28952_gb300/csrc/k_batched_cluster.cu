// k_batched_cluster.cu -- the batched EVD for matrices too large for one
// CTA's shared memory: one thread-block cluster of C CTAs per matrix.
//
// The method is the batched form's: the scalar parallel-ordered Jacobi of
// the pivot solves (Algorithm 2 applied with b = 1 to the whole matrix,
// rotations in Rutishauser's form, diagonal carried as hi + lo), swept until
// a sweep applies no rotation.  The layout over the cluster follows the
// pivot cluster kernel: the packed lower triangle split by row ranges over
// the C CTAs' shared memory (reached through DSMEM addresses), V split by
// rows (local column rotations), every CTA with its own replica of the
// diagonal so that all CTAs choose identical rotations.  A split cluster
// barrier (arrive after choosing, wait before the rotated a_pq are zeroed)
// and a full barrier per round order the rounds.  Every loop has the same
// trip count in all CTAs of the cluster, so the barriers always match.
//
// Launch: grid = count x C, cluster (C, 1, 1), 512 threads; cluster c solves
// matrix order[c].  Orders up to 512 (FP32 with C = 8, FP64 with C = 16).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "batched.h"
#include "cluster_common.cuh"
#include "jacobi_core.cuh"

namespace cg = cooperative_groups;

namespace jac {

namespace {

constexpr int BC_T = 512;
constexpr int BC_MAXC = 16;

template <typename T>
__global__ void __launch_bounds__(BC_T) k_batched_evd_cluster(BatchedEvdArgs<T> a, const int* list, int C)
{
    extern __shared__ __align__(16) unsigned char bcs[];
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    const int mat = list[blockIdx.x / C];
    const int tid = threadIdx.x, nt = blockDim.x, gtid = r * nt + tid, gnt = C * nt;
    // order padded with zero rows/columns to a multiple of C (never rotated)
    const int n = a.n[mat], k = (n + C - 1) / C * C, half = k >> 1, nq = half * (half - 1) / 2;
    const int rows = k / C, r_lo = r * rows;
    const bool vec = a.Q != nullptr;

    Split sp;
    make_split(k, C, sp);
    int chunk_max = 0;
    for (int u = 0; u < C; ++u) chunk_max = max(chunk_max, sp.base[u + 1] - sp.base[u]);
    T* my_chunk = (T*)bcs;
    T* Vl = my_chunk + ((chunk_max + 1) & ~1);   // rows x k (ld rows): V(r_lo + i, j) at Vl[i + rows j]
    T* dhi = Vl + (vec ? (size_t)rows * k : 0);
    T* dlo = dhi + k;
    T* rtau = dlo + k;
    T* rs = rtau + half;
    T* rt = rs + half;
    T* rapq = rt + half;
    int* rp = (int*)(rapq + half);
    int* rq = rp + half;
    int* ron = rq + half;
    int* rinfo = ron + half;                     // [k] owner << 20 | local offset of row i
    __shared__ int s_cnt, s_bad, s_bad_all;
    __shared__ int s_dest[kBatchedMaxK];
    if (tid == 0) {
        s_bad = 0;
        s_bad_all = 0;
    }
    for (int i = tid; i < k; i += nt) {
        int ow = 0;
        for (int u = 1; u < C; ++u)
            if (i >= sp.row0[u]) ow = u;
        rinfo[i] = (ow << 20) | (tri(i) - sp.base[ow]);
    }
    const DistRows<T> dr{(uint32_t)__cvta_generic_to_shared(my_chunk), rinfo};
    __syncthreads();

    // ---- load the entries this CTA owns (lower triangle, zero padding), V rows = I.
    // Column-wise over the owned rows, so consecutive threads read
    // consecutive rows of one column of A.
    const int my_lo = sp.row0[r], my_hi = sp.row0[r + 1], nr = my_hi - my_lo;
    const T* A = a.A[mat];
    const size_t lda = (size_t)a.lda[mat];
    int bad = 0;
    for (int idx = tid; idx < nr * my_hi; idx += nt) {
        const int ii = my_lo + idx % nr, jj = idx / nr;
        if (jj > ii) continue;
        T v = T(0);
        if (ii < n) {
            v = A[ii + lda * jj];
            if (!isfinite(v)) bad = 1;
        }
        my_chunk[tri(ii) + jj - sp.base[r]] = v;
    }
    if (vec)
        for (int idx = tid; idx < rows * k; idx += nt) {
            const int i = idx % rows, j = idx / rows;
            Vl[idx] = (r_lo + i == j) ? T(1) : T(0);
        }
    if (bad) atomicExch(&s_bad, 1);
    __syncthreads();
    cluster.sync();   // every CTA has started and loaded: DSMEM is usable
    if (tid == 0 && s_bad) atomicExch(cluster.map_shared_rank(&s_bad_all, 0), 1);
    cluster.sync();
    if (tid == 0) s_bad = *cluster.map_shared_rank(&s_bad_all, 0);
    for (int x = tid; x < k; x += nt) {
        dhi[x] = dsm_ld(dr.addr(x, x), T(0));
        dlo[x] = T(0);
    }
    __syncthreads();
    const bool nonfinite = s_bad != 0;
    // V rows: thread -> row vi, rotations ve0, ve0 + vstep, ... (threads past
    // vstep * rows idle in that loop)
    const int vi = tid % rows, ve0 = tid / rows, vstep = nt / rows;

    // ---- sweeps until one applies no rotation
    const T tol = a.tol;
    const int max_sweeps = nonfinite ? 0 : a.max_sweeps;
    int total_rot = 0, sweeps = 0, last_cnt = 1;
    for (int sw = 0; sw < max_sweeps; ++sw) {
        if (tid == 0) s_cnt = 0;
        __syncthreads();
        for (int rd = 0; rd < k - 1; ++rd) {
            for (int ee = tid; ee < half; ee += nt) {
                const int pa = ee, pb = k - 1 - ee;
                const int ia = pa == 0 ? 0 : 1 + (pa - 1 + rd) % (k - 1);
                const int ib = 1 + (pb - 1 + rd) % (k - 1);
                const int p = ia < ib ? ia : ib, q = ia < ib ? ib : ia;
                const T app = dhi[p], aqq = dhi[q], apq = dsm_ld(dr.addr(q, p), T(0));
                const bool on = rotation_wanted(app, aqq, apq, tol);
                rp[ee] = p;
                rq[ee] = q;
                ron[ee] = on;
                if (on) {
                    T s, t, tau;
                    schur2(app, aqq, apq, s, t, tau);
                    rtau[ee] = tau;
                    rs[ee] = s;
                    rt[ee] = t;
                    rapq[ee] = apq;
                    atomicAdd(&s_cnt, 1);
                }
            }
            __syncthreads();
            asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
            for (int qi = gtid; qi < nq; qi += gnt) {
                int e1, e2;
                quad_decode(qi, e1, e2);
                const int on1 = ron[e1], on2 = ron[e2];
                if (!(on1 | on2)) continue;
                const int p1 = rp[e1], q1 = rq[e1], p2 = rp[e2], q2 = rq[e2];
                const uint32_t a00 = dr.addr(p1, p2), a01 = dr.addr(p1, q2);
                const uint32_t a10 = dr.addr(q1, p2), a11 = dr.addr(q1, q2);
                T x00 = dsm_ld(a00, T(0)), x01 = dsm_ld(a01, T(0)), x10 = dsm_ld(a10, T(0)),
                  x11 = dsm_ld(a11, T(0));
                if (on1) {
                    const T s = rs[e1], tau = rtau[e1];
                    rot2(s, tau, x00, x10);
                    rot2(s, tau, x01, x11);
                }
                if (on2) {
                    const T s = rs[e2], tau = rtau[e2];
                    rot2(s, tau, x00, x01);
                    rot2(s, tau, x10, x11);
                }
                dsm_st(a00, x00);
                dsm_st(a01, x01);
                dsm_st(a10, x10);
                dsm_st(a11, x11);
            }
            for (int ee = tid; ee < half; ee += nt) {
                if (!ron[ee]) continue;
                const int p = rp[ee], q = rq[ee];
                dd_add_prod(dhi[p], dlo[p], rt[ee], rapq[ee], T(-1));
                dd_add_prod(dhi[q], dlo[q], rt[ee], rapq[ee], T(1));
            }
            if (vec && ve0 < vstep)
                for (int ee = ve0; ee < half; ee += vstep) {
                    if (!ron[ee]) continue;
                    const int p = rp[ee], q = rq[ee];
                    T vp = Vl[vi + rows * p], vq = Vl[vi + rows * q];
                    rot2(rs[ee], rtau[ee], vp, vq);
                    Vl[vi + rows * p] = vp;
                    Vl[vi + rows * q] = vq;
                }
            asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
            if (r == 0)
                for (int ee = tid; ee < half; ee += nt)
                    if (ron[ee]) dsm_st(dr.addr(rq[ee], rp[ee]), T(0));
            cluster.sync();
        }
        const int cnt = s_cnt;
        total_rot += cnt;
        sweeps = sw + 1;
        last_cnt = cnt;
        __syncthreads();
        if (cnt == 0) break;
    }
    for (int x = tid; x < k; x += nt) dhi[x] += dlo[x];
    __syncthreads();

    // ---- ascending, stable rank among the n real positions; outputs
    for (int x = tid; x < n; x += nt) {
        const T dx = dhi[x];
        int rr = 0;
        for (int y = 0; y < n; ++y) {
            const T dy = dhi[y];
            rr += (dy < dx) || (dy == dx && y < x);
        }
        s_dest[x] = rr;
    }
    __syncthreads();
    if (r == 0) {
        T* w = a.w[mat];
        for (int x = tid; x < n; x += nt) w[s_dest[x]] = dhi[x];
    }
    if (vec) {
        T* Q = a.Q[mat];
        const size_t ldq = (size_t)a.ldq[mat];
        for (int idx = tid; idx < rows * k; idx += nt) {
            const int i = idx % rows, j = idx / rows;
            if (r_lo + i < n && j < n) Q[(r_lo + i) + ldq * s_dest[j]] = Vl[idx];
        }
    }
    if (r == 0 && tid == 0) {
        const bool converged = !nonfinite && last_cnt == 0;
        a.info[mat] = nonfinite ? -100 : (converged ? 0 : sweeps);
        atomicAdd(&a.cnt->rotations, (unsigned long long)total_rot);
        atomicAdd(&a.cnt->inner_sweeps, (unsigned long long)sweeps);
        atomicAdd(&a.cnt->pair_solves, 1ull);
        const unsigned long long f = (unsigned long long)total_rot * (unsigned long long)(6 * k + (vec ? 6 * k : 0));
        if (sizeof(T) == 8) atomicAdd(&a.cnt->flops_fp64, f);
        else atomicAdd(&a.cnt->flops_fp32, f);
    }
    // no CTA may leave while others can still read its shared memory
    cluster.sync();
}

}  // namespace

template <typename T>
size_t batched_cluster_smem(int k, int C, bool vec)
{
    if (k % C || k / C < 8) return (size_t)-1;
    const int half = k / 2;
    const size_t chunk = ((size_t)split_max_chunk(k, C) + 1) & ~(size_t)1;
    const size_t vrows = vec ? (size_t)(k / C) * k : 0;
    return (chunk + vrows + 2 * (size_t)k + 4 * (size_t)half) * sizeof(T) + (3 * (size_t)half + k) * sizeof(int) + 64;
}

// Whether clusters of 16 CTAs (a non-portable size) with this shared memory
// can be resident on the device at all.
template <typename T>
static bool cluster16_ok(size_t smem)
{
    if (cudaFuncSetAttribute(k_batched_evd_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_batched_evd_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(BC_T);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_batched_evd_cluster<T>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nc > 0;
}

template <typename T>
int batched_cluster_size(int k, bool vec, size_t smem_cap)
{
    for (int C = 2; C <= BC_MAXC; C *= 2) {
        const size_t smem = batched_cluster_smem<T>((k + C - 1) / C * C, C, vec);
        if (smem > smem_cap) continue;
        if (C > 8 && !cluster16_ok<T>(smem_cap)) return 0;
        return C;
    }
    return 0;
}

template <typename T>
cudaError_t launch_batched_evd_cluster(const BatchedEvdArgs<T>& a, const int* list, int count, int kmax,
                                       int C, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = batched_cluster_smem<T>(kmax, C, a.Q != nullptr);
    cudaError_t e = cudaFuncSetAttribute(k_batched_evd_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (C > 8 && (e = cudaFuncSetAttribute(k_batched_evd_cluster<T>,
                                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(count * C);
    cfg.blockDim = dim3(BC_T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batched_evd_cluster<T>, a, list, C);
}

template size_t batched_cluster_smem<float>(int, int, bool);
template size_t batched_cluster_smem<double>(int, int, bool);
template int batched_cluster_size<float>(int, bool, size_t);
template int batched_cluster_size<double>(int, bool, size_t);
template cudaError_t launch_batched_evd_cluster<float>(const BatchedEvdArgs<float>&, const int*, int, int, int,
                                                       cudaStream_t);
template cudaError_t launch_batched_evd_cluster<double>(const BatchedEvdArgs<double>&, const int*, int, int, int,
                                                        cudaStream_t);

}  // namespace jac
