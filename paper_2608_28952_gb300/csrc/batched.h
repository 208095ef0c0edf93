// batched.h -- argument blocks and launchers of the batched kernels.
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace jac {

constexpr int kBatchedMaxK = 512;   // largest (even-padded) order in the batched forms

template <typename T>
struct BatchedEvdArgs {
    int batch;
    const int* order;        // [batch] matrix indices, largest n first
    const int* n;            // [batch] orders
    T* const* A;             // [batch] device pointers (read only, lower triangle)
    const int* lda;
    T* const* w;             // [batch] eigenvalues, ascending
    T* const* Q;             // [batch] eigenvectors or null (no vectors)
    const int* ldq;
    int* info;               // [batch] 0 converged, >0 sweeps run, -100 non-finite
    unsigned* queue;         // work counter, zero at launch
    T* gscratch;             // grid x slot_elems for matrices beyond smem_kmax
    size_t slot_elems;
    int smem_kmax;           // even orders up to this run in shared memory
    const unsigned* qtab;    // quad table for half = kBatchedMaxK / 2
    T tol;                   // relative rotation threshold
    int max_sweeps;
    DevCounters* cnt;
};

template <typename T>
struct BatchedSvdArgs {
    int batch;
    const int* order;
    const int* m;
    const int* n;
    T* const* G;             // [batch] in: G, out: U
    const int* ldg;
    T* const* sigma;
    T* const* V;             // or null
    const int* ldv;
    int* info;
    unsigned* queue;
    const unsigned* qtab;
    T tol;                   // stop / rotation threshold (normalised)
    int max_sweeps;
    int inner_max_sweeps;
    DevCounters* cnt;
};

__host__ __device__ size_t batched_tri_pad(int k);
template <typename T>
size_t batched_evd_smem(int smem_kmax, bool vec);
template <typename T>
size_t batched_svd_smem(int kmax, int threads);
template <typename T>
cudaError_t launch_batched_evd(const BatchedEvdArgs<T>& a, int grid, int threads, cudaStream_t s);
template <typename T>
cudaError_t launch_batched_svd(const BatchedSvdArgs<T>& a, int kmax, int grid, int threads,
                               cudaStream_t s);
cudaError_t launch_quad_table(unsigned* qtab, int h, cudaStream_t s);
template <typename T>
int batched_evd_occupancy(int threads, int smem_kmax, bool vec);   // resident CTAs per SM
// Matrices above the shared-memory size: one cluster of C CTAs per matrix
// (order padded to a multiple of C).  list: `count` matrix indices; kmax:
// the largest padded order among them.
template <typename T>
size_t batched_cluster_smem(int k, int C, bool vec);
template <typename T>
int batched_cluster_size(int k, bool vec, size_t smem_cap);   // smallest C that fits, 0 if none
template <typename T>
cudaError_t launch_batched_evd_cluster(const BatchedEvdArgs<T>& a, const int* list, int count, int kmax,
                                       int C, cudaStream_t s);
template <typename T>
int batched_svd_occupancy(int threads, int kmax);
// Matrices above the shared-memory size by the blocked method, one CTA per
// matrix (persistent over `list`, its own queue word); slots: grid x
// slot_elems working storage (A and Q, padded).
template <typename T>
size_t batched_blocked_smem();
template <typename T>
int batched_blocked_ctas_per_sm();
template <typename T>
size_t batched_blocked_slot_elems(int nmax);
template <typename T>
cudaError_t launch_batched_evd_blocked(const BatchedEvdArgs<T>& a, const int* list, int count, unsigned* queue,
                                       T* slots, size_t slot_elems, int grid, cudaStream_t s);

}  // namespace jac
