// k_mixed.cu -- elementwise kernels of the mixed-precision form: FP32
// working copies, the return to FP64, and one refinement step of Ogita and
// Aishima (2018) for an approximate eigenvector matrix X of the original A0:
//     G = X^T X (so R = I - G),  S = X^T A0 X,
//     lam_i = s_ii / g_ii  (Rayleigh quotients; s_ii / (1 - r_ii)),
//     E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i)  for a resolved pair,
//     E_ij = r_ij / 2                                 otherwise, E_ii = r_ii / 2,
//     X <- X + X E.
// A pair counts as resolved when the quotient is small (|E_ij| <= 1e-2):
// the Newton correction is then a small rotation between two eigenvectors;
// otherwise (eigenvalues too close for the current accuracy) only the
// orthogonality part is applied and the closing FP64 Jacobi sweeps resolve
// the pair.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"

namespace jac {

// A32 <- mirrored lower triangle of A (n x n, lda) padded to np; Q32 <- I.
__global__ void k_load_sym32(int n, int np, const double* __restrict__ A, int lda,
                             float* __restrict__ A32, float* __restrict__ Q32, DevCounters* cnt)
{
    const long long total = (long long)np * np;
    int bad = 0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % np), j = (int)(idx / np);
        double v = 0.0;
        if (i < n && j < n) {
            v = i >= j ? A[i + (size_t)lda * j] : A[j + (size_t)lda * i];
            if (!isfinite(v)) bad = 1;
        }
        A32[idx] = (float)v;
        if (Q32) Q32[idx] = i == j ? 1.f : 0.f;
    }
    if (bad) atomicExch(&cnt->nonfinite, 1);
}

cudaError_t launch_load_sym32(int n, int np, const double* A, int lda, float* A32, float* Q32,
                              DevCounters* cnt, cudaStream_t s)
{
    long long total = (long long)np * np;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_load_sym32<<<blocks, 256, 0, s>>>(n, np, A, lda, A32, Q32, cnt);
    return cudaGetLastError();
}

// A0p (np x np FP64) <- mirrored lower triangle of A padded with zeros.
__global__ void k_pad_sym64(int n, int np, const double* __restrict__ A, int lda, double* __restrict__ A0p)
{
    const long long total = (long long)np * np;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % np), j = (int)(idx / np);
        double v = 0.0;
        if (i < n && j < n) v = i >= j ? A[i + (size_t)lda * j] : A[j + (size_t)lda * i];
        A0p[idx] = v;
    }
}

__global__ void k_f32_to_f64(long long count, const float* __restrict__ x, double* __restrict__ y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

// lam_i = s_ii / g_ii
__global__ void k_oa_lambda(int np, const double* __restrict__ S, const double* __restrict__ G,
                            double* __restrict__ lam)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) {
        const double g = G[i + (size_t)np * i];
        lam[i] = g != 0.0 ? S[i + (size_t)np * i] / g : 0.0;
    }
}

// G <- E (in place): r_ij = delta_ij - g_ij.
__global__ void k_oa_correction(int np, const double* __restrict__ S, double* __restrict__ G,
                                const double* __restrict__ lam, double eta)
{
    const long long total = (long long)np * np;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % np), j = (int)(idx / np);
        const double r = (i == j ? 1.0 : 0.0) - G[idx];
        double e = 0.5 * r;
        if (i != j) {
            const double d = lam[j] - lam[i];
            const double num = S[idx] + lam[j] * r;
            if (d != 0.0 && fabs(num) <= eta * fabs(d)) e = num / d;
        }
        G[idx] = e;
    }
}

// G <- (I - G) / 2: the Newton-Schulz correction X <- X + X (I - X^T X) / 2.
__global__ void k_ns_halfres(int np, double* __restrict__ G)
{
    const long long total = (long long)np * np;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % np), j = (int)(idx / np);
        G[idx] = 0.5 * ((i == j ? 1.0 : 0.0) - G[idx]);
    }
}

// B <- (S + S^T) / 2
__global__ void k_symmetrize(int np, const double* __restrict__ S, double* __restrict__ B)
{
    const long long total = (long long)np * np;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % np), j = (int)(idx / np);
        B[idx] = 0.5 * (S[idx] + S[j + (size_t)np * i]);
    }
}

static int grid_for(long long total)
{
    long long b = (total + 255) / 256;
    return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

cudaError_t launch_pad_sym64(int n, int np, const double* A, int lda, double* A0p, cudaStream_t s)
{
    k_pad_sym64<<<grid_for((long long)np * np), 256, 0, s>>>(n, np, A, lda, A0p);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(long long count, const float* x, double* y, cudaStream_t s)
{
    k_f32_to_f64<<<grid_for(count), 256, 0, s>>>(count, x, y);
    return cudaGetLastError();
}

cudaError_t launch_oa_step_elementwise(int np, const double* S, double* G, double* lam, double eta,
                                       cudaStream_t s)
{
    k_oa_lambda<<<(np + 255) / 256, 256, 0, s>>>(np, S, G, lam);
    k_oa_correction<<<grid_for((long long)np * np), 256, 0, s>>>(np, S, G, lam, eta);
    return cudaGetLastError();
}

cudaError_t launch_ns_halfres(int np, double* G, cudaStream_t s)
{
    k_ns_halfres<<<grid_for((long long)np * np), 256, 0, s>>>(np, G);
    return cudaGetLastError();
}

cudaError_t launch_symmetrize(int np, const double* S, double* B, cudaStream_t s)
{
    k_symmetrize<<<grid_for((long long)np * np), 256, 0, s>>>(np, S, B);
    return cudaGetLastError();
}

}  // namespace jac
