// qrcp.cuh -- the pivoting step of Sec. 2.1 inside a pivot kernel: column-
// pivoted QR (Businger-Golub) of the leading rows of Vhat, whose column order
// becomes the permutation Vhat <- Vhat P (the condition of Drmac's
// convergence proof for block Jacobi).
//
// Run by one whole CTA on M (r1 x nr, column-major, ld r1, in the pair's
// global scratch, overwritten): at step t the remaining column of largest
// norm over rows t.. (recomputed at every step in a fixed order, ties to the
// smaller index) is swapped to position t and a Householder reflection
// clears it below row t.  perm (shared memory, nr entries) receives the
// column order; cn (nr doubles) and vh (r1 doubles) are shared scratch.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace jac {

__device__ inline void qrcp_order(int r1, int nr, double* M, int* perm, double* cn, double* vh)
{
    __shared__ int s_best;
    __shared__ double s_h[3];   // tau, scale, skip
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    for (int j = tid; j < nr; j += nt) perm[j] = j;
    __syncthreads();
    const int steps = r1 < nr ? r1 : nr;
    for (int t = 0; t < steps; ++t) {
        for (int j = t + tid; j < nr; j += nt) {
            double s = 0.0;
            for (int i = t; i < r1; ++i) s = fma(M[i + (size_t)r1 * j], M[i + (size_t)r1 * j], s);
            cn[j] = s;
        }
        __syncthreads();
        if (warp == 0) {   // argmax, ties to the smaller index
            double bv = -1.0;
            int bi = t;
            for (int j = t + lane; j < nr; j += 32)
                if (cn[j] > bv) { bv = cn[j]; bi = j; }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_down_sync(0xffffffffu, bv, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            if (lane == 0) s_best = bi;
        }
        __syncthreads();
        const int best = s_best;
        if (best != t) {
            for (int i = tid; i < r1; i += nt) {
                const double a = M[i + (size_t)r1 * t];
                M[i + (size_t)r1 * t] = M[i + (size_t)r1 * best];
                M[i + (size_t)r1 * best] = a;
            }
            if (tid == 0) {
                const int p = perm[t];
                perm[t] = perm[best];
                perm[best] = p;
            }
        }
        __syncthreads();
        if (warp == 0) {   // the reflection for column t over rows t..r1-1
            double ss = 0.0;
            for (int i = t + 1 + lane; i < r1; i += 32) ss = fma(M[i + (size_t)r1 * t], M[i + (size_t)r1 * t], ss);
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
            if (lane == 0) {
                const double alpha = M[t + (size_t)r1 * t], xn = sqrt(ss);
                if (xn == 0.0) {
                    s_h[2] = 1.0;
                } else {
                    const double beta = -copysign(hypot(alpha, xn), alpha);
                    s_h[0] = (beta - alpha) / beta;
                    s_h[1] = 1.0 / (alpha - beta);
                    s_h[2] = 0.0;
                }
            }
        }
        __syncthreads();
        if (s_h[2] != 0.0) continue;   // H = I (uniform: every thread reads the same flag)
        const double tau = s_h[0], sc = s_h[1];
        for (int i = t + tid; i < r1; i += nt) vh[i] = i == t ? 1.0 : M[i + (size_t)r1 * t] * sc;
        __syncthreads();
        for (int j = t + 1 + tid; j < nr; j += nt) {
            double w = 0.0;
            for (int i = t; i < r1; ++i) w = fma(vh[i], M[i + (size_t)r1 * j], w);
            w *= tau;
            for (int i = t; i < r1; ++i) M[i + (size_t)r1 * j] = fma(-w, vh[i], M[i + (size_t)r1 * j]);
        }
        __syncthreads();
    }
}

}  // namespace jac
