// k_qr.cu -- Householder QR of a tall FP64 matrix, G = QR, in the blocked
// compact-WY form, for the one-sided SVD preconditioned by a reduced QR
// factorisation (Sec. 6, "Preprocessing with QR"): the one-sided method then
// runs on R^T and the left singular vectors are Q times its rotations.
//
// Column i of a panel of QR_NB columns: the reflector H_i = I - tau_i v_i v_i^T
// with v_i(i) = 1 that maps G(i:m, i) to beta e_1 (beta = -sign(alpha) ||x||,
// tau = (beta - alpha)/beta, v = x/(alpha - beta): the Householder vector as
// in LAPACK's dlarfg), applied to the rest of the panel.  The panel's
// reflectors are kept explicitly in Y (m x n, column i = v_i, zero above row
// i) with the upper-triangular T of H_1 ... H_nb = I - Y T Y^T (the forward
// recurrence T(0:i, i) = -tau_i T(0:i, 0:i) Y(:, 0:i)^T v_i, as in dlarft),
// so that the trailing columns and, later, the left factor are updated by
// matrix products: C <- C - Y T^T (Y^T C) and X <- X - Y T (Y^T X).
// Every reduction runs in a fixed order (bitwise reproducible).
#include <cuda_runtime.h>

#include "internal.h"

namespace jac {

namespace {

constexpr int QR_T = 1024;   // threads of the column kernels
constexpr int QR_KR = 512;   // rows per split of the Y^T X products

__device__ double block_reduce(double v, double* red, bool is_max)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_down_sync(0xffffffffu, v, o);
        v = is_max ? fmax(v, u) : v + u;
    }
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_down_sync(0xffffffffu, v, o);
            v = is_max ? fmax(v, u) : v + u;
        }
        if (lane == 0) red[32] = v;
    }
    __syncthreads();
    const double r = red[32];
    __syncthreads();
    return r;
}

// Householder vector of x = A(i:m, i): A(i, i) <- beta, Y(j0:m, i) <- v (zero
// above row i), tau[i] <- tau.  One CTA.
__global__ void __launch_bounds__(QR_T) k_house_vec(int m, double* __restrict__ A, int lda, int i,
                                                    double* __restrict__ Y, int ldy, int j0,
                                                    double* __restrict__ tau)
{
    __shared__ double red[33];
    const int tid = threadIdx.x;
    const double* x = A + (size_t)lda * i;
    const double alpha = x[i];
    double mx = 0.0;
    for (int r = i + 1 + tid; r < m; r += QR_T) mx = fmax(mx, fabs(x[r]));
    mx = block_reduce(mx, red, true);
    double xnorm = 0.0;
    if (mx > 0.0) {   // ||tail|| = mx ||tail / mx||, no overflow or underflow in the squares
        const double inv = 1.0 / mx;
        double ss = 0.0;
        for (int r = i + 1 + tid; r < m; r += QR_T) {
            const double y = x[r] * inv;
            ss = fma(y, y, ss);
        }
        xnorm = mx * sqrt(block_reduce(ss, red, false));
    }
    double* y = Y + (size_t)ldy * i;
    if (xnorm == 0.0) {   // already reduced: H = I
        if (tid == 0) tau[i] = 0.0;
        for (int r = j0 + tid; r < m; r += QR_T) y[r] = r == i ? 1.0 : 0.0;
        return;
    }
    const double big = fmax(fabs(alpha), xnorm), sml = fmin(fabs(alpha), xnorm), q = sml / big;
    const double h = big * sqrt(fma(q, q, 1.0));
    const double beta = alpha >= 0.0 ? -h : h;
    const double sc = 1.0 / (alpha - beta);
    if (tid == 0) {
        tau[i] = (beta - alpha) / beta;
        A[i + (size_t)lda * i] = beta;
    }
    for (int r = j0 + tid; r < m; r += QR_T) y[r] = r < i ? 0.0 : (r == i ? 1.0 : x[r] * sc);
}

// Block c < nrest: H_i applied to panel column i + 1 + c.  Block c >= nrest:
// S(kk, ii) = Y(:, j0 + kk)^T v_i for the earlier panel columns kk < ii
// (ii = i - j0), the inputs of T's column ii.
__global__ void __launch_bounds__(QR_T) k_house_apply(int m, double* __restrict__ A, int lda, int i, int j0,
                                                      int nrest, const double* __restrict__ Y, int ldy,
                                                      const double* __restrict__ tau, double* __restrict__ S)
{
    __shared__ double red[33];
    const int tid = threadIdx.x, c = blockIdx.x, ii = i - j0;
    const double* v = Y + (size_t)ldy * i;
    if (c < nrest) {
        double* col = A + (size_t)lda * (i + 1 + c);
        double d = 0.0;
        for (int r = i + tid; r < m; r += QR_T) d = fma(v[r], col[r], d);
        const double w = tau[i] * block_reduce(d, red, false);
        if (w != 0.0)
            for (int r = i + tid; r < m; r += QR_T) col[r] = fma(-w, v[r], col[r]);
    } else {
        const int kk = c - nrest;
        const double* yk = Y + (size_t)ldy * (j0 + kk);
        double d = 0.0;
        for (int r = i + tid; r < m; r += QR_T) d = fma(yk[r], v[r], d);
        d = block_reduce(d, red, false);
        if (tid == 0) S[kk + QR_NB * ii] = d;
    }
}

// T (upper triangular, nbp x nbp, ld QR_NB) of the panel and its transpose.
__global__ void k_house_T(int nbp, const double* __restrict__ S, const double* __restrict__ tau,
                          double* __restrict__ T, double* __restrict__ Tt)
{
    __shared__ double t[QR_NB][QR_NB + 1];
    const int r = threadIdx.x;   // QR_NB threads
    for (int c = 0; c < QR_NB; ++c) t[r][c] = 0.0;
    __syncthreads();
    for (int ii = 0; ii < nbp; ++ii) {
        double acc = 0.0;
        if (r < ii)
            for (int k = r; k < ii; ++k) acc = fma(t[r][k], S[k + QR_NB * ii], acc);
        __syncthreads();
        if (r < ii) t[r][ii] = -tau[ii] * acc;
        if (r == ii) t[r][ii] = tau[ii];
        __syncthreads();
    }
    for (int c = 0; c < QR_NB; ++c) {
        T[r + QR_NB * c] = t[r][c];
        Tt[c + QR_NB * r] = t[r][c];
    }
}

// Wpart[split] (nbp x ncol, ld QR_NB) = Y(rows of the split, panel)^T X(rows, cols):
// a 32 x 32 output tile per block, rows in chunks of 32 through shared memory;
// thread (a = t % 32, g = t / 32) owns row a and columns 4g .. 4g + 3.
__global__ void __launch_bounds__(256) k_qr_ytx(int rows, int nbp, int ncol, const double* __restrict__ Yp, int ldy,
                                                const double* __restrict__ Xp, int ldx, double* __restrict__ Wpart)
{
    __shared__ double ys[32][33], xs[32][33];
    const int tid = threadIdx.x, a = tid & 31, g = tid >> 5;
    const int c0 = blockIdx.x * 32, split = blockIdx.y;
    const int r0 = split * QR_KR, r1 = min(rows, r0 + QR_KR);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int rb = r0; rb < r1; rb += 32) {
        for (int e = tid; e < 32 * 32; e += 256) {
            const int rr = e & 31, cc = e >> 5, r = rb + rr;
            ys[rr][cc] = (r < r1 && cc < nbp) ? Yp[r + (size_t)ldy * cc] : 0.0;
            xs[rr][cc] = (r < r1 && c0 + cc < ncol) ? Xp[r + (size_t)ldx * (c0 + cc)] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
            const double yv = ys[rr][a];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(yv, xs[rr][4 * g + u], acc[u]);
        }
        __syncthreads();
    }
    double* W = Wpart + (size_t)split * QR_NB * ncol;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = c0 + 4 * g + u;
        if (a < nbp && c < ncol) W[a + (size_t)QR_NB * c] = acc[u];
    }
}

__global__ void k_qr_wsum(int nsplit, int count, const double* __restrict__ Wpart, double* __restrict__ W)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double s = 0.0;
    for (int p = 0; p < nsplit; ++p) s += Wpart[(size_t)p * count + i];   // fixed order
    W[i] = s;
}

// X = R^T (n x n, ld n) from the upper triangle of A.
__global__ void k_qr_rt(int n, const double* __restrict__ A, int lda, double* __restrict__ X)
{
    __shared__ double t[32][33];
    const int bi = blockIdx.x * 32, bj = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
    for (int q = ty; q < 32; q += 8) {   // t[q][tx] = A(bj + q, bi + tx) (row j, column i)
        const int j = bj + q, i = bi + tx;
        t[q][tx] = (i < n && j < n && j <= i) ? A[j + (size_t)lda * i] : 0.0;
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {   // X(i, j) = R(j, i)
        const int i = bi + tx, j = bj + q;
        if (i < n && j < n) X[i + (size_t)n * j] = t[q][tx];
    }
}

// G(0:m, 0:n) = [W; 0].
__global__ void k_qr_fill(int m, int n, const double* __restrict__ W, double* __restrict__ G, int ldg)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)m * n) return;
    const int r = (int)(e % m), c = (int)(e / m);
    G[r + (size_t)ldg * c] = r < n ? W[r + (size_t)n * c] : 0.0;
}

}  // namespace

size_t qr_wpart_doubles(int m, int n) { return (size_t)((m + QR_KR - 1) / QR_KR) * QR_NB * n; }

cudaError_t launch_house_panel(int m, double* A, int lda, int j0, int nbp, double* Y, int ldy, double* tau,
                               double* S, double* T, double* Tt, cudaStream_t s)
{
    for (int ii = 0; ii < nbp; ++ii) {
        const int i = j0 + ii;
        k_house_vec<<<1, QR_T, 0, s>>>(m, A, lda, i, Y, ldy, j0, tau);
        const int nrest = nbp - 1 - ii;
        if (nrest + ii > 0) k_house_apply<<<nrest + ii, QR_T, 0, s>>>(m, A, lda, i, j0, nrest, Y, ldy, tau, S);
    }
    k_house_T<<<1, QR_NB, 0, s>>>(nbp, S, tau + j0, T, Tt);
    return cudaGetLastError();
}

// X(j0:m, 0:ncol) <- X - Y_p M (Y_p^T X) with M = T^T (trans = 1, the
// trailing update of the factorisation) or T (trans = 0, applying Q).
cudaError_t launch_house_update(int m, int j0, int nbp, const double* Y, int ldy, const double* T,
                                const double* Tt, int trans, double* X, int ldx, int ncol, double* Wpart,
                                double* W, double* YT, cudaStream_t s)
{
    if (ncol <= 0) return cudaSuccess;
    const int rows = m - j0, nsplit = (rows + QR_KR - 1) / QR_KR;
    const double* Yp = Y + j0 + (size_t)ldy * j0;
    double* Xp = X + j0;
    k_qr_ytx<<<dim3((ncol + 31) / 32, nsplit), 256, 0, s>>>(rows, nbp, ncol, Yp, ldy, Xp, ldx, Wpart);
    const int count = QR_NB * ncol;
    k_qr_wsum<<<(count + 255) / 256, 256, 0, s>>>(nsplit, count, Wpart, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // YT = Y_p M (rows x nbp, ld m), then X -= YT W
    if ((e = launch_gemm64(rows, nbp, nbp, 1.0, Yp, ldy, 0, trans ? Tt : T, QR_NB, 0.0, YT, m, s)) != cudaSuccess)
        return e;
    return launch_gemm64(rows, ncol, nbp, -1.0, YT, m, 0, W, QR_NB, 1.0, Xp, ldx, s);
}

// The same update with FP64-accurate products on the tensor cores:
// W = (X^T Y_p)^T split over K (rows), then X += (-Y_p M) W.
cudaError_t launch_house_update_emu(int m, int j0, int nbp, const double* Y, int ldy, const double* T,
                                    const double* Tt, int trans, double* X, int ldx, int ncol, double* part,
                                    double* W, double* YT, int* xA, int* xB, int* err, cudaStream_t s)
{
    if (ncol <= 0) return cudaSuccess;
    const int rows = m - j0;
    const double* Yp = Y + j0 + (size_t)ldy * j0;
    double* Xp = X + j0;
    const int tiles = (ncol + 127) / 128, want = (3 * 152 + tiles - 1) / tiles;
    int kchunk = (rows + want - 1) / want;
    kchunk = ((kchunk + 255) / 256) * 256;
    if (kchunk < QR_KR) kchunk = QR_KR;   // the partial buffer holds ceil(rows / QR_KR) splits
    cudaError_t e = launch_emu_gemm_tsplit(ncol, nbp, rows, Xp, ldx, 1, Yp, ldy, W, QR_NB, kchunk, part, xA, xB, err, s);
    if (e != cudaSuccess) return e;
    if ((e = launch_gemm64(rows, nbp, nbp, -1.0, Yp, ldy, 0, trans ? Tt : T, QR_NB, 0.0, YT, m, s)) != cudaSuccess)
        return e;
    return launch_emu_gemm_big(rows, ncol, nbp, YT, m, 0, W, QR_NB, 1, Xp, ldx, 0, xA, xB, err, s);
}

cudaError_t launch_qr_rt(int n, const double* A, int lda, double* X, cudaStream_t s)
{
    k_qr_rt<<<dim3((n + 31) / 32, (n + 31) / 32), dim3(32, 8), 0, s>>>(n, A, lda, X);
    return cudaGetLastError();
}

cudaError_t launch_qr_fill(int m, int n, const double* W, double* G, int ldg, cudaStream_t s)
{
    const long long total = (long long)m * n;
    k_qr_fill<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(m, n, W, G, ldg);
    return cudaGetLastError();
}

}  // namespace jac
