// api_f32.cu -- jacobi_syev_f32: the two-sided method on FP32 data.
//
// The caller's FP32 matrix is widened (exactly) into an FP64 working copy,
// the solve runs through jacobi_syev with the caller's parameters (FP64, the
// mixed forms or FP64_EMU), and D, the eigenvalues and Q are rounded back to
// FP32.  The result is therefore the FP64 solve of the widened input, rounded
// once: no FP32 sweep loses accuracy on the way.
#include <cuda_runtime.h>

#include "host.h"

using namespace jac;

namespace {

// y(r, c) = x(r, c) converted, for a rows x cols column-major block.
template <class S, class D>
__global__ void k_convert2d(int rows, int cols, const S* __restrict__ x, int ldx, D* __restrict__ y, int ldy)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * cols) return;
    const long long r = i % rows, c = i / rows;
    y[r + (long long)ldy * c] = (D)x[r + (long long)ldx * c];
}

template <class S, class D>
cudaError_t convert2d(int rows, int cols, const S* x, int ldx, D* y, int ldy, cudaStream_t s)
{
    const long long total = (long long)rows * cols;
    if (total <= 0) return cudaSuccess;
    const long long blocks = (total + 255) / 256;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_convert2d<S, D><<<(unsigned)blocks, 256, 0, s>>>(rows, cols, x, ldx, y, ldy);
    return cudaGetLastError();
}

}  // namespace

static int syev_f32(int n, float* A, int lda, float* w, float* Q, int ldq, const jacobi_params& p,
                    jacobi_stats* st, cudaStream_t s)
{
    const bool vec = p.want_vectors != 0;
    Workspace ws(s);
    double* dA = ws.get<double>((size_t)n * n);
    double* dw = ws.get<double>(n);
    double* dQ = vec ? ws.get<double>((size_t)n * n) : nullptr;
    if (ws.failed) return JACOBI_ERR_ALLOC;
    if (convert2d(n, n, A, lda, dA, n, s) != cudaSuccess) return JACOBI_ERR_CUDA;
    if (vec && p.warm_start && convert2d(n, n, Q, ldq, dQ, n, s) != cudaSuccess) return JACOBI_ERR_CUDA;
    const int rc = jacobi_syev(n, dA, n, dw, dQ, n, &p, st, (void*)s);
    if (rc < 0) return rc;
    if (convert2d(n, n, dA, n, A, lda, s) != cudaSuccess || convert2d(n, 1, dw, n, w, n, s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    if (vec && convert2d(n, n, dQ, n, Q, ldq, s) != cudaSuccess) return JACOBI_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return JACOBI_ERR_CUDA;
    return rc;
}

extern "C" int jacobi_syev_f32(int n, float* A, int lda, float* w, float* Q, int ldq,
                               const jacobi_params* pin, jacobi_stats* st, void* stream)
{
    jacobi_params p;
    if (pin) p = *pin; else jacobi_params_default(&p);
    if (n < 1) return -1;
    if (!A) return -2;
    if (lda < n) return -3;
    if (!w) return -4;
    if (p.want_vectors && !Q) return -5;
    if (p.want_vectors && ldq < n) return -6;
    const int e = check_params(p);
    if (e) return e;
    if (st) memset(st, 0, sizeof(*st));
    const int rc = syev_f32(n, A, lda, w, Q, ldq, p, st, (cudaStream_t)stream);
    if (st) st->status = rc;
    return rc;
}
