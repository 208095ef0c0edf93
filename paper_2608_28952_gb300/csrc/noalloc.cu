// noalloc.cu -- one parallel Jacobi step that allocates no memory.
//
// jacobi_syev_step_noalloc does what jacobi_syev_step does (the pivot solves
// of one step of the sweep schedule, then the block-row/column updates of A
// and the column updates of Q), but every buffer it needs besides the
// caller's A and Q lives in one fixed array in device global memory,
// g_noalloc_scratch below, so the call performs no cudaMalloc, cudaFree or
// other allocation, on the device or on the host.  This is for callers that
// cannot allocate: code running inside a framework that owns all device memory
// through its own pool (a foreign cudaMalloc would fail, or fragment the
// pool), and latency-critical loops that cannot afford the implicit
// synchronisation and unpredictable latency of an allocation.
//
// The array holds at most an order of kNoAllocMaxN = 768 and a block size of
// kNoAllocMaxB = 128; larger sizes are rejected with JACOBI_ERR_UNSUPPORTED,
// and so are the modes whose buffers it does not hold (emulated FP64
// products, the QRCP pivoting step).  The pivot solves run one CTA per pair,
// so the step agrees with jacobi_syev_step to rounding (bit for bit when that
// call runs one CTA per pair as well).
// It is statically sized, so every process that loads this library keeps it
// resident on every GPU it uses until the process exits (about 24 MB).
//
// Sharing: all calls use the same array and leave their contents in it; what
// must start at zero (the counters) is cleared by every call.  Two calls
// whose work overlaps on the GPU (on different streams, or from different
// host threads) race on the array and give wrong results: serialise them.
//
// Set-up: the first call on a device looks up the array's device address
// (cudaGetSymbolAddress, with that device current) and keeps it for later
// calls on that device.  Make that first call before any stream capture.
// The address is not looked up again, so after cudaDeviceReset the entry
// point must not be used on that device in the same process.
#include <cuda_runtime.h>
#include <string.h>

#include <atomic>

#include "host.h"

using namespace jac;

namespace {

constexpr int kNoAllocMaxN = 768;    // largest np (a multiple of b)
constexpr int kNoAllocMaxB = 128;    // largest block size
constexpr int kNoAllocMaxDevices = 64;

// Layout, in doubles: current and next A, current and next Q (np^2 each, ld
// np), Vhat and Vhat^T per pair (max pairs x 2 k^2 = 4 np b), global pivot
// scratch for k > 128 ((np / 256) pairs x (packed 256 + 256^2)), then the
// integer parts.
constexpr size_t kA = (size_t)kNoAllocMaxN * kNoAllocMaxN;
constexpr size_t kV = (size_t)4 * kNoAllocMaxN * kNoAllocMaxB;
constexpr size_t kG = (size_t)(kNoAllocMaxN / 256) * (((size_t)256 * 257 / 2 + 1) / 2 * 2 + 256 * 256);
constexpr size_t kInts = 2 * kNoAllocMaxN + kNoAllocMaxN + 64;   // pairs (int2), rot, counters
constexpr size_t kDoubles = 4 * kA + kV + kG + (kInts + 1) / 2;

__device__ __align__(256) double g_noalloc_scratch[kDoubles];

std::atomic<double*> g_scratch_addr[kNoAllocMaxDevices];

double* scratch_address(int dev)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices) return nullptr;
    double* p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (p) return p;
    void* q = nullptr;
    if (cudaGetSymbolAddress(&q, g_noalloc_scratch) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    g_scratch_addr[dev].store((double*)q, std::memory_order_release);
    return (double*)q;
}

// Pairs of step `step` of the sweep schedule (the same rule as the library's
// allocating schedule builder), written to out as {I, J}; blocks a step of
// Algorithm 3 leaves out are emitted as one frozen entry {-1-I, -1-J}.
// Returns the entry count (N/2) or -1.
int step_entries(int kind, int N, int step, int2* out)
{
    if (N < 2 || (N & 1)) return -1;
    const int half = N / 2;
    if (kind == JACOBI_ORDER_ROUND_ROBIN) {
        if (step < 0 || step >= N - 1) return -1;
        for (int j = 0; j < half; ++j) {
            const int pa = j, pb = N - 1 - j;
            const int x = pa == 0 ? 0 : 1 + (pa - 1 + step) % (N - 1);
            const int y = 1 + (pb - 1 + step) % (N - 1);
            out[j] = make_int2(x < y ? x : y, x < y ? y : x);
        }
        return half;
    }
    if (kind != JACOBI_ORDER_ANTI_DIAGONAL || step < 0 || step >= N) return -1;
    unsigned char used[kNoAllocMaxN];
    memset(used, 0, (size_t)N);
    int c = 0;
    for (int I = 1; I < N; ++I)
        for (int J = I + 1; J <= N; ++J)
            if ((I + J) % N == step) {
                out[c++] = make_int2(I - 1, J - 1);
                used[I - 1] = used[J - 1] = 1;
            }
    int left[2], nl = 0;
    for (int x = 0; x < N && nl < 2; ++x)
        if (!used[x]) left[nl++] = x;
    if (nl == 2) out[c++] = make_int2(-1 - left[0], -1 - left[1]);
    return c == half ? c : -1;
}

}  // namespace

extern "C" int jacobi_syev_step_noalloc(int np, double* A, int lda, double* Q, int ldq,
                                        const jacobi_params* pin, int step, void* stream)
{
    jacobi_params p;
    if (pin) p = *pin; else jacobi_params_default(&p);
    // The same parameter checks as jacobi_syev_step, then the limits of this
    // entry point: plain FP64 products (the emulated products need a stage-1
    // buffer sized by the step), no QRCP pivoting step (its scratch is sized
    // by the pairs), and the array's size.
    const int e = check_params(p);
    if (e) return e == -7 ? -6 : e;
    if (p.precision != JACOBI_PREC_FP64 || p.fp64_products != 0 || p.pivot_order == 2)
        return JACOBI_ERR_UNSUPPORTED;
    if (p.b > kNoAllocMaxB) return JACOBI_ERR_UNSUPPORTED;
    if (p.inner_max_sweeps == 0) p.inner_max_sweeps = 1;  // automatic, as in jacobi_syev_step
    if (np < 2 * p.b || np % p.b || (np / p.b) % 2) return -1;
    if (np > kNoAllocMaxN) return JACOBI_ERR_UNSUPPORTED;
    if (!A) return -2;
    if (lda < np) return -3;
    if (Q && ldq < np) return -5;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return JACOBI_ERR_CUDA;
    double* base = scratch_address(dev);
    if (!base) return JACOBI_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int b = p.b, k = 2 * b, N = np / b;
    int2 h_pairs[kNoAllocMaxN / 2];
    const int npairs = step_entries(p.ordering, N, step, h_pairs);
    if (npairs < 0) return -7;

    double* Acur = base;
    double* Anext = Acur + kA;
    double* Qcur = Anext + kA;
    double* Qnext = Qcur + kA;
    double* Vb = Qnext + kA;
    double* gscr = Vb + kV;
    int* ints = (int*)(gscr + kG);
    int2* d_pairs = (int2*)ints;
    int* d_rot = ints + 2 * kNoAllocMaxN;
    DevCounters* d_cnt = (DevCounters*)(((uintptr_t)(d_rot + kNoAllocMaxN) + 15) & ~(uintptr_t)15);

    const size_t bytes = (size_t)np * 8;
    if (cudaMemcpyAsync(d_pairs, h_pairs, sizeof(int2) * npairs, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(d_cnt, 0, sizeof(DevCounters), s) != cudaSuccess ||
        cudaMemcpy2DAsync(Acur, bytes, A, (size_t)lda * 8, bytes, np, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpy2DAsync(Anext, bytes, A, (size_t)lda * 8, bytes, np, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    if (Q && cudaMemcpy2DAsync(Qcur, bytes, Q, (size_t)ldq * 8, bytes, np, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    PivotArgs pa{};
    pa.Ain = Acur;
    pa.Aout = Anext;
    pa.ld = np;
    pa.pairs = d_pairs;
    pa.npairs = npairs;
    pa.b = b;
    pa.k = k;
    pa.V = Vb;
    pa.rot = d_rot;
    pa.tol_rel = p.inner_tol;
    pa.max_sweeps = p.inner_max_sweeps;
    pa.order = p.pivot_order;
    pa.n_real = np;
    pa.gscratch = gscr;
    pa.cnt = d_cnt;
    if (launch_pivot(pa, s) != cudaSuccess) return JACOBI_ERR_CUDA;
    UpdateArgs ua{};
    ua.Ain = Acur;
    ua.Aout = Anext;
    ua.lda = np;
    ua.Qin = Q ? Qcur : nullptr;
    ua.Qout = Q ? Qnext : nullptr;
    ua.ldq = np;
    ua.qrows = np;
    ua.pairs = d_pairs;
    ua.npairs = npairs;
    ua.b = b;
    ua.k = k;
    ua.V = Vb;
    ua.rot = d_rot;
    ua.cnt = d_cnt;
    if (launch_update_evd(ua, s) != cudaSuccess) return JACOBI_ERR_CUDA;
    if (cudaMemcpy2DAsync(A, (size_t)lda * 8, Anext, bytes, bytes, np, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    if (Q && cudaMemcpy2DAsync(Q, (size_t)ldq * 8, Qnext, bytes, bytes, np, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return JACOBI_ERR_CUDA;
    return 0;
}
