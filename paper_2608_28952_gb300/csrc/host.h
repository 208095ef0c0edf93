// host.h -- host-side helpers shared by the C-ABI drivers (workspace,
// timing, CUDA-graph capture of a sweep, parameter checks) and the FP64
// two-sided sweep runner used by the plain and the mixed-precision drivers.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "internal.h"

namespace jac {

constexpr double U64 = 1.1102230246251565e-16;  // 2^-53

// Stream-ordered workspace that is released when the call returns.  The
// environment variable JACOBI_WORKSPACE_LIMIT=<bytes> caps what one
// Workspace may hold (host-side fault injection: the call then returns
// JACOBI_ERR_ALLOC before it launches anything, as on a real allocation
// failure).
struct Workspace {
    cudaStream_t s;
    std::vector<void*> ptrs;
    bool failed = false;
    size_t used = 0, limit = (size_t)-1;
    explicit Workspace(cudaStream_t st) : s(st)
    {
        if (const char* e = getenv("JACOBI_WORKSPACE_LIMIT")) limit = (size_t)strtoull(e, nullptr, 10);
    }
    template <class T>
    T* get(size_t count)
    {
        if (count == 0) count = 1;
        const size_t bytes = count * sizeof(T);
        if (failed || bytes > limit - used) {
            failed = true;
            return nullptr;
        }
        void* p = nullptr;
        if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
            failed = true;
            cudaGetLastError();
            return nullptr;
        }
        used += bytes;
        ptrs.push_back(p);
        return (T*)p;
    }
    ~Workspace()
    {
        for (void* p : ptrs) cudaFreeAsync(p, s);
        cudaStreamSynchronize(s);
    }
};

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st)
    {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    double stop()
    {
        float ms = 0.f;
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
    ~Timer()
    {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

// Events recorded between the kernels of a sweep (inside the captured graph),
// read after the sweep to split the device time into pivot and update phases.
struct PhaseEvents {
    std::vector<cudaEvent_t> ev;
    explicit PhaseEvents(size_t n) : ev(n, nullptr)
    {
        for (auto& e : ev) cudaEventCreate(&e);
    }
    ~PhaseEvents()
    {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
    float ms(size_t a, size_t b) const
    {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ev[a], ev[b]) != cudaSuccess) {
            cudaGetLastError();
            return 0.f;
        }
        return t;
    }
};

// A captured sweep, replayed on the caller's stream.
struct SweepGraph {
    cudaGraphExec_t exec = nullptr;
    ~SweepGraph()
    {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

// Capture `body` (a function issuing launches on stream cs) into g; returns
// false when capture is not possible, in which case the caller launches
// directly.
template <class F>
inline bool capture(SweepGraph& g, F body)
{
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    bool ok = false;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        bool launched = body(cs);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (launched && e == cudaSuccess && graph) {
            ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
        }
        if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
    cudaStreamDestroy(cs);
    return ok;
}

// The emulated FP64 products slice an operand once into an image (V once
// per step in the update; both operands once per refinement product) by
// default; JACOBI_EMU_IMAGE=0 makes every tile slice its operands itself
// (the same slices, so the same results bit for bit).
inline bool emu_image_wanted()
{
    const char* e = getenv("JACOBI_EMU_IMAGE");
    return !(e && e[0] == '0');
}

// Cluster size for the pivot solves of a step with npairs pairs of order k:
// automatic unless JACOBI_PIVOT_CLUSTER is set ("1" = one CTA per pair, a
// power of two <= 8 = that size when it fits).
inline int choose_pivot_cluster(int k, int npairs)
{
    int dev = 0, sms = 0, smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int C = pivot_cluster_size(k, npairs, sms, (size_t)smem);
    if (const char* env = getenv("JACOBI_PIVOT_CLUSTER")) {
        const int want = atoi(env);
        if (want == 1) C = 1;
        else if (want == 2 || want == 4 || want == 8) {
            if (k % want == 0 && k / want >= 8 && pivot_cluster_smem(k, want) + 8192 <= (size_t)smem) C = want;
        }
    }
    return C;
}

inline int check_params(const jacobi_params& p)
{
    if (p.b < 1) return -7;
    if (p.b > 128) return JACOBI_ERR_UNSUPPORTED;
    if (p.ordering != JACOBI_ORDER_ROUND_ROBIN && p.ordering != JACOBI_ORDER_ANTI_DIAGONAL) return -7;
    if (p.max_sweeps < 0 || p.max_sweeps > 1000 || p.inner_max_sweeps < 0) return -7;
    if (!(p.tol >= 0.0) || !(p.inner_tol >= 0.0)) return -7;
    if (p.conv != JACOBI_CONV_OFF_ABS && p.conv != JACOBI_CONV_REL) return -7;
    if (p.pivot_order < 0 || p.pivot_order > 2) return -7;
    if (p.precision < JACOBI_PREC_FP64 || p.precision > JACOBI_PREC_FP64_EMU) return -7;
    if (p.fp64_products != 0 && p.fp64_products != 1) return -7;
    if (p.svd_qr != 0 && p.svd_qr != 1) return -7;
    return 0;
}

inline void fill_counters(jacobi_stats* st, const DevCounters& c)
{
    st->rotations = (long long)c.rotations;
    st->inner_sweeps = (long long)c.inner_sweeps;
    st->pair_solves = (long long)c.pair_solves;
    st->flops_fp64 = (double)c.flops_fp64;
    st->flops_update = (double)c.flops_update;
    st->flops_fp32 = (double)c.flops_fp32;
    st->flops_lowp = (double)c.flops_lowp;
}


// Plain FP64 two-sided driver on an already loaded, padded working pair
// (Aw[cur], Qw[cur]).  Runs until the stop test passes; on return *cur
// indexes the buffers holding the result.  Used by jacobi_syev and by the
// closing sweeps of the mixed form.
struct EvdState {
    int np, b, k;
    int n_real;   // rows/columns >= n_real are zero padding
    int pcl = 1;  // pivot cluster size (1: one CTA per pair)
    unsigned* qtab = nullptr;
    Ordering ord;
    int2* dpairs;
    double* Aw[2];
    double* Qw[2];
    double* Vb;
    int* rot;
    double* gscratch;
    double* partial;
    unsigned* ticket;
    double* result;
    DevCounters* cnt;
    // FP64 products on the tensor cores (JACOBI_PREC_FP64_EMU): the stage-1
    // products and the timeout word
    double* T64 = nullptr;
    int* err = nullptr;
    // the step's V sliced once (bf16 digit images) and its column scales
    unsigned char* vimg = nullptr;
    int* vexp = nullptr;
    // and the step's stage-1 operands (A's pair-blocks, Q's column pairs)
    unsigned char* aimg = nullptr;
    int* atab = nullptr;
    unsigned char* qimg = nullptr;
    int* qexp = nullptr;
    // pivot_order == 2: the per-pair QRCP scratch of the pivoting step
    double* qrws = nullptr;
    // emulated products: balance by the diagonal (relative stop criterion)
    int balance = 0;
};

// Result of a run of sweeps: code 0 converged, 1 max_sweeps ran out, <0 error.
struct SweepResult {
    int code;
    int sweeps;
};

SweepResult run_evd_sweeps(EvdState& E, const jacobi_params& p, int& cur, double target,
                           int sweep0, jacobi_stats* st, cudaStream_t s, bool use_rel);

// Mixed-precision two-sided driver (low-precision sweeps on the tensor
// cores, refinement against A0 in FP64, FP64 closing sweeps).
int syev_mixed(int n, double* A, int lda, double* w, double* Q, int ldq, const jacobi_params& p,
               jacobi_stats* st, cudaStream_t s);

}  // namespace jac
