// api_batched.cu -- batched C ABI: thousands of independent matrices per call,
// one persistent launch per batch, captured once into a CUDA graph (plan API)
// and replayed; launch shape chosen by an autotuner with an in-process cache
// (optionally persisted to the file named by JACOBI_TUNE_CACHE).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "batched.h"
#include "batched_svd.h"

using namespace jac;

namespace {

constexpr double U64 = 1.1102230246251565e-16;
constexpr double U32 = 5.9604644775390625e-08;

// ------------------------------------------------------------------ launch shapes
struct Shape {
    int threads = 256;
    int smem_kmax = 0;   // EVD: even orders up to this are solved in shared memory
    int blk_min = -1;    // EVD: orders above this use the blocked method (b = 16), orders
                         // from smem_kmax up to it the unblocked solve on a cluster
                         // (-1: the measured default, 320 in FP64, 0 in FP32)
};

constexpr int kBatchedBlockB = 16;   // the block size of the batched blocked method

int blk_min_of(const Shape& sh, int esize) { return sh.blk_min >= 0 ? sh.blk_min : (esize == 8 ? 320 : 0); }

std::mutex g_tune_mu;
std::map<std::string, Shape> g_tune;  // key -> tuned shape
bool g_tune_loaded = false;

void tune_load_locked()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = getenv("JACOBI_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char line[512], key[256];
    while (fgets(line, sizeof(line), f)) {
        int th = 0, sk = 0, bm = -1;
        const int got = sscanf(line, "%255s %d %d %d", key, &th, &sk, &bm);
        if (got >= 3) g_tune[key] = Shape{th, sk, got == 4 ? bm : -1};
    }
    fclose(f);
}

void tune_store_locked()
{
    const char* path = getenv("JACOBI_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "w");
    if (!f) return;
    for (auto& kv : g_tune)
        fprintf(f, "%s %d %d %d\n", kv.first.c_str(), kv.second.threads, kv.second.smem_kmax, kv.second.blk_min);
    fclose(f);
}

// Tuning key: kind, element size, vectors, and the size mix (log2 buckets of
// the largest and the median order).
std::string tune_key(int kind, int esize, int vec, const std::vector<int>& n)
{
    std::vector<int> s(n);
    std::sort(s.begin(), s.end());
    auto lg = [](int x) { int l = 0; while ((1 << l) < x) ++l; return l; };
    char buf[96];
    snprintf(buf, sizeof(buf), "k%d_e%d_v%d_max%d_med%d", kind, esize, vec, lg(s.back()),
             lg(s[s.size() / 2]));
    return buf;
}

int device_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

size_t device_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)v;
}

// Candidate shapes for the EVD kernel: thread counts x shared-memory limits
// that fit the opt-in maximum.
template <typename T>
std::vector<Shape> evd_candidates(bool vec)
{
    const size_t cap = device_smem_optin() - 4096;  // static shared memory of the kernel
    std::vector<Shape> out;
    const int ks[] = {0, 32, 64, 96, 128, 160, 192, 224, 256, 320};
    for (int th : {128, 256, 512}) {
        int best = 0;
        for (int k : ks)
            if (batched_evd_smem<T>(k, vec) <= cap) best = k;
        out.push_back(Shape{th, best});
        if (best >= 64) out.push_back(Shape{th, best / 2});  // 2 CTAs/SM variant
    }
    return out;
}

Shape evd_default(int esize, bool vec)
{
    Shape s;
    s.threads = 256;
    s.smem_kmax = esize == 8 ? (vec ? 128 : 224) : (vec ? 160 : 320);
    return s;
}

}  // namespace

// ============================================================================ plan
struct jacobi_plan {
    int kind;            // 0 syev, 1 gesvd
    int precision;       // JACOBI_PREC_FP64 / FP32
    int esize;
    int batch;
    int vec;
    jacobi_params p;
    std::vector<int> h_m, h_n, h_lda, h_ldq, h_order;
    Shape shape;
    int grid = 0;
    int kmax = 0;
    // device workspace
    int *d_order = nullptr, *d_m = nullptr, *d_n = nullptr, *d_lda = nullptr, *d_ldq = nullptr;
    void** d_ptrs = nullptr;          // 3 * batch device pointers (A|G, w|sigma, Q|V)
    void** h_ptrs = nullptr;          // pinned staging of the same
    unsigned* d_queue = nullptr;
    unsigned* d_qtab = nullptr;
    void* d_scratch = nullptr;
    size_t slot_elems = 0;
    DevCounters* d_cnt = nullptr;
    cudaGraphExec_t exec = nullptr;
    int* graph_info = nullptr;        // info pointer baked into the graph
    int large_mode = 2;               // EVD orders above the smem size: 0 L2 slots, 1 clusters, 2 blocked
    bool svd_tiled = false;           // one-sided: the row-tiled kernel (default; JACOBI_BATCHED_SVD=rowwise: the other)
    void* d_blk = nullptr;            // blocked-form slots
    size_t blk_slot = 0;
    int blk_grid = 0;
    float last_ms = 0.f;
};

namespace {

size_t max_slot_elems(int kmax, bool vec)
{
    return batched_tri_pad(kmax) + (vec ? (size_t)kmax * kmax : 0);
}

// Launch the batch (or the sub-list `h_list` / `d_list`, matrix indices in
// longest-first order): EVD matrices above the shared-memory size go to the
// cluster kernel (grouped by cluster size, largest first), the rest to the
// persistent kernel.
template <typename T>
cudaError_t plan_launch(jacobi_plan* pl, int* info, cudaStream_t s, const Shape& sh, int grid,
                        const std::vector<int>& h_list, const int* d_list)
{
    cudaError_t e = cudaMemsetAsync(pl->d_queue, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const int B = pl->batch, count = (int)h_list.size();
    if (pl->kind == 0) {
        BatchedEvdArgs<T> a{};
        a.n = pl->d_n;
        a.A = (T* const*)pl->d_ptrs;
        a.lda = pl->d_lda;
        a.w = (T* const*)(pl->d_ptrs + B);
        a.Q = pl->vec ? (T* const*)(pl->d_ptrs + 2 * B) : nullptr;
        a.ldq = pl->d_ldq;
        a.info = info;
        a.queue = pl->d_queue;
        a.gscratch = (T*)pl->d_scratch;
        a.slot_elems = pl->slot_elems;
        a.smem_kmax = sh.smem_kmax;
        a.qtab = pl->d_qtab;
        a.tol = (T)pl->p.inner_tol;
        a.max_sweeps = pl->p.max_sweeps;
        a.cnt = pl->d_cnt;
        // the prefix of orders above the shared-memory size
        const size_t cap = device_smem_optin() - 4096;
        int nl = 0;
        if (pl->large_mode == 2 && pl->d_blk) {
            // blocked method for the largest orders; in FP64, where both are
            // bound by the FP64 pipe, orders up to 320 go to clusters (the
            // scalar method issues fewer operations there: measured on GB300,
            // 64 matrices of order 256 in 0.12 s on clusters, 0.20 s blocked;
            // order 384: 0.77 s / 0.69 s)
            const int blk_min = blk_min_of(sh, pl->esize);
            int nb = 0;
            while (nb < count) {
                const int n = pl->h_n[h_list[nb]], k = n + (n & 1);
                if (k <= sh.smem_kmax || k <= blk_min) break;
                ++nb;
            }
            if ((e = launch_batched_evd_blocked<T>(a, d_list, nb, pl->d_queue + 1, (T*)pl->d_blk, pl->blk_slot,
                                                   pl->blk_grid, s)) != cudaSuccess)
                return e;
            nl = nb;
            while (nl < count) {
                const int n = pl->h_n[h_list[nl]], k = n + (n & 1);
                if (k <= sh.smem_kmax || batched_cluster_size<T>(k, pl->vec, cap) == 0) break;
                ++nl;
            }
            for (int i = nb; i < nl;) {
                const int n0 = pl->h_n[h_list[i]];
                const int C = batched_cluster_size<T>(n0 + (n0 & 1), pl->vec, cap);
                int j = i + 1;
                while (j < nl) {
                    const int nj = pl->h_n[h_list[j]];
                    if (batched_cluster_size<T>(nj + (nj & 1), pl->vec, cap) != C) break;
                    ++j;
                }
                const int kmax = (n0 + C - 1) / C * C;
                if ((e = launch_batched_evd_cluster<T>(a, d_list + i, j - i, kmax, C, s)) != cudaSuccess) return e;
                i = j;
            }
        } else if (pl->large_mode == 1) {
            while (nl < count) {
                const int n = pl->h_n[h_list[nl]], k = n + (n & 1);
                if (k <= sh.smem_kmax) break;
                if (batched_cluster_size<T>(k, pl->vec, cap) == 0) {  // too large: all stay on L2 slots
                    nl = 0;
                    break;
                }
                ++nl;
            }
            for (int i = 0; i < nl;) {
                const int n0 = pl->h_n[h_list[i]];
                const int C = batched_cluster_size<T>(n0 + (n0 & 1), pl->vec, cap);
                int j = i + 1;
                while (j < nl) {
                    const int nj = pl->h_n[h_list[j]];
                    if (batched_cluster_size<T>(nj + (nj & 1), pl->vec, cap) != C) break;
                    ++j;
                }
                const int kmax = (n0 + C - 1) / C * C;
                if ((e = launch_batched_evd_cluster<T>(a, d_list + i, j - i, kmax, C, s)) != cudaSuccess) return e;
                i = j;
            }
        }
        a.batch = count - nl;
        a.order = d_list + nl;
        if (a.batch == 0) return cudaSuccess;
        return launch_batched_evd<T>(a, grid, sh.threads, s);
    }
    BatchedSvdArgs<T> a{};
    a.batch = count;
    a.order = d_list;
    a.m = pl->d_m;
    a.n = pl->d_n;
    a.G = (T* const*)pl->d_ptrs;
    a.ldg = pl->d_lda;
    a.sigma = (T* const*)(pl->d_ptrs + B);
    a.V = pl->vec ? (T* const*)(pl->d_ptrs + 2 * B) : nullptr;
    a.ldv = pl->d_ldq;
    a.info = info;
    a.queue = pl->d_queue;
    a.qtab = pl->d_qtab;
    int mmax = *std::max_element(pl->h_m.begin(), pl->h_m.end());
    const double ueps = pl->esize == 8 ? U64 : U32;
    a.tol = (T)std::max(pl->p.tol, sqrt((double)mmax) * ueps);
    a.max_sweeps = pl->p.max_sweeps;
    a.inner_max_sweeps = pl->p.inner_max_sweeps;
    a.cnt = pl->d_cnt;
    if (pl->svd_tiled) return launch_batched_svd_tiled<T>(a, pl->kmax, grid, sh.threads, s);
    return launch_batched_svd<T>(a, pl->kmax, grid, sh.threads, s);
}

cudaError_t plan_launch_any(jacobi_plan* pl, int* info, cudaStream_t s, const Shape& sh, int grid,
                            const std::vector<int>& h_list, const int* d_list)
{
    return pl->esize == 8 ? plan_launch<double>(pl, info, s, sh, grid, h_list, d_list)
                          : plan_launch<float>(pl, info, s, sh, grid, h_list, d_list);
}

template <typename T>
int occupancy_grid(jacobi_plan* pl, const Shape& sh)
{
    const int per_sm = pl->kind == 0 ? batched_evd_occupancy<T>(sh.threads, sh.smem_kmax, pl->vec)
                       : pl->svd_tiled ? batched_svd_tiled_occupancy<T>(sh.threads, pl->kmax)
                                       : batched_svd_occupancy<T>(sh.threads, pl->kmax);
    return device_sms() * std::max(1, std::min(per_sm, 4));
}

int grid_for(jacobi_plan* pl, const Shape& sh)
{
    return pl->esize == 8 ? occupancy_grid<double>(pl, sh) : occupancy_grid<float>(pl, sh);
}

}  // namespace

extern "C" void jacobi_plan_destroy(jacobi_plan* pl);

extern "C" int jacobi_plan_create_batched(jacobi_plan** out, int kind, int precision, int batch,
                                          const int* h_m, const int* h_n, const int* h_lda,
                                          const int* h_ldq, const jacobi_params* pin, void* stream)
{
    if (!out) return -1;
    *out = nullptr;
    if (kind != 0 && kind != 1) return -2;
    if (precision != JACOBI_PREC_FP64 && precision != JACOBI_PREC_FP32) return -3;
    if (batch < 1) return -4;
    if (kind == 1 && !h_m) return -5;
    if (!h_n) return -6;
    jacobi_params p;
    if (pin) p = *pin; else jacobi_params_default(&p);
    if (p.inner_max_sweeps == 0) p.inner_max_sweeps = 30;  // one-sided: full pivot solves
    if (p.max_sweeps < 1 || p.inner_max_sweeps < 1 || !(p.tol >= 0) || !(p.inner_tol >= 0)) return -10;
    cudaStream_t s = (cudaStream_t)stream;
    auto* pl = new jacobi_plan();
    pl->kind = kind;
    pl->precision = precision;
    pl->esize = precision == JACOBI_PREC_FP64 ? 8 : 4;
    pl->batch = batch;
    pl->vec = p.want_vectors != 0;
    pl->p = p;
    // JACOBI_BATCHED_LARGE = l2 | cluster | blocked (default) selects the
    // route of the orders above the shared-memory size
    if (const char* env = getenv("JACOBI_BATCHED_LARGE")) {
        if (!strcmp(env, "l2")) pl->large_mode = 0;
        else if (!strcmp(env, "cluster")) pl->large_mode = 1;
    }
    pl->svd_tiled = kind == 1;
    if (const char* env = getenv("JACOBI_BATCHED_SVD")) pl->svd_tiled = kind == 1 && strcmp(env, "rowwise") != 0;
    if (precision == JACOBI_PREC_FP32 && p.inner_tol == 4.0 * U64) pl->p.inner_tol = 4.0 * U32;
    pl->h_n.assign(h_n, h_n + batch);
    pl->h_m = kind == 1 ? std::vector<int>(h_m, h_m + batch) : pl->h_n;
    pl->h_lda.resize(batch);
    pl->h_ldq.resize(batch);
    for (int i = 0; i < batch; ++i) {
        const int n = pl->h_n[i], m = pl->h_m[i];
        if (n < 1 || n > kBatchedMaxK || m < n) { delete pl; return -6; }
        if ((long long)m * n > 0x7fffffffLL) { delete pl; return -5; }   // kernels index m x n in int
        pl->h_lda[i] = h_lda ? h_lda[i] : m;
        pl->h_ldq[i] = h_ldq ? h_ldq[i] : n;
        if (pl->h_lda[i] < m || (pl->vec && pl->h_ldq[i] < n)) { delete pl; return -7; }
        pl->kmax = std::max(pl->kmax, n + (n & 1));
    }
    if (kind == 1 && (precision == JACOBI_PREC_FP64 ? batched_svd_smem<double>(pl->kmax, 128)
                                                    : batched_svd_smem<float>(pl->kmax, 128)) > device_smem_optin()) {
        delete pl;
        return JACOBI_ERR_UNSUPPORTED;
    }
    // longest-processing-time order: largest work (m n^2 ~ n^3) first, stable
    pl->h_order.resize(batch);
    std::iota(pl->h_order.begin(), pl->h_order.end(), 0);
    std::stable_sort(pl->h_order.begin(), pl->h_order.end(), [&](int a, int b) {
        return (double)pl->h_m[a] * pl->h_n[a] * pl->h_n[a] > (double)pl->h_m[b] * pl->h_n[b] * pl->h_n[b];
    });
    // shape: tuned cache, else the default
    const std::string key = tune_key(kind, pl->esize, pl->vec, pl->h_n);
    bool tuned = false;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) { pl->shape = it->second; tuned = true; }
    }
    if (!tuned) {
        pl->shape = kind == 0 ? evd_default(pl->esize, pl->vec) : Shape{256, 0};
        if (kind == 1)
            while (pl->shape.threads > 128 &&
                   (pl->esize == 8 ? batched_svd_smem<double>(pl->kmax, pl->shape.threads)
                                   : batched_svd_smem<float>(pl->kmax, pl->shape.threads)) > device_smem_optin())
                pl->shape.threads /= 2;
    }
    // workspace
    auto fail = [&](int code) { jacobi_plan_destroy(pl); return code; };
    const int maxgrid = device_sms() * 4;
    pl->slot_elems = kind == 0 ? max_slot_elems(pl->kmax, pl->vec) : 0;
    if (cudaMalloc(&pl->d_order, sizeof(int) * batch) != cudaSuccess ||
        cudaMalloc(&pl->d_m, sizeof(int) * batch) != cudaSuccess ||
        cudaMalloc(&pl->d_n, sizeof(int) * batch) != cudaSuccess ||
        cudaMalloc(&pl->d_lda, sizeof(int) * batch) != cudaSuccess ||
        cudaMalloc(&pl->d_ldq, sizeof(int) * batch) != cudaSuccess ||
        cudaMalloc(&pl->d_ptrs, sizeof(void*) * 3 * batch) != cudaSuccess ||
        cudaMallocHost(&pl->h_ptrs, sizeof(void*) * 3 * batch) != cudaSuccess ||
        cudaMalloc(&pl->d_queue, 2 * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&pl->d_qtab, sizeof(unsigned) * (kBatchedMaxK / 2) * (kBatchedMaxK / 2 - 1) / 2) != cudaSuccess ||
        cudaMalloc(&pl->d_cnt, sizeof(DevCounters)) != cudaSuccess) {
        cudaGetLastError();
        return fail(JACOBI_ERR_ALLOC);
    }
    if (kind == 0 && cudaMalloc(&pl->d_scratch, pl->slot_elems * pl->esize * (size_t)maxgrid) != cudaSuccess) {
        cudaGetLastError();
        return fail(JACOBI_ERR_ALLOC);
    }
    if (kind == 0 && pl->large_mode == 2) {
        const int nmax = *std::max_element(pl->h_n.begin(), pl->h_n.end());
        pl->blk_slot = pl->esize == 8 ? batched_blocked_slot_elems<double>(nmax) : batched_blocked_slot_elems<float>(nmax);
        pl->blk_grid = device_sms() * (pl->esize == 8 ? batched_blocked_ctas_per_sm<double>() : batched_blocked_ctas_per_sm<float>());
        if (cudaMalloc(&pl->d_blk, pl->blk_slot * pl->esize * (size_t)pl->blk_grid) != cudaSuccess) {
            cudaGetLastError();
            return fail(JACOBI_ERR_ALLOC);
        }
    }
    memset(pl->h_ptrs, 0, sizeof(void*) * 3 * batch);
    if (cudaMemcpyAsync(pl->d_order, pl->h_order.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(pl->d_m, pl->h_m.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(pl->d_n, pl->h_n.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(pl->d_lda, pl->h_lda.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(pl->d_ldq, pl->h_ldq.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(pl->d_cnt, 0, sizeof(DevCounters), s) != cudaSuccess ||
        launch_quad_table(pl->d_qtab, kBatchedMaxK / 2, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(JACOBI_ERR_CUDA);
    pl->grid = std::min(grid_for(pl, pl->shape), maxgrid);
    *out = pl;
    return 0;
}

// Time every candidate shape on a sample of the batch (the matrices at evenly
// spaced positions of the longest-first order; their outputs are written and
// later overwritten) and keep the fastest in the cache.  The caller's pointer
// arrays must be given (as for execute).
extern "C" int jacobi_plan_autotune(jacobi_plan* pl, void* const* A_or_G, void* const* w_or_sigma,
                                    void* const* Q_or_V, int* info, void* stream)
{
    if (!pl || !A_or_G || !w_or_sigma || !info) return -1;
    if (pl->vec && !Q_or_V) return -4;
    cudaStream_t s = (cudaStream_t)stream;
    const int B = pl->batch;
    for (int i = 0; i < B; ++i) {
        pl->h_ptrs[i] = A_or_G[i];
        pl->h_ptrs[B + i] = w_or_sigma[i];
        pl->h_ptrs[2 * B + i] = pl->vec ? Q_or_V[i] : nullptr;
    }
    if (cudaMemcpyAsync(pl->d_ptrs, pl->h_ptrs, sizeof(void*) * 3 * B, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    const int sample = std::min(B, device_sms() * 2);
    std::vector<int> h_sub(sample);
    for (int i = 0; i < sample; ++i) h_sub[i] = pl->h_order[(size_t)i * B / sample];
    int* d_sub = nullptr;
    if (cudaMalloc(&d_sub, sizeof(int) * sample) != cudaSuccess) { cudaGetLastError(); return JACOBI_ERR_ALLOC; }
    cudaMemcpyAsync(d_sub, h_sub.data(), sizeof(int) * sample, cudaMemcpyHostToDevice, s);
    std::vector<Shape> cands;
    if (pl->kind == 0) {
        cands = pl->esize == 8 ? evd_candidates<double>(pl->vec) : evd_candidates<float>(pl->vec);
    } else {
        for (int th : {128, 256, 512})
            if ((pl->esize == 8 ? batched_svd_smem<double>(pl->kmax, th) : batched_svd_smem<float>(pl->kmax, th)) <= device_smem_optin())
                cands.push_back(Shape{th, 0});
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Shape bestsh = pl->shape;
    int rc = 0;
    for (const Shape& sh : cands) {
        const int grid = std::min(grid_for(pl, sh), device_sms() * 4);
        // warm, then time
        if (plan_launch_any(pl, info, s, sh, grid, h_sub, d_sub) != cudaSuccess) { cudaGetLastError(); continue; }
        cudaEventRecord(e0, s);
        if (plan_launch_any(pl, info, s, sh, grid, h_sub, d_sub) != cudaSuccess) { cudaGetLastError(); continue; }
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = JACOBI_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; bestsh = sh; }
    }
    // then the block size per size class: the order above which the blocked
    // method (b = 16) takes over from the unblocked solve on a cluster
    if (rc == 0 && pl->kind == 0 && pl->large_mode == 2 && pl->d_blk) {
        for (int bm : {0, 192, 256, 320, 384, 448, 512}) {
            Shape sh = bestsh;
            sh.blk_min = bm;
            const int grid = std::min(grid_for(pl, sh), device_sms() * 4);
            if (plan_launch_any(pl, info, s, sh, grid, h_sub, d_sub) != cudaSuccess) { cudaGetLastError(); continue; }
            cudaEventRecord(e0, s);
            if (plan_launch_any(pl, info, s, sh, grid, h_sub, d_sub) != cudaSuccess) { cudaGetLastError(); continue; }
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = JACOBI_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; bestsh = sh; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_sub);
    if (rc) return rc;
    pl->shape = bestsh;
    pl->grid = std::min(grid_for(pl, bestsh), device_sms() * 4);
    if (pl->exec) { cudaGraphExecDestroy(pl->exec); pl->exec = nullptr; }
    cudaMemsetAsync(pl->d_cnt, 0, sizeof(DevCounters), s);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune[tune_key(pl->kind, pl->esize, pl->vec, pl->h_n)] = bestsh;
        tune_store_locked();
    }
    return cudaStreamSynchronize(s) == cudaSuccess ? 0 : JACOBI_ERR_CUDA;
}

// Run the batch: the pointer arrays (host arrays of device pointers) are
// staged into pinned memory and uploaded by the first node of the plan's
// graph, followed by the queue reset and the persistent kernel.
extern "C" int jacobi_plan_execute(jacobi_plan* pl, void* const* A_or_G, void* const* w_or_sigma,
                                   void* const* Q_or_V, int* info, jacobi_stats* st, void* stream)
{
    if (!pl) return -1;
    if (!A_or_G) return -2;
    if (!w_or_sigma) return -3;
    if (pl->vec && !Q_or_V) return -4;
    if (!info) return -5;
    cudaStream_t s = (cudaStream_t)stream;
    const int B = pl->batch;
    // the graph reads h_ptrs: wait for the previous execute before rewriting it
    if (cudaStreamSynchronize(s) != cudaSuccess) return JACOBI_ERR_CUDA;
    for (int i = 0; i < B; ++i) {
        pl->h_ptrs[i] = A_or_G[i];
        pl->h_ptrs[B + i] = w_or_sigma[i];
        pl->h_ptrs[2 * B + i] = pl->vec ? Q_or_V[i] : nullptr;
    }
    if (pl->exec && pl->graph_info != info) {
        cudaGraphExecDestroy(pl->exec);
        pl->exec = nullptr;
    }
    if (!pl->exec) {
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return JACOBI_ERR_CUDA;
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
            ok = cudaMemcpyAsync(pl->d_ptrs, pl->h_ptrs, sizeof(void*) * 3 * B, cudaMemcpyHostToDevice, cs) == cudaSuccess &&
                 plan_launch_any(pl, info, cs, pl->shape, pl->grid, pl->h_order, pl->d_order) == cudaSuccess;
            ok = (cudaStreamEndCapture(cs, &g) == cudaSuccess) && ok && g;
        }
        if (ok) ok = cudaGraphInstantiate(&pl->exec, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        cudaGetLastError();
        if (!ok) {
            pl->exec = nullptr;
            return JACOBI_ERR_CUDA;
        }
        pl->graph_info = info;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    DevCounters hc;
    const bool ok = cudaMemsetAsync(pl->d_cnt, 0, sizeof(DevCounters), s) == cudaSuccess &&
                    cudaEventRecord(e0, s) == cudaSuccess && cudaGraphLaunch(pl->exec, s) == cudaSuccess &&
                    cudaEventRecord(e1, s) == cudaSuccess &&
                    cudaMemcpyAsync(&hc, pl->d_cnt, sizeof(hc), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                    cudaStreamSynchronize(s) == cudaSuccess;
    float ms = 0.f;
    if (ok) cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!ok) return JACOBI_ERR_CUDA;
    pl->last_ms = ms;
    if (st) {
        memset(st, 0, sizeof(*st));
        st->rotations = (long long)hc.rotations;
        st->inner_sweeps = (long long)hc.inner_sweeps;
        st->pair_solves = (long long)hc.pair_solves;
        st->flops_fp64 = (double)hc.flops_fp64;
        st->flops_fp32 = (double)hc.flops_fp32;
        st->ms_total = ms;
        st->ms_update = ms;
        st->launches = 1;
        st->update_launches = 1;
    }
    return 0;
}

extern "C" void jacobi_plan_destroy(jacobi_plan* pl)
{
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    cudaFree(pl->d_order);
    cudaFree(pl->d_m);
    cudaFree(pl->d_n);
    cudaFree(pl->d_lda);
    cudaFree(pl->d_ldq);
    cudaFree(pl->d_ptrs);
    if (pl->h_ptrs) cudaFreeHost(pl->h_ptrs);
    cudaFree(pl->d_queue);
    cudaFree(pl->d_qtab);
    cudaFree(pl->d_scratch);
    cudaFree(pl->d_blk);
    cudaFree(pl->d_cnt);
    delete pl;
}

extern "C" int jacobi_plan_blocking(const jacobi_plan* pl, int* b, int* min_order)
{
    if (!pl) return -1;
    if (pl->kind != 0 || pl->large_mode != 2 || !pl->d_blk) {   // no blocked route in this plan
        if (b) *b = 0;
        if (min_order) *min_order = 0;
        return 0;
    }
    if (b) *b = kBatchedBlockB;
    if (min_order) *min_order = std::max(blk_min_of(pl->shape, pl->esize), pl->shape.smem_kmax);
    return 0;
}

extern "C" int jacobi_plan_shape(const jacobi_plan* pl, int* threads, int* smem_kmax, int* grid)
{
    if (!pl) return -1;
    if (threads) *threads = pl->shape.threads;
    if (smem_kmax) *smem_kmax = pl->shape.smem_kmax;
    if (grid) *grid = pl->grid;
    return 0;
}

// ============================================================================ one-shot batched calls
static int batched_once(int kind, int precision, int batch, const int* h_m, const int* h_n,
                        void* const* X, const int* h_ldx, void* const* y, void* const* Z,
                        const int* h_ldz, const jacobi_params* p, int* info, jacobi_stats* st,
                        void* stream)
{
    jacobi_plan* pl = nullptr;
    int rc = jacobi_plan_create_batched(&pl, kind, precision, batch, h_m, h_n, h_ldx, h_ldz, p, stream);
    if (rc) return rc;
    rc = jacobi_plan_execute(pl, X, y, Z, info, st, stream);
    jacobi_plan_destroy(pl);
    return rc;
}

extern "C" int jacobi_syev_batched(int batch, const int* h_n, double* const* A, const int* h_lda,
                                   double* const* w, double* const* Q, const int* h_ldq,
                                   const jacobi_params* p, int* info, jacobi_stats* st, void* stream)
{
    return batched_once(0, JACOBI_PREC_FP64, batch, nullptr, h_n, (void* const*)A, h_lda,
                        (void* const*)w, (void* const*)Q, h_ldq, p, info, st, stream);
}

extern "C" int jacobi_syev_batched_f32(int batch, const int* h_n, float* const* A, const int* h_lda,
                                       float* const* w, float* const* Q, const int* h_ldq,
                                       const jacobi_params* p, int* info, jacobi_stats* st, void* stream)
{
    return batched_once(0, JACOBI_PREC_FP32, batch, nullptr, h_n, (void* const*)A, h_lda,
                        (void* const*)w, (void* const*)Q, h_ldq, p, info, st, stream);
}

extern "C" int jacobi_gesvd_batched_f32(int batch, const int* h_m, const int* h_n, float* const* G,
                                        const int* h_ldg, float* const* sigma, float* const* V,
                                        const int* h_ldv, const jacobi_params* p, int* info,
                                        jacobi_stats* st, void* stream)
{
    return batched_once(1, JACOBI_PREC_FP32, batch, h_m, h_n, (void* const*)G, h_ldg,
                        (void* const*)sigma, (void* const*)V, h_ldv, p, info, st, stream);
}
