// api_mixed.cu -- the mixed-precision two-sided driver.
//
// Phase 1 (low precision): the working A_w and Q_w are FP32.  Each step runs
// the FP64 pivot solves on the promoted 2b x 2b blocks (the pivot kernels
// read and write the FP32 copies) and the block updates on the tensor cores
// (bf16 hi/lo splits, three products, FP32 accumulation in TMEM).  Sweeps
// continue until off(A_w) <= switch_tol ||A||_F, or off(A_w) stops falling.
//
// Phase 2 (return to FP64): the low-precision updates perturb A_w by about
// 2^-17 ||A|| per step, so A_w itself is never finished in FP64.  Instead
// X = fl64(Q_w) is refined against the original A0:
//   - refine_steps steps of Ogita and Aishima (2018): G = X^T X, W = A0 X,
//     S = X^T W, E from (S, G) (k_oa_correction), X <- X + X E;
//   - Newton-Schulz steps X <- X + X (I - X^T X) / 2 until ||I - X^T X||_F
//     is at the FP64 rounding level;
//   - S = X^T A0 X, symmetrised.
// Phase 3: FP64 closing sweeps (the plain FP64 driver) on S with the warm
// start Q = X, then the usual finalisation.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <utility>

#include "host.h"

namespace jac {

namespace {

constexpr double U32 = 5.9604644775390625e-08;  // 2^-24

struct LowpState {
    int np, b, k, n_real;
    int pcl = 1;
    const unsigned* qtab = nullptr;
    const Ordering* ord;
    const int2* dpairs;
    float* Aw[2];
    float* Qw[2];
    float* T;
    unsigned char* vimg;
    unsigned* tmax;
    int kind;
    double* Vb;
    int* rot;
    double* gscratch;
    double* qrws = nullptr;   // pivot_order == 2: the QRCP scratch
    double* partial;
    unsigned* ticket;
    double* result;
    int* err;
    DevCounters* cnt;
};

cudaError_t launch_step32(const LowpState& L, int s, int cur, cudaStream_t cs, double inner_tol,
                          int inner_max, int order, cudaEvent_t mid)
{
    const int nps = L.ord->dev_per_step, p0 = s * nps;
    PivotArgs pa{};
    pa.Ain32 = L.Aw[cur];
    pa.Aout32 = L.Aw[cur ^ 1];
    pa.ld = L.np;
    pa.pairs = L.dpairs + p0;
    pa.npairs = nps;
    pa.b = L.b;
    pa.k = L.k;
    pa.V = L.Vb;
    pa.v32 = 1;   // V only feeds the split products, which take it rounded to FP32
    pa.rot = L.rot;
    pa.tol_rel = inner_tol;
    pa.max_sweeps = inner_max;
    pa.order = order;
    pa.n_real = L.n_real;
    pa.gscratch = L.gscratch;
    pa.qrws = L.qrws;
    pa.cnt = L.cnt;
    cudaError_t e = L.pcl > 1 ? launch_pivot_cluster(pa, L.pcl, L.qtab, cs) : launch_pivot(pa, cs);
    if (e != cudaSuccess) return e;
    if (mid && (e = cudaEventRecordWithFlags(mid, cs, cudaEventRecordExternal)) != cudaSuccess) return e;
    TcUpdArgs ua{};
    ua.Ain = L.Aw[cur];
    ua.Aout = L.Aw[cur ^ 1];
    ua.lda = L.np;
    ua.Qin = L.Qw[cur];
    ua.Qout = L.Qw[cur ^ 1];
    ua.ldq = L.np;
    ua.qrows = L.np;
    ua.T = L.T;
    ua.vimg = L.vimg;
    ua.tmax = L.tmax;
    ua.kind = L.kind;
    ua.pairs = L.dpairs + p0;
    ua.npairs = nps;
    ua.b = L.b;
    ua.k = L.k;
    ua.V = L.Vb;
    ua.rot = L.rot;
    ua.err = L.err;
    ua.cnt = L.cnt;
    return launch_tc_update(ua, cs);
}

// Low-precision sweeps until off(A_w) <= target or it stalls.  Returns the
// sweep count (>= 0) or a negative status.
int run_lowp_sweeps(LowpState& L, const jacobi_params& p, int& cur, double target,
                    jacobi_stats* st, cudaStream_t s)
{
    SweepGraph graphs[2];
    bool tried[2] = {false, false}, have[2] = {false, false};
    PhaseEvents pe(2 * (size_t)L.ord->S + 1);
    // A rotation whose a_pq is below the FP32 rounding of the pivot's diagonal
    // changes nothing the FP32 working copy can hold: skip it in this phase.
    const double inner_tol = p.inner_tol > U32 ? p.inner_tol : U32;
    double prev = INFINITY;
    int sw = 0;
    for (; sw < p.max_sweeps; ++sw) {
        const int start = cur;
        auto body = [&](cudaStream_t cs) -> bool {
            int c = start;
            if (cudaEventRecordWithFlags(pe.ev[0], cs, cudaEventRecordExternal) != cudaSuccess) return false;
            for (int si = 0; si < L.ord->S; ++si) {
                if (launch_step32(L, si, c, cs, inner_tol, p.inner_max_sweeps, p.pivot_order,
                                  pe.ev[2 * si + 1]) != cudaSuccess)
                    return false;
                if (cudaEventRecordWithFlags(pe.ev[2 * si + 2], cs, cudaEventRecordExternal) != cudaSuccess)
                    return false;
                c ^= 1;
            }
            return launch_offnorm32(L.np, L.Aw[c], L.partial, L.ticket, L.result, cs) == cudaSuccess;
        };
        if (!tried[start]) {
            tried[start] = true;
            have[start] = capture(graphs[start], body);
        }
        if (have[start]) {
            if (cudaGraphLaunch(graphs[start].exec, s) != cudaSuccess) return JACOBI_ERR_CUDA;
        } else if (!body(s)) {
            return JACOBI_ERR_CUDA;
        }
        cur = start ^ (L.ord->S & 1);
        double h_res[3];
        int h_err = 0;
        if (cudaMemcpyAsync(h_res, L.result, sizeof(h_res), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&h_err, L.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (h_err) return JACOBI_ERR_TIMEOUT;
        st->steps += L.ord->S;
        for (int si = 0; si < L.ord->S; ++si) {
            const double tp = pe.ms(2 * si, 2 * si + 1), tu = pe.ms(2 * si + 1, 2 * si + 2);
            st->ms_pivot += tp;
            st->ms_update += tu;
            st->ms_pivot_lowp += tp;
            st->ms_update_lowp += tu;
        }
        // pivot, V split and two tensor-core stages per step, one off-norm per sweep
        st->launches += 4 * L.ord->S + 1;
        st->pivot_launches += L.ord->S;
        st->update_launches += 3 * L.ord->S;
        const double off = sqrt(h_res[0]);
        if (sw < 64) st->off_hist[sw] = off;
        st->off_final = off;
        if (!isfinite(off)) return JACOBI_ERR_NONFINITE;
        if (off <= target) return sw + 1;
        // no longer converging at this precision
        if (off > 0.9 * prev || (off <= 100.0 * target && off > 0.5 * prev)) return sw + 1;
        prev = off;
    }
    return sw;
}

}  // namespace

int syev_mixed(int n, double* A, int lda, double* w, double* Q, int ldq, const jacobi_params& pin,
               jacobi_stats* st, cudaStream_t s)
{
    if (pin.precision != JACOBI_PREC_MIXED_BF16X3 && pin.precision != JACOBI_PREC_MIXED_FP16X3 &&
        pin.precision != JACOBI_PREC_MIXED_TF32)
        return JACOBI_ERR_UNSUPPORTED;
    if (pin.warm_start) return JACOBI_ERR_UNSUPPORTED;
    jacobi_params p = pin;
    if (p.refine_steps < 0 || p.refine_steps > 8 || !(p.switch_tol >= 0.0)) return -7;
    Timer timer(s);
    const int N = padded_blocks(n, p.b, p.ordering);
    Ordering ord;
    if (!make_ordering(p.ordering, N, &ord)) return -7;
    const int np = N * p.b, k = 2 * p.b;
    const size_t np2 = (size_t)np * np;
    const bool vec = p.want_vectors != 0;
    const double switch_tol = p.switch_tol > 0.0 ? p.switch_tol : 64.0 * U32 * sqrt((double)n);
    int rc = 0;
    Workspace ws(s);
    EvdState E{};
    E.np = np;
    E.b = p.b;
    E.k = k;
    E.n_real = n;
    E.ord = ord;
    LowpState L{};
    L.np = np;
    L.b = p.b;
    L.k = k;
    L.n_real = n;
    L.ord = &E.ord;
    // FP64 state (closing sweeps and refinement)
    E.Aw[0] = ws.get<double>(np2);
    E.Aw[1] = ws.get<double>(np2);
    E.Qw[0] = ws.get<double>(np2);
    E.Qw[1] = ws.get<double>(np2);
    double* A0p = ws.get<double>(np2);
    double* lam = ws.get<double>(np);
    E.Vb = ws.get<double>((size_t)E.ord.max_pairs * 2 * k * k);
    E.rot = ws.get<int>(E.ord.max_pairs);
    const size_t gsz = pivot_gscratch_doubles(k);
    E.gscratch = gsz ? ws.get<double>(gsz * E.ord.max_pairs) : nullptr;
    E.dpairs = ws.get<int2>(E.ord.dev_pairs.size() / 2);
    E.partial = ws.get<double>(3 * (size_t)reduce_blocks_for(np));
    E.ticket = ws.get<unsigned>(1);
    E.result = ws.get<double>(3);
    E.cnt = ws.get<DevCounters>(1);
    int* rank = ws.get<int>(n);
    E.pcl = choose_pivot_cluster(k, E.ord.dev_per_step);
    E.qtab = E.pcl > 1 ? ws.get<unsigned>(128 * 127 / 2) : nullptr;
    if (p.pivot_order == 2) E.qrws = ws.get<double>((size_t)E.ord.max_pairs * p.b * k);
    // FP32 state (low-precision sweeps); pivot scratch shared with E
    L.Aw[0] = ws.get<float>(np2);
    L.Aw[1] = ws.get<float>(np2);
    L.Qw[0] = ws.get<float>(np2);
    L.Qw[1] = ws.get<float>(np2);
    L.T = ws.get<float>(tc_update_tbuf_floats(E.ord.dev_per_step, k));
    L.vimg = ws.get<unsigned char>(tc_update_vimg_bytes(E.ord.dev_per_step, k));
    L.tmax = ws.get<unsigned>(tc_update_tmax_words(E.ord.dev_per_step, k));
    L.kind = p.precision == JACOBI_PREC_MIXED_FP16X3 ? 1 : (p.precision == JACOBI_PREC_MIXED_TF32 ? 2 : 0);
    L.err = ws.get<int>(1);
    int* xexp = nullptr;          // line exponents of the emulated refinement products
    unsigned char* gimg[2] = {nullptr, nullptr};   // their slice images
    if (p.fp64_products == 1) {   // refinement and closing sweeps with FP64-accurate tensor-core products
        E.T64 = ws.get<double>(emu_update_tbuf_doubles(E.ord.dev_per_step, k));
        E.err = L.err;
        if (emu_image_wanted()) {
            E.vimg = ws.get<unsigned char>(emu_update_vimg_bytes(E.ord.dev_per_step, k));
            E.vexp = ws.get<int>(emu_update_vexp_ints(E.ord.dev_per_step, k));
            if (p.conv != JACOBI_CONV_REL) {   // (balanced products slice per tile)
                E.aimg = ws.get<unsigned char>(emu_update_aimg_bytes(E.ord.dev_per_step, k));
                E.atab = ws.get<int>((size_t)E.ord.dev_per_step * np);
                E.qimg = ws.get<unsigned char>(emu_update_qimg_bytes(E.ord.dev_per_step, k, np));
                E.qexp = ws.get<int>((size_t)E.ord.dev_per_step * np);
            }
        }
        E.balance = p.conv == JACOBI_CONV_REL;
        xexp = ws.get<int>(2 * (size_t)np);
        if (emu_image_wanted()) {   // the refinement products' operands sliced once per product
            gimg[0] = ws.get<unsigned char>(emu_gemm_img_bytes(np, np));
            gimg[1] = ws.get<unsigned char>(emu_gemm_img_bytes(np, np));
        }
    }
    if (ws.failed) return JACOBI_ERR_ALLOC;
    L.pcl = E.pcl;
    L.qtab = E.qtab;
    L.dpairs = E.dpairs;
    L.Vb = E.Vb;
    L.rot = E.rot;
    L.gscratch = E.gscratch;
    L.qrws = E.qrws;
    L.partial = E.partial;
    L.ticket = E.ticket;
    L.result = E.result;
    L.cnt = E.cnt;

    if (E.qtab && launch_quad_table(E.qtab, 128, s) != cudaSuccess) return JACOBI_ERR_CUDA;
    if (cudaMemcpyAsync(E.dpairs, E.ord.dev_pairs.data(), E.ord.dev_pairs.size() * sizeof(int),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(E.cnt, 0, sizeof(DevCounters), s) != cudaSuccess ||
        cudaMemsetAsync(E.ticket, 0, sizeof(unsigned), s) != cudaSuccess ||
        cudaMemsetAsync(L.err, 0, sizeof(int), s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    // A0 (FP64, padded) for ||A||_F and the refinement; A_w, Q_w (FP32)
    if (launch_pad_sym64(n, np, A, lda, A0p, s) != cudaSuccess ||
        launch_load_sym32(n, np, A, lda, L.Aw[0], L.Qw[0], E.cnt, s) != cudaSuccess ||
        launch_offnorm(np, A0p, E.partial, E.ticket, E.result, p.conv == JACOBI_CONV_REL, s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    st->launches += 3;
    double h_res[3];
    DevCounters hc;
    if (cudaMemcpyAsync(h_res, E.result, sizeof(h_res), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&hc, E.cnt, sizeof(hc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    if (hc.nonfinite) return JACOBI_ERR_NONFINITE;
    st->norm_fro = sqrt(h_res[1]);
    st->off_initial = sqrt(h_res[0]);
    st->off_final = st->off_initial;
    const bool rel = p.conv == JACOBI_CONV_REL;
    const double target = rel ? p.tol : p.tol * st->norm_fro;
    const double meas0 = rel ? h_res[2] : st->off_initial;

    int cur = 0;        // FP64 buffers holding (S, X)
    int sweeps_low = 0, sweeps_hi = 0;
    if (meas0 > target) {
        // ---------------------------------------------------------------- phase 1
        cudaEvent_t ev[2];
        cudaEventCreate(&ev[0]);
        cudaEventCreate(&ev[1]);
        cudaEventRecord(ev[0], s);
        int c32 = 0;
        const int r = run_lowp_sweeps(L, p, c32, switch_tol * st->norm_fro, st, s);
        if (r < 0) {
            cudaEventDestroy(ev[0]);
            cudaEventDestroy(ev[1]);
            return r;
        }
        sweeps_low = r;
        cudaEventRecord(ev[1], s);
        // ---------------------------------------------------------------- phase 2
        double* X = E.Qw[0];
        double* Xn = E.Qw[1];
        double* G = E.Aw[0];
        double* W = E.Aw[1];
        bool ok = launch_f32_to_f64((long long)np2, L.Qw[c32], X, s) == cudaSuccess;
        st->launches += 1;
        const double nn = (double)np, n3 = nn * nn * nn;
        // C = op(Am) Bm (+ C when acc): FP64 FMA, or FP64-accurate on the tensor cores
        auto g64 = [&](const double* Am, int transA, const double* Bm, int acc, double* Cm, int lower) {
            if (xexp && gimg[0])
                return launch_emu_gemm_img(np, np, np, Am, np, transA, Bm, np, acc, Cm, np, lower, xexp, xexp + np,
                                           gimg[0], gimg[1], L.err, s) == cudaSuccess;
            if (xexp)
                return launch_emu_gemm_big(np, np, np, Am, np, transA, Bm, np, acc, Cm, np, lower, xexp, xexp + np,
                                           L.err, s) == cudaSuccess;
            return launch_gemm64(np, np, np, 1.0, Am, np, transA, Bm, np, acc ? 1.0 : 0.0, Cm, np, s, lower) ==
                   cudaSuccess;
        };
        // X^T B for a symmetric result: the tiles meeting the lower triangle,
        // then mirrored (about half the flops of the full product)
        auto sym_xtb = [&](const double* B, double* out) {
            return g64(X, 1, B, 0, out, 1) && launch_mirror_lower(np, out, np, s) == cudaSuccess;
        };
        const double sym_flops = n3 + 2.0 * nn * nn * 128.0;  // lower tiles incl. the diagonal band
        double fl = 0.0;
        for (int it = 0; ok && it < p.refine_steps; ++it) {
            ok = sym_xtb(X, G) &&
                 g64(A0p, 0, X, 0, W, 0) &&
                 sym_xtb(W, Xn) &&
                 // Xn holds S now; E overwrites G
                 launch_oa_step_elementwise(np, Xn, G, lam, 1e-2, s) == cudaSuccess &&
                 cudaMemcpyAsync(Xn, X, np2 * sizeof(double), cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
                 g64(X, 0, G, 1, Xn, 0);
            std::swap(X, Xn);
            fl += 2.0 * sym_flops + 4.0 * n3;
            st->launches += 8;
        }
        // Newton-Schulz, X <- X + X (I - X^T X) / 2, until ||I - X^T X||_F
        // reaches the rounding level.  A step maps r = ||I - X^T X|| to about
        // 3 r^2 / 4, so once that prediction is below the goal the step is
        // taken without forming X^T X again.
        const double orth_goal = 8.0 * U64 * sqrt(nn);
        for (int it = 0; ok && it < 4; ++it) {
            ok = sym_xtb(X, G) && launch_ns_halfres(np, G, s) == cudaSuccess &&
                 launch_offnorm(np, G, E.partial, E.ticket, E.result, false, s) == cudaSuccess &&
                 cudaMemcpyAsync(h_res, E.result, sizeof(h_res), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                 cudaStreamSynchronize(s) == cudaSuccess;
            fl += sym_flops;
            st->launches += 4;
            if (!ok) break;
            const double rnorm = 2.0 * sqrt(h_res[1]);
            if (!isfinite(rnorm)) {
                ok = false;
                break;
            }
            if (rnorm <= orth_goal) break;
            ok = cudaMemcpyAsync(Xn, X, np2 * sizeof(double), cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
                 g64(X, 0, G, 1, Xn, 0);
            std::swap(X, Xn);
            fl += 2.0 * n3;
            st->launches += 1;
            if (0.75 * rnorm * rnorm <= 0.5 * orth_goal) break;
        }
        // S = X^T A0 X into the A buffer paired with X (its lower tiles, mirrored)
        cur = X == E.Qw[0] ? 0 : 1;
        double* Wt = E.Aw[cur ^ 1];
        ok = ok && g64(A0p, 0, X, 0, Wt, 0) && sym_xtb(Wt, E.Aw[cur]);
        fl += 2.0 * n3 + sym_flops;
        st->launches += 3;
        st->flops_fp64 += fl;
        st->flops_refine += fl;
        cudaEvent_t ev2;
        cudaEventCreate(&ev2);
        cudaEventRecord(ev2, s);
        if (!ok || cudaStreamSynchronize(s) != cudaSuccess) {
            cudaEventDestroy(ev[0]);
            cudaEventDestroy(ev[1]);
            cudaEventDestroy(ev2);
            return JACOBI_ERR_CUDA;
        }
        float t1 = 0.f, t2 = 0.f;
        cudaEventElapsedTime(&t1, ev[0], ev[1]);
        cudaEventElapsedTime(&t2, ev[1], ev2);
        st->ms_lowp = t1;
        st->ms_refine = t2;
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        cudaEventDestroy(ev2);
        // ---------------------------------------------------------------- phase 3
        if (launch_offnorm(np, E.Aw[cur], E.partial, E.ticket, E.result, rel, s) != cudaSuccess ||
            cudaMemcpyAsync(h_res, E.result, sizeof(h_res), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        st->launches += 1;
        const double m1 = rel ? h_res[2] : sqrt(h_res[0]);
        st->off_final = sqrt(h_res[0]);
        if (m1 > target) {
            jacobi_params p2 = p;
            p2.max_sweeps = sweeps_low + p.max_sweeps;
            SweepResult res = run_evd_sweeps(E, p2, cur, target, sweeps_low, st, s, rel);
            if (res.code < 0) return res.code;
            sweeps_hi = res.sweeps - sweeps_low;
            rc = res.code == 0 ? 0 : sweeps_low + sweeps_hi;
        }
    } else {
        // already diagonal to the tolerance: finish from A0 and Q = I
        if (launch_load_sym(n, np, A, lda, E.Aw[0], nullptr, 0, E.Qw[0], 0, E.cnt, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        st->launches += 1;
    }
    st->sweeps = sweeps_low + sweeps_hi;
    st->sweeps_lowp = sweeps_low;
    if (launch_finalize_evd(n, np, E.Aw[cur], vec ? E.Qw[cur] : nullptr, w, vec ? Q : nullptr, ldq, A,
                            lda, rank, s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    st->launches += 2;
    int h_err = 0;
    if (cudaMemcpyAsync(&hc, E.cnt, sizeof(hc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&h_err, L.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    if (h_err) return JACOBI_ERR_TIMEOUT;
    const double host_fp64 = st->flops_fp64;
    fill_counters(st, hc);
    st->flops_fp64 += host_fp64;
    st->ms_total = timer.stop();
    return rc;
}

}  // namespace jac

using namespace jac;

extern "C" int jacobi_syev_step_lowp(int np, float* A, int lda, float* Q, int ldq,
                                     const jacobi_params* pin, int step, void* stream)
{
    jacobi_params p;
    if (pin) p = *pin; else jacobi_params_default(&p);
    int e = check_params(p);
    if (e) return e == -7 ? -6 : e;
    if (p.precision != JACOBI_PREC_MIXED_BF16X3 && p.precision != JACOBI_PREC_MIXED_FP16X3 &&
        p.precision != JACOBI_PREC_MIXED_TF32)
        return JACOBI_ERR_UNSUPPORTED;
    if (p.inner_max_sweeps == 0) p.inner_max_sweeps = 1;
    if (np < 2 * p.b || np % p.b || (np / p.b) % 2) return -1;
    if (!A) return -2;
    if (lda < np) return -3;
    if (Q && ldq < np) return -5;
    cudaStream_t s = (cudaStream_t)stream;
    Ordering ord;
    if (!make_ordering(p.ordering, np / p.b, &ord)) return -1;
    if (step < 0 || step >= ord.S) return -7;
    const int k = 2 * p.b;
    const size_t np2 = (size_t)np * np;
    Workspace ws(s);
    LowpState L{};
    L.np = np;
    L.b = p.b;
    L.k = k;
    L.n_real = np;
    L.ord = &ord;
    L.Aw[0] = ws.get<float>(np2);
    L.Aw[1] = ws.get<float>(np2);
    L.Qw[0] = ws.get<float>(np2);
    L.Qw[1] = ws.get<float>(np2);
    L.T = ws.get<float>(tc_update_tbuf_floats(ord.dev_per_step, k));
    L.vimg = ws.get<unsigned char>(tc_update_vimg_bytes(ord.dev_per_step, k));
    L.tmax = ws.get<unsigned>(tc_update_tmax_words(ord.dev_per_step, k));
    L.kind = p.precision == JACOBI_PREC_MIXED_FP16X3 ? 1 : (p.precision == JACOBI_PREC_MIXED_TF32 ? 2 : 0);
    L.Vb = ws.get<double>((size_t)ord.max_pairs * 2 * k * k);
    L.rot = ws.get<int>(ord.max_pairs);
    const size_t gsz = pivot_gscratch_doubles(k);
    L.gscratch = gsz ? ws.get<double>(gsz * ord.max_pairs) : nullptr;
    L.qrws = p.pivot_order == 2 ? ws.get<double>((size_t)ord.max_pairs * p.b * k) : nullptr;
    int2* dpairs = ws.get<int2>(ord.dev_pairs.size() / 2);
    L.dpairs = dpairs;
    L.err = ws.get<int>(1);
    L.cnt = ws.get<DevCounters>(1);
    L.pcl = choose_pivot_cluster(k, ord.dev_per_step);
    unsigned* qtab = L.pcl > 1 ? ws.get<unsigned>(128 * 127 / 2) : nullptr;
    L.qtab = qtab;
    if (ws.failed) return JACOBI_ERR_ALLOC;
    if (qtab && launch_quad_table(qtab, 128, s) != cudaSuccess) return JACOBI_ERR_CUDA;
    const size_t row = (size_t)np * sizeof(float);
    if (cudaMemcpyAsync(dpairs, ord.dev_pairs.data(), ord.dev_pairs.size() * sizeof(int),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(L.cnt, 0, sizeof(DevCounters), s) != cudaSuccess ||
        cudaMemsetAsync(L.err, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemcpy2DAsync(L.Aw[0], row, A, (size_t)lda * 4, row, np, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpy2DAsync(L.Aw[1], row, A, (size_t)lda * 4, row, np, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    if (Q) {
        if (cudaMemcpy2DAsync(L.Qw[0], row, Q, (size_t)ldq * 4, row, np, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
    } else {
        L.Qw[0] = L.Qw[1] = nullptr;
    }
    if (launch_step32(L, step, 0, s, p.inner_tol, p.inner_max_sweeps, p.pivot_order, nullptr) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    int h_err = 0;
    if (cudaMemcpy2DAsync(A, (size_t)lda * 4, L.Aw[1], row, row, np, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        (Q && cudaMemcpy2DAsync(Q, (size_t)ldq * 4, L.Qw[1], row, row, np, cudaMemcpyDeviceToDevice, s) != cudaSuccess) ||
        cudaMemcpyAsync(&h_err, L.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    return h_err ? JACOBI_ERR_TIMEOUT : 0;
}
