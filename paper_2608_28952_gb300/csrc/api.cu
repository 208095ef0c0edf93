// api.cu -- C ABI entry points and the host-side sweep driver.
//
// A call validates its arguments, builds the pair schedule (round-robin or
// Algorithm 3), allocates its workspace stream-ordered, and runs sweeps until
// the stop test passes.  One sweep is a sequence of parallel steps; a step
// launches the pivot kernel (all 2b x 2b solves of the step, one CTA per pair)
// and the update kernel (all block-row/column updates of the step, Algorithm
// 2).  A sweep's launches are captured once into a CUDA graph and replayed;
// the only device->host traffic per sweep is the stop statistic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "host.h"

using namespace jac;


extern "C" int jacobi_params_default(jacobi_params* p)
{
    if (!p) return -1;
    memset(p, 0, sizeof(*p));
    p->b = 32;
    p->ordering = JACOBI_ORDER_ROUND_ROBIN;
    p->max_sweeps = 60;
    p->inner_max_sweeps = 0;
    p->tol = 1e-14;
    p->inner_tol = 4.0 * U64;
    p->precision = JACOBI_PREC_FP64;
    p->conv = JACOBI_CONV_OFF_ABS;
    p->want_vectors = 1;
    p->warm_start = 0;
    p->switch_tol = 0.0;
    p->refine_steps = 1;
    p->pivot_order = 1;
    return 0;
}

extern "C" const char* jacobi_status_string(int status)
{
    if (status == 0) return "converged";
    if (status > 0) return "not converged within max_sweeps";
    switch (status) {
        case JACOBI_ERR_NONFINITE: return "non-finite input";
        case JACOBI_ERR_CUDA: return "CUDA runtime error";
        case JACOBI_ERR_ALLOC: return "workspace allocation failed";
        case JACOBI_ERR_TIMEOUT: return "bounded device wait ran out";
        case JACOBI_ERR_UNSUPPORTED: return "unsupported argument combination";
        default: return "invalid argument";
    }
}

// ============================================================================ EVD (FP64)
namespace jac {

static cudaError_t launch_step(EvdState& E, int s, int cur, cudaStream_t cs, double inner_tol,
                               int inner_max, int order, cudaEvent_t mid = nullptr)
{
    const int np_s = E.ord.dev_per_step, p0 = s * np_s;
    PivotArgs pa{};
    pa.Ain = E.Aw[cur];
    pa.Aout = E.Aw[cur ^ 1];
    pa.ld = E.np;
    pa.gram = nullptr;
    pa.npanels = 0;
    pa.pairs = E.dpairs + p0;
    pa.npairs = np_s;
    pa.b = E.b;
    pa.k = E.k;
    pa.V = E.Vb;
    pa.rot = E.rot;
    pa.relmax = nullptr;
    pa.tol_rel = inner_tol;
    pa.max_sweeps = inner_max;
    pa.order = order;
    pa.n_real = E.n_real;
    pa.gscratch = E.gscratch;
    pa.qrws = E.qrws;
    pa.cnt = E.cnt;
    cudaError_t e = E.pcl > 1 ? launch_pivot_cluster(pa, E.pcl, E.qtab, cs) : launch_pivot(pa, cs);
    if (e != cudaSuccess) return e;
    if (mid && (e = cudaEventRecordWithFlags(mid, cs, cudaEventRecordExternal)) != cudaSuccess) return e;
    UpdateArgs ua{};
    ua.Ain = E.Aw[cur];
    ua.Aout = E.Aw[cur ^ 1];
    ua.lda = E.np;
    ua.Qin = E.Qw[cur];
    ua.Qout = E.Qw[cur ^ 1];
    ua.ldq = E.np;
    ua.qrows = E.np;
    ua.pairs = E.dpairs + p0;
    ua.npairs = np_s;
    ua.b = E.b;
    ua.k = E.k;
    ua.V = E.Vb;
    ua.rot = E.rot;
    ua.cnt = E.cnt;
    if (E.T64) {
        EmuUpdArgs ea{ua, E.T64, E.err, E.balance, E.vimg, E.vexp, E.aimg, E.atab, E.qimg, E.qexp};
        return launch_emu_update(ea, cs);
    }
    return launch_update_evd(ua, cs);
}

SweepResult run_evd_sweeps(EvdState& E, const jacobi_params& p, int& cur, double target,
                           int sweep0, jacobi_stats* st, cudaStream_t s, bool use_rel)
{
    SweepGraph graphs[2];
    bool tried[2] = {false, false}, have[2] = {false, false};
    double h_res[3];
    double prev = INFINITY;
    int sw = sweep0;
    PhaseEvents pe(2 * (size_t)E.ord.S + 1);
    for (; sw < p.max_sweeps; ++sw) {
        const int start = cur;
        auto body = [&](cudaStream_t cs) -> bool {
            int c = start;
            if (cudaEventRecordWithFlags(pe.ev[0], cs, cudaEventRecordExternal) != cudaSuccess) return false;
            for (int si = 0; si < E.ord.S; ++si) {
                if (launch_step(E, si, c, cs, p.inner_tol, p.inner_max_sweeps, p.pivot_order,
                                pe.ev[2 * si + 1]) != cudaSuccess)
                    return false;
                if (cudaEventRecordWithFlags(pe.ev[2 * si + 2], cs, cudaEventRecordExternal) != cudaSuccess) return false;
                c ^= 1;
            }
            return launch_offnorm(E.np, E.Aw[c], E.partial, E.ticket, E.result, use_rel, cs) ==
                   cudaSuccess;
        };
        if (!tried[start]) {
            tried[start] = true;
            have[start] = capture(graphs[start], body);
        }
        if (have[start]) {
                if (cudaGraphLaunch(graphs[start].exec, s) != cudaSuccess) return {JACOBI_ERR_CUDA, sw};
        } else if (!body(s)) {
            return {JACOBI_ERR_CUDA, sw};
        }
        cur = start ^ (E.ord.S & 1);
        if (cudaMemcpyAsync(h_res, E.result, sizeof(h_res), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return {JACOBI_ERR_CUDA, sw};
        st->steps += E.ord.S;
        for (int si = 0; si < E.ord.S; ++si) {
            st->ms_pivot += pe.ms(2 * si, 2 * si + 1);
            st->ms_update += pe.ms(2 * si + 1, 2 * si + 2);
        }
        st->launches += 2 * E.ord.S + 1;
        st->pivot_launches += E.ord.S;
        st->update_launches += E.ord.S;
        const double off = sqrt(h_res[0]);
        const double meas = use_rel ? h_res[2] : off;
        if (sw < 64) {
            st->off_hist[sw] = off;
            st->rel_hist[sw] = use_rel ? h_res[2] : 0.0;
        }
        st->off_final = off;
        st->rel_final = use_rel ? h_res[2] : 0.0;
        if (meas <= target) return {0, sw + 1};
        if (meas <= 100.0 * target && meas > 0.5 * prev) {
            st->stalled = 1;
            return {0, sw + 1};
        }
        prev = meas;
    }
    return {1, sw};
}

}  // namespace jac

static int syev_fp64(int n, double* A, int lda, double* w, double* Q, int ldq,
                     const jacobi_params& p, jacobi_stats* st, cudaStream_t s)
{
    Timer timer(s);
    EvdState E{};
    E.b = p.b;
    E.k = 2 * p.b;
    E.n_real = n;
    const int N = padded_blocks(n, p.b, p.ordering);
    E.np = N * p.b;
    if (!make_ordering(p.ordering, N, &E.ord)) return -7;
    const bool vec = p.want_vectors != 0;
    const size_t np2 = (size_t)E.np * E.np;
    int rc = 0;
    {
        Workspace ws(s);
        E.Aw[0] = ws.get<double>(np2);
        E.Aw[1] = ws.get<double>(np2);
        E.Qw[0] = vec ? ws.get<double>(np2) : nullptr;
        E.Qw[1] = vec ? ws.get<double>(np2) : nullptr;
        E.Vb = ws.get<double>((size_t)E.ord.max_pairs * 2 * E.k * E.k);
        E.rot = ws.get<int>(E.ord.max_pairs);
        const size_t gsz = pivot_gscratch_doubles(E.k);
        E.gscratch = gsz ? ws.get<double>(gsz * E.ord.max_pairs) : nullptr;
        E.dpairs = ws.get<int2>(E.ord.dev_pairs.size() / 2);
        E.partial = ws.get<double>(3 * (size_t)reduce_blocks_for(E.np));
        E.ticket = ws.get<unsigned>(1);
        E.result = ws.get<double>(3);
        E.cnt = ws.get<DevCounters>(1);
        int* rank = ws.get<int>(n);
        E.pcl = choose_pivot_cluster(E.k, E.ord.dev_per_step);
        E.qtab = E.pcl > 1 ? ws.get<unsigned>(128 * 127 / 2) : nullptr;
        if (p.pivot_order == 2) E.qrws = ws.get<double>((size_t)E.ord.max_pairs * E.b * E.k);
        if (p.precision == JACOBI_PREC_FP64_EMU || p.fp64_products == 1) {
            E.T64 = ws.get<double>(emu_update_tbuf_doubles(E.ord.dev_per_step, E.k));
            E.err = ws.get<int>(1);
            if (emu_image_wanted()) {
                E.vimg = ws.get<unsigned char>(emu_update_vimg_bytes(E.ord.dev_per_step, E.k));
                E.vexp = ws.get<int>(emu_update_vexp_ints(E.ord.dev_per_step, E.k));
                if (p.conv != JACOBI_CONV_REL) {   // (balanced products slice per tile)
                    E.aimg = ws.get<unsigned char>(emu_update_aimg_bytes(E.ord.dev_per_step, E.k));
                    E.atab = ws.get<int>((size_t)E.ord.dev_per_step * E.np);
                    if (vec) {
                        E.qimg = ws.get<unsigned char>(emu_update_qimg_bytes(E.ord.dev_per_step, E.k, E.np));
                        E.qexp = ws.get<int>((size_t)E.ord.dev_per_step * E.np);
                    }
                }
            }
        }
        E.balance = p.conv == JACOBI_CONV_REL;
        if (ws.failed) return JACOBI_ERR_ALLOC;
        if (E.qtab && launch_quad_table(E.qtab, 128, s) != cudaSuccess) return JACOBI_ERR_CUDA;
        if (E.err && cudaMemsetAsync(E.err, 0, sizeof(int), s) != cudaSuccess) return JACOBI_ERR_CUDA;
        if (cudaMemcpyAsync(E.dpairs, E.ord.dev_pairs.data(), E.ord.dev_pairs.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(E.cnt, 0, sizeof(DevCounters), s) != cudaSuccess ||
            cudaMemsetAsync(E.ticket, 0, sizeof(unsigned), s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (launch_load_sym(n, E.np, A, lda, E.Aw[0], Q, ldq, E.Qw[0], vec && p.warm_start, E.cnt, s) != cudaSuccess ||
            launch_offnorm(E.np, E.Aw[0], E.partial, E.ticket, E.result,
                           p.conv == JACOBI_CONV_REL, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
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
        st->rel_final = rel ? h_res[2] : 0.0;
        const double target = rel ? p.tol : p.tol * st->norm_fro;
        const double meas0 = rel ? h_res[2] : st->off_initial;
        int cur = 0;
        int sweeps = 0;
        if (meas0 <= target) {
            rc = 0;
        } else {
            SweepResult r = run_evd_sweeps(E, p, cur, target, 0, st, s, rel);
            if (r.code < 0) return r.code;
            sweeps = r.sweeps;
            rc = r.code == 0 ? 0 : r.sweeps;
        }
        st->sweeps = sweeps;
        st->pair_solves = 0;
        if (launch_finalize_evd(n, E.np, E.Aw[cur], vec ? E.Qw[cur] : nullptr, w, vec ? Q : nullptr,
                                ldq, A, lda, rank, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        st->launches += 4;  // load, first off-norm, rank, finalise
        int h_err = 0;
        if (cudaMemcpyAsync(&hc, E.cnt, sizeof(hc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            (E.err && cudaMemcpyAsync(&h_err, E.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (h_err) return JACOBI_ERR_TIMEOUT;
        fill_counters(st, hc);
    }
    st->ms_total = timer.stop();
    return rc;
}

extern "C" int jacobi_syev(int n, double* A, int lda, double* w, double* Q, int ldq,
                           const jacobi_params* pin, jacobi_stats* stout, void* stream)
{
    jacobi_params p;
    if (pin) p = *pin; else jacobi_params_default(&p);
    if (n < 1) return -1;
    if (!A) return -2;
    if (lda < n) return -3;
    if (!w) return -4;
    if (p.want_vectors && !Q) return -5;
    if (p.want_vectors && ldq < n) return -6;
    int e = check_params(p);
    if (e) return e;
    if (p.inner_max_sweeps == 0) p.inner_max_sweeps = 1;
    jacobi_stats st;
    memset(&st, 0, sizeof(st));
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if (p.precision == JACOBI_PREC_FP64 || p.precision == JACOBI_PREC_FP64_EMU) {
        rc = syev_fp64(n, A, lda, w, Q, ldq, p, &st, s);
    } else {
        rc = syev_mixed(n, A, lda, w, Q, ldq, p, &st, s);
    }
    st.status = rc;
    if (stout) *stout = st;
    return rc;
}

// ============================================================================ SVD (FP64)
static int gesvd_fp64(int m, int n, double* G, int ldg, double* sigma, double* V, int ldv,
                      const jacobi_params& p, jacobi_stats* st, cudaStream_t s)
{
    Timer timer(s);
    const int b = p.b, k = 2 * b;
    const int N = padded_blocks(n, b, p.ordering), np = N * b;
    Ordering ord;
    if (!make_ordering(p.ordering, N, &ord)) return -7;
    const bool vec = p.want_vectors != 0;
    const double tol = std::max(p.tol, sqrt((double)m) * U64);
    const int npanels = gram_panels_for(m);
    int rc = 0;
    {
        Workspace ws(s);
        double* Gw[2] = {ws.get<double>((size_t)m * np), ws.get<double>((size_t)m * np)};
        double* Vw[2] = {vec ? ws.get<double>((size_t)np * np) : nullptr,
                         vec ? ws.get<double>((size_t)np * np) : nullptr};
        double* Vb = ws.get<double>((size_t)ord.max_pairs * 2 * k * k);
        int* rot = ws.get<int>(ord.max_pairs);
        double* relmax = ws.get<double>(ord.max_pairs);
        double* part = ws.get<double>((size_t)ord.max_pairs * npanels * k * k);
        const size_t gsz = pivot_gscratch_doubles(k);
        double* gscr = gsz ? ws.get<double>(gsz * ord.max_pairs) : nullptr;
        int2* dpairs = ws.get<int2>(ord.dev_pairs.size() / 2);
        double* sweepmax = ws.get<double>(1);
        double* norms = ws.get<double>(n);
        int* rank = ws.get<int>(n);
        DevCounters* cnt = ws.get<DevCounters>(1);
        const int pcl = choose_pivot_cluster(k, ord.dev_per_step);
        unsigned* qtab = pcl > 1 ? ws.get<unsigned>(128 * 127 / 2) : nullptr;
        double* qrws = p.pivot_order == 2 ? ws.get<double>((size_t)ord.max_pairs * b * k) : nullptr;
        const bool emu = p.precision == JACOBI_PREC_FP64_EMU || p.fp64_products == 1;
        int* err = emu ? ws.get<int>(1) : nullptr;
        if (ws.failed) return JACOBI_ERR_ALLOC;
        if (qtab && launch_quad_table(qtab, 128, s) != cudaSuccess) return JACOBI_ERR_CUDA;
        if (cudaMemcpyAsync(dpairs, ord.dev_pairs.data(), ord.dev_pairs.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(cnt, 0, sizeof(DevCounters), s) != cudaSuccess ||
            (err && cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess))
            return JACOBI_ERR_CUDA;
        if (launch_load_svd(m, n, np, G, ldg, Gw[0], Vw[0], cnt, s) != cudaSuccess) return JACOBI_ERR_CUDA;
        DevCounters hc;
        if (cudaMemcpyAsync(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (hc.nonfinite) return JACOBI_ERR_NONFINITE;

        int cur = 0, sw = 0;
        double prev = INFINITY;
        unsigned long long rot_before = 0;
        SweepGraph graphs[2];
        bool tried[2] = {false, false}, have[2] = {false, false};
        PhaseEvents pe(3 * (size_t)ord.S + 1);
        rc = -1;
        for (sw = 0; sw < p.max_sweeps; ++sw) {
            const int start = cur;
            auto body = [&](cudaStream_t cs) -> bool {
                if (cudaMemsetAsync(sweepmax, 0, sizeof(double), cs) != cudaSuccess) return false;
                if (cudaEventRecordWithFlags(pe.ev[0], cs, cudaEventRecordExternal) != cudaSuccess) return false;
                int c = start;
                for (int si = 0; si < ord.S; ++si) {
                    const int nps = ord.dev_per_step, p0 = si * nps;
                    EmuSvdArgs sa{Gw[c], Gw[c ^ 1], m, m, Vw[c], Vw[c ^ 1], np, np, dpairs + p0, nps, b, k,
                                  Vb, rot, part, npanels, gram_panel_rows(), err, cnt};
                    if ((emu ? launch_emu_gram(sa, cs)
                             : launch_gram(Gw[c], m, m, dpairs + p0, nps, b, k, part, cnt, cs)) != cudaSuccess)
                        return false;
                    if (cudaEventRecordWithFlags(pe.ev[3 * si + 1], cs, cudaEventRecordExternal) != cudaSuccess) return false;
                    PivotArgs pa{};
                    pa.ld = np;
                    pa.gram = part;
                    pa.npanels = npanels;
                    pa.pairs = dpairs + p0;
                    pa.npairs = nps;
                    pa.b = b;
                    pa.k = k;
                    pa.V = Vb;
                    pa.rot = rot;
                    pa.relmax = relmax;
                    pa.tol_rel = tol;
                    pa.max_sweeps = p.inner_max_sweeps;
                    pa.order = p.pivot_order;
                    pa.n_real = n;
                    pa.gscratch = gscr;
                    pa.qrws = qrws;
                    pa.cnt = cnt;
                    if ((pcl > 1 ? launch_pivot_cluster(pa, pcl, qtab, cs) : launch_pivot(pa, cs)) != cudaSuccess)
                        return false;
                    if (launch_max_into(relmax, nps, sweepmax, cs) != cudaSuccess) return false;
                    if (cudaEventRecordWithFlags(pe.ev[3 * si + 2], cs, cudaEventRecordExternal) != cudaSuccess) return false;
                    ColUpdateArgs ca{};
                    ca.Gin = Gw[c];
                    ca.Gout = Gw[c ^ 1];
                    ca.ldg = m;
                    ca.m = m;
                    ca.Vin = Vw[c];
                    ca.Vout = Vw[c ^ 1];
                    ca.ldv = np;
                    ca.vrows = np;
                    ca.pairs = dpairs + p0;
                    ca.npairs = nps;
                    ca.b = b;
                    ca.k = k;
                    ca.Vh = Vb;
                    ca.rot = rot;
                    ca.cnt = cnt;
                    if ((emu ? launch_emu_cols(sa, cs) : launch_update_cols(ca, cs)) != cudaSuccess) return false;
                    if (cudaEventRecordWithFlags(pe.ev[3 * si + 3], cs, cudaEventRecordExternal) != cudaSuccess) return false;
                    c ^= 1;
                }
                return true;
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
            cur = start ^ (ord.S & 1);
            double mx;
            if (cudaMemcpyAsync(&mx, sweepmax, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return JACOBI_ERR_CUDA;
            st->steps += ord.S;
            for (int si = 0; si < ord.S; ++si) {
                st->ms_update += pe.ms(3 * si, 3 * si + 1) + pe.ms(3 * si + 2, 3 * si + 3);
                st->ms_pivot += pe.ms(3 * si + 1, 3 * si + 2);
            }
            st->launches += 4 * ord.S;
            st->pivot_launches += ord.S;
            st->update_launches += 2 * ord.S;
            if (sw < 64) st->off_hist[sw] = mx;
            if (sw == 0) st->off_initial = mx;
            st->off_final = mx;
            const bool none = hc.rotations == rot_before;
            rot_before = hc.rotations;
            if (mx <= tol || none) { rc = 0; ++sw; break; }
            if (mx <= 100.0 * tol && mx > 0.5 * prev) { rc = 0; st->stalled = 1; ++sw; break; }
            prev = mx;
        }
        if (rc != 0) rc = sw;
        st->sweeps = sw;
        if (launch_finalize_svd(m, n, Gw[cur], m, vec ? Vw[cur] : nullptr, np, G, ldg, sigma,
                                vec ? V : nullptr, ldv, norms, rank, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        st->launches += 4;  // load, column norms, rank, finalise
        int h_err = 0;
        if (cudaMemcpyAsync(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            (err && cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (h_err) return JACOBI_ERR_TIMEOUT;
        fill_counters(st, hc);
    }
    st->ms_total = timer.stop();
    return rc;
}

// One-sided SVD preconditioned by a reduced QR factorisation (Sec. 6,
// "Preprocessing with QR"): G = QR (blocked Householder, in place), the
// one-sided method on X = R^T, X W = U_X Sigma, then U = Q [W; 0] (the
// reflectors applied last panel first) and V = U_X.
static int gesvd_qr(int m, int n, double* G, int ldg, double* sigma, double* V, int ldv,
                    const jacobi_params& p, jacobi_stats* st, cudaStream_t s)
{
    Timer timer(s);
    const int nb = QR_NB, npan = (n + nb - 1) / nb;
    int rc = 0;
    {
        Workspace ws(s);
        double* Y = ws.get<double>((size_t)m * n);
        double* tau = ws.get<double>(n);
        double* S = ws.get<double>((size_t)nb * nb);
        double* T = ws.get<double>((size_t)npan * nb * nb);
        double* Tt = ws.get<double>((size_t)npan * nb * nb);
        double* Wpart = ws.get<double>(qr_wpart_doubles(m, n));
        double* W = ws.get<double>((size_t)nb * n);
        double* YT = ws.get<double>((size_t)m * nb);
        double* X = ws.get<double>((size_t)n * n);
        double* Wv = ws.get<double>((size_t)n * n);
        const bool emu = p.precision == JACOBI_PREC_FP64_EMU || p.fp64_products == 1;
        int* xexp = emu ? ws.get<int>((size_t)m + n + 1) : nullptr;   // line exponents + the timeout word
        if (ws.failed) return JACOBI_ERR_ALLOC;
        if (xexp && cudaMemsetAsync(xexp + m + n, 0, sizeof(int), s) != cudaSuccess) return JACOBI_ERR_CUDA;
        auto update = [&](int j0, int nbp, const double* Tp, const double* Ttp, int trans, double* Xm, int ncol) {
            if (emu)
                return launch_house_update_emu(m, j0, nbp, Y, m, Tp, Ttp, trans, Xm, ldg, ncol, Wpart, W, YT, xexp,
                                               xexp + m, xexp + m + n, s);
            return launch_house_update(m, j0, nbp, Y, m, Tp, Ttp, trans, Xm, ldg, ncol, Wpart, W, YT, s);
        };
        cudaEvent_t ev[4];
        for (auto& e : ev) cudaEventCreate(&e);
        auto destroy = [&] {
            for (auto& e : ev) cudaEventDestroy(e);
        };
        double fl = 0.0;
        bool ok = cudaEventRecord(ev[0], s) == cudaSuccess;
        for (int pi = 0; ok && pi < npan; ++pi) {
            const int j0 = pi * nb, nbp = std::min(nb, n - j0), rows = m - j0, nc = n - j0 - nbp;
            double* Tp = T + (size_t)pi * nb * nb;
            double* Ttp = Tt + (size_t)pi * nb * nb;
            ok = launch_house_panel(m, G, ldg, j0, nbp, Y, m, tau, S, Tp, Ttp, s) == cudaSuccess &&
                 update(j0, nbp, Tp, Ttp, 1, G + (size_t)ldg * (j0 + nbp), nc) == cudaSuccess;
            fl += 5.0 * rows * nbp * nbp + 4.0 * rows * nbp * nc;   // panel 3 r nb^2, Y T^T 2 r nb^2, update
            st->launches += 2 * nbp + 1 + (nc > 0 ? 4 : 0);
        }
        ok = ok && launch_qr_rt(n, G, ldg, X, s) == cudaSuccess && cudaEventRecord(ev[1], s) == cudaSuccess;
        if (!ok) {
            destroy();
            return JACOBI_ERR_CUDA;
        }
        jacobi_params pin = p;
        pin.want_vectors = 1;
        pin.svd_qr = 0;
        rc = gesvd_fp64(n, n, X, n, sigma, Wv, n, pin, st, s);
        if (rc < 0) {
            destroy();
            return rc;
        }
        ok = cudaEventRecord(ev[2], s) == cudaSuccess;
        if (ok && p.want_vectors)
            ok = cudaMemcpy2DAsync(V, (size_t)ldv * sizeof(double), X, (size_t)n * sizeof(double),
                                   (size_t)n * sizeof(double), n, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
        ok = ok && launch_qr_fill(m, n, Wv, G, ldg, s) == cudaSuccess;
        for (int pi = npan - 1; ok && pi >= 0; --pi) {
            const int j0 = pi * nb, nbp = std::min(nb, n - j0), rows = m - j0;
            ok = update(j0, nbp, T + (size_t)pi * nb * nb, Tt + (size_t)pi * nb * nb, 0, G, n) == cudaSuccess;
            fl += 2.0 * rows * nbp * nbp + 4.0 * rows * nbp * n;
            st->launches += 4;
        }
        ok = ok && cudaEventRecord(ev[3], s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
        if (!ok) {
            destroy();
            return JACOBI_ERR_CUDA;
        }
        int h_err = 0;
        if (xexp && cudaMemcpy(&h_err, xexp + m + n, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            destroy();
            return JACOBI_ERR_CUDA;
        }
        if (h_err) {
            destroy();
            return JACOBI_ERR_TIMEOUT;
        }
        float t01 = 0.f, t23 = 0.f;
        cudaEventElapsedTime(&t01, ev[0], ev[1]);
        cudaEventElapsedTime(&t23, ev[2], ev[3]);
        destroy();
        st->ms_precond = (double)t01 + (double)t23;
        st->flops_precond = fl;
        st->flops_fp64 += fl;
        st->launches += 2;
    }
    st->ms_total = timer.stop();
    return rc;
}

extern "C" int jacobi_gesvd(int m, int n, double* G, int ldg, double* sigma, double* V, int ldv,
                            const jacobi_params* pin, jacobi_stats* stout, void* stream)
{
    jacobi_params p;
    if (pin) p = *pin; else jacobi_params_default(&p);
    if (m < 1) return -1;
    if (n < 1 || n > m) return -2;
    if (!G) return -3;
    if (ldg < m) return -4;
    if (!sigma) return -5;
    if (p.want_vectors && !V) return -6;
    if (p.want_vectors && ldv < n) return -7;
    int e = check_params(p);
    if (e) return e == -7 ? -8 : e;
    if (p.precision != JACOBI_PREC_FP64 && p.precision != JACOBI_PREC_FP64_EMU) return JACOBI_ERR_UNSUPPORTED;
    if (p.inner_max_sweeps == 0) p.inner_max_sweeps = p.svd_qr ? 2 : 30;
    jacobi_stats st;
    memset(&st, 0, sizeof(st));
    int rc = p.svd_qr ? gesvd_qr(m, n, G, ldg, sigma, V, ldv, p, &st, (cudaStream_t)stream)
                      : gesvd_fp64(m, n, G, ldg, sigma, V, ldv, p, &st, (cudaStream_t)stream);
    st.status = rc;
    if (stout) *stout = st;
    return rc;
}

// ============================================================================ host-buffer forms
extern "C" int jacobi_syev_h(int n, double* h_A, int lda, double* h_w, double* h_Q, int ldq,
                             const jacobi_params* pin, jacobi_stats* st, void* stream)
{
    jacobi_params p;
    if (pin) p = *pin; else jacobi_params_default(&p);
    if (n < 1) return -1;
    if (!h_A) return -2;
    if (lda < n) return -3;
    if (!h_w) return -4;
    if (p.want_vectors && !h_Q) return -5;
    if (p.want_vectors && ldq < n) return -6;
    cudaStream_t s = (cudaStream_t)stream;
    const bool vec = p.want_vectors != 0;
    int rc;
    {
        Workspace ws(s);
        double* dA = ws.get<double>((size_t)n * n);
        double* dw = ws.get<double>(n);
        double* dQ = vec ? ws.get<double>((size_t)n * n) : nullptr;
        if (ws.failed) return JACOBI_ERR_ALLOC;
        if (cudaMemcpy2DAsync(dA, (size_t)n * 8, h_A, (size_t)lda * 8, (size_t)n * 8, n,
                              cudaMemcpyHostToDevice, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (vec && p.warm_start &&
            cudaMemcpy2DAsync(dQ, (size_t)n * 8, h_Q, (size_t)ldq * 8, (size_t)n * 8, n,
                              cudaMemcpyHostToDevice, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        rc = jacobi_syev(n, dA, n, dw, dQ, n, &p, st, stream);
        if (rc < 0) return rc;
        if (cudaMemcpy2DAsync(h_A, (size_t)lda * 8, dA, (size_t)n * 8, (size_t)n * 8, n,
                              cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(h_w, dw, (size_t)n * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (vec && cudaMemcpy2DAsync(h_Q, (size_t)ldq * 8, dQ, (size_t)n * 8, (size_t)n * 8, n,
                                     cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return JACOBI_ERR_CUDA;
    }
    return rc;
}

extern "C" int jacobi_gesvd_h(int m, int n, double* h_G, int ldg, double* h_sigma, double* h_V,
                              int ldv, const jacobi_params* pin, jacobi_stats* st, void* stream)
{
    jacobi_params p;
    if (pin) p = *pin; else jacobi_params_default(&p);
    if (m < 1) return -1;
    if (n < 1 || n > m) return -2;
    if (!h_G) return -3;
    if (ldg < m) return -4;
    if (!h_sigma) return -5;
    if (p.want_vectors && !h_V) return -6;
    if (p.want_vectors && ldv < n) return -7;
    cudaStream_t s = (cudaStream_t)stream;
    const bool vec = p.want_vectors != 0;
    int rc;
    {
        Workspace ws(s);
        double* dG = ws.get<double>((size_t)m * n);
        double* ds = ws.get<double>(n);
        double* dV = vec ? ws.get<double>((size_t)n * n) : nullptr;
        if (ws.failed) return JACOBI_ERR_ALLOC;
        if (cudaMemcpy2DAsync(dG, (size_t)m * 8, h_G, (size_t)ldg * 8, (size_t)m * 8, n,
                              cudaMemcpyHostToDevice, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        rc = jacobi_gesvd(m, n, dG, m, ds, dV, n, &p, st, stream);
        if (rc < 0) return rc;
        if (cudaMemcpy2DAsync(h_G, (size_t)ldg * 8, dG, (size_t)m * 8, (size_t)m * 8, n,
                              cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(h_sigma, ds, (size_t)n * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (vec && cudaMemcpy2DAsync(h_V, (size_t)ldv * 8, dV, (size_t)n * 8, (size_t)n * 8, n,
                                     cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return JACOBI_ERR_CUDA;
    }
    return rc;
}

// ============================================================================ stop statistic
extern "C" int jacobi_off_norm(int n, const double* A, int lda, int want_rel, double* h_out, void* stream)
{
    if (n < 1) return -1;
    if (!A) return -2;
    if (lda < n) return -3;
    if (!h_out) return -5;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    double* partial = ws.get<double>(3 * (size_t)reduce_blocks_for(n));
    unsigned* ticket = ws.get<unsigned>(1);
    double* result = ws.get<double>(3);
    if (ws.failed) return JACOBI_ERR_ALLOC;
    double h[3];
    if (cudaMemsetAsync(ticket, 0, sizeof(unsigned), s) != cudaSuccess ||
        launch_offnorm_ld(n, A, lda, partial, ticket, result, want_rel != 0, s) != cudaSuccess ||
        cudaMemcpyAsync(h, result, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    h_out[0] = sqrt(h[0]);
    h_out[1] = sqrt(h[1]);
    h_out[2] = want_rel ? h[2] : 0.0;
    return 0;
}

// ============================================================================ single steps
extern "C" int jacobi_syev_step(int np, double* A, int lda, double* Q, int ldq,
                                const jacobi_params* pin, int step, void* stream)
{
    jacobi_params p;
    if (pin) p = *pin; else jacobi_params_default(&p);
    int e = check_params(p);
    if (e) return e == -7 ? -6 : e;
    if (p.inner_max_sweeps == 0) p.inner_max_sweeps = 1;
    if (np < 2 * p.b || np % p.b || (np / p.b) % 2) return -1;
    if (!A) return -2;
    if (lda < np) return -3;
    if (Q && ldq < np) return -5;
    cudaStream_t s = (cudaStream_t)stream;
    EvdState E{};
    E.b = p.b;
    E.k = 2 * p.b;
    E.np = np;
    E.n_real = np;
    if (!make_ordering(p.ordering, np / p.b, &E.ord)) return -1;
    if (step < 0 || step >= E.ord.S) return -7;
    const size_t np2 = (size_t)np * np;
    {
        Workspace ws(s);
        E.Aw[0] = ws.get<double>(np2);
        E.Aw[1] = ws.get<double>(np2);
        E.Qw[0] = Q ? ws.get<double>(np2) : nullptr;
        E.Qw[1] = Q ? ws.get<double>(np2) : nullptr;
        E.Vb = ws.get<double>((size_t)E.ord.max_pairs * 2 * E.k * E.k);
        E.rot = ws.get<int>(E.ord.max_pairs);
        const size_t gsz = pivot_gscratch_doubles(E.k);
        E.gscratch = gsz ? ws.get<double>(gsz * E.ord.max_pairs) : nullptr;
        E.dpairs = ws.get<int2>(E.ord.dev_pairs.size() / 2);
        E.cnt = ws.get<DevCounters>(1);
        E.pcl = choose_pivot_cluster(E.k, E.ord.dev_per_step);
        E.qtab = E.pcl > 1 ? ws.get<unsigned>(128 * 127 / 2) : nullptr;
        if (p.pivot_order == 2) E.qrws = ws.get<double>((size_t)E.ord.max_pairs * E.b * E.k);
        if (p.precision == JACOBI_PREC_FP64_EMU || (p.precision == JACOBI_PREC_FP64 && p.fp64_products == 1)) {
            E.T64 = ws.get<double>(emu_update_tbuf_doubles(E.ord.dev_per_step, E.k));
            E.err = ws.get<int>(1);
            if (emu_image_wanted()) {
                E.vimg = ws.get<unsigned char>(emu_update_vimg_bytes(E.ord.dev_per_step, E.k));
                E.vexp = ws.get<int>(emu_update_vexp_ints(E.ord.dev_per_step, E.k));
                if (p.conv != JACOBI_CONV_REL) {   // (balanced products slice per tile)
                    E.aimg = ws.get<unsigned char>(emu_update_aimg_bytes(E.ord.dev_per_step, E.k));
                    E.atab = ws.get<int>((size_t)E.ord.dev_per_step * E.np);
                    if (Q) {
                        E.qimg = ws.get<unsigned char>(emu_update_qimg_bytes(E.ord.dev_per_step, E.k, E.np));
                        E.qexp = ws.get<int>((size_t)E.ord.dev_per_step * E.np);
                    }
                }
            }
        } else if (p.precision != JACOBI_PREC_FP64) {
            return JACOBI_ERR_UNSUPPORTED;
        }
        E.balance = p.conv == JACOBI_CONV_REL;
        if (ws.failed) return JACOBI_ERR_ALLOC;
        if (E.err && cudaMemsetAsync(E.err, 0, sizeof(int), s) != cudaSuccess) return JACOBI_ERR_CUDA;
        if (E.qtab && launch_quad_table(E.qtab, 128, s) != cudaSuccess) return JACOBI_ERR_CUDA;
        if (cudaMemcpyAsync(E.dpairs, E.ord.dev_pairs.data(), E.ord.dev_pairs.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(E.cnt, 0, sizeof(DevCounters), s) != cudaSuccess ||
            cudaMemcpy2DAsync(E.Aw[0], (size_t)np * 8, A, (size_t)lda * 8, (size_t)np * 8, np,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpy2DAsync(E.Aw[1], (size_t)np * 8, A, (size_t)lda * 8, (size_t)np * 8, np,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (Q && cudaMemcpy2DAsync(E.Qw[0], (size_t)np * 8, Q, (size_t)ldq * 8, (size_t)np * 8, np,
                                   cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (launch_step(E, step, 0, s, p.inner_tol, p.inner_max_sweeps, p.pivot_order) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (cudaMemcpy2DAsync(A, (size_t)lda * 8, E.Aw[1], (size_t)np * 8, (size_t)np * 8, np,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (Q && cudaMemcpy2DAsync(Q, (size_t)ldq * 8, E.Qw[1], (size_t)np * 8, (size_t)np * 8, np,
                                   cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        int h_err = 0;
        if ((E.err && cudaMemcpyAsync(&h_err, E.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (h_err) return JACOBI_ERR_TIMEOUT;
    }
    return 0;
}

extern "C" int jacobi_gesvd_step(int m, int np, double* G, int ldg, double* V, int ldv,
                                 const jacobi_params* pin, int step, double* relmax_out,
                                 void* stream)
{
    jacobi_params p;
    if (pin) p = *pin; else jacobi_params_default(&p);
    int e = check_params(p);
    if (e) return e == -7 ? -7 : e;
    if (p.precision != JACOBI_PREC_FP64 && p.precision != JACOBI_PREC_FP64_EMU) return JACOBI_ERR_UNSUPPORTED;
    if (p.inner_max_sweeps == 0) p.inner_max_sweeps = 30;
    if (m < 1) return -1;
    if (np < 2 * p.b || np % p.b || (np / p.b) % 2 || np > m) return -2;
    if (!G) return -3;
    if (ldg < m) return -4;
    if (V && ldv < np) return -6;
    cudaStream_t s = (cudaStream_t)stream;
    const int b = p.b, k = 2 * b;
    Ordering ord;
    if (!make_ordering(p.ordering, np / b, &ord)) return -2;
    if (step < 0 || step >= ord.S) return -8;
    const double tol = std::max(p.tol, sqrt((double)m) * U64);
    const int npanels = gram_panels_for(m);
    const int nps = ord.dev_per_step, p0 = step * nps;
    {
        Workspace ws(s);
        double* Gw[2] = {ws.get<double>((size_t)m * np), ws.get<double>((size_t)m * np)};
        double* Vw[2] = {V ? ws.get<double>((size_t)np * np) : nullptr,
                         V ? ws.get<double>((size_t)np * np) : nullptr};
        double* Vb = ws.get<double>((size_t)ord.max_pairs * 2 * k * k);
        int* rot = ws.get<int>(ord.max_pairs);
        double* relmax = ws.get<double>(ord.max_pairs);
        double* part = ws.get<double>((size_t)ord.max_pairs * npanels * k * k);
        const size_t gsz = pivot_gscratch_doubles(k);
        double* gscr = gsz ? ws.get<double>(gsz * ord.max_pairs) : nullptr;
        int2* dpairs = ws.get<int2>(ord.dev_pairs.size() / 2);
        double* smax = ws.get<double>(1);
        DevCounters* cnt = ws.get<DevCounters>(1);
        const int pcl = choose_pivot_cluster(k, nps);
        unsigned* qtab = pcl > 1 ? ws.get<unsigned>(128 * 127 / 2) : nullptr;
        double* qrws = p.pivot_order == 2 ? ws.get<double>((size_t)ord.max_pairs * b * k) : nullptr;
        const bool emu = p.precision == JACOBI_PREC_FP64_EMU || p.fp64_products == 1;
        int* err = emu ? ws.get<int>(1) : nullptr;
        if (ws.failed) return JACOBI_ERR_ALLOC;
        if (err && cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return JACOBI_ERR_CUDA;
        if (qtab && launch_quad_table(qtab, 128, s) != cudaSuccess) return JACOBI_ERR_CUDA;
        if (cudaMemcpyAsync(dpairs, ord.dev_pairs.data(), ord.dev_pairs.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(cnt, 0, sizeof(DevCounters), s) != cudaSuccess ||
            cudaMemsetAsync(smax, 0, sizeof(double), s) != cudaSuccess ||
            cudaMemcpy2DAsync(Gw[0], (size_t)m * 8, G, (size_t)ldg * 8, (size_t)m * 8, np,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (V && cudaMemcpy2DAsync(Vw[0], (size_t)np * 8, V, (size_t)ldv * 8, (size_t)np * 8, np,
                                   cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        EmuSvdArgs sa{Gw[0], Gw[1], m, m, Vw[0], Vw[1], np, np, dpairs + p0, nps, b, k,
                      Vb, rot, part, npanels, gram_panel_rows(), err, cnt};
        if ((emu ? launch_emu_gram(sa, s) : launch_gram(Gw[0], m, m, dpairs + p0, nps, b, k, part, cnt, s)) !=
            cudaSuccess)
            return JACOBI_ERR_CUDA;
        PivotArgs pa{};
        pa.ld = np;
        pa.gram = part;
        pa.npanels = npanels;
        pa.pairs = dpairs + p0;
        pa.npairs = nps;
        pa.b = b;
        pa.k = k;
        pa.V = Vb;
        pa.rot = rot;
        pa.relmax = relmax;
        pa.tol_rel = tol;
        pa.max_sweeps = p.inner_max_sweeps;
        pa.order = p.pivot_order;
        pa.n_real = np;
        pa.gscratch = gscr;
        pa.qrws = qrws;
        pa.cnt = cnt;
        if ((pcl > 1 ? launch_pivot_cluster(pa, pcl, qtab, s) : launch_pivot(pa, s)) != cudaSuccess ||
            launch_max_into(relmax, nps, smax, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        ColUpdateArgs ca{};
        ca.Gin = Gw[0];
        ca.Gout = Gw[1];
        ca.ldg = m;
        ca.m = m;
        ca.Vin = Vw[0];
        ca.Vout = Vw[1];
        ca.ldv = np;
        ca.vrows = np;
        ca.pairs = dpairs + p0;
        ca.npairs = nps;
        ca.b = b;
        ca.k = k;
        ca.Vh = Vb;
        ca.rot = rot;
        ca.cnt = cnt;
        if ((emu ? launch_emu_cols(sa, s) : launch_update_cols(ca, s)) != cudaSuccess) return JACOBI_ERR_CUDA;
        // columns of pairs outside this step are unchanged: copy them through
        if (cudaMemcpy2DAsync(G, (size_t)ldg * 8, Gw[0], (size_t)m * 8, (size_t)m * 8, np,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        for (int e2 = 0; e2 < nps; ++e2) {
            int I = ord.dev_pairs[2 * (p0 + e2)], J = ord.dev_pairs[2 * (p0 + e2) + 1];
            if (I < 0) { I = -1 - I; J = -1 - J; }
            for (int blk : {I, J}) {
                if (cudaMemcpy2DAsync(G + (size_t)ldg * blk * b, (size_t)ldg * 8,
                                      Gw[1] + (size_t)m * blk * b, (size_t)m * 8, (size_t)m * 8, b,
                                      cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                    return JACOBI_ERR_CUDA;
                if (V && cudaMemcpy2DAsync(V + (size_t)ldv * blk * b, (size_t)ldv * 8,
                                           Vw[1] + (size_t)np * blk * b, (size_t)np * 8,
                                           (size_t)np * 8, b, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                    return JACOBI_ERR_CUDA;
            }
        }
        double h;
        int h_err = 0;
        if (cudaMemcpyAsync(&h, smax, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            (err && cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
        if (h_err) return JACOBI_ERR_TIMEOUT;
        if (relmax_out) *relmax_out = h;
    }
    return 0;
}

extern "C" int jacobi_rotation_params(int count, const double* app, const double* aqq, const double* apq,
                                      double tol, double* out, void* stream)
{
    if (count < 0) return -1;
    if (count > 0 && !app) return -2;
    if (count > 0 && !aqq) return -3;
    if (count > 0 && !apq) return -4;
    if (!(tol >= 0.0)) return -5;
    if (count > 0 && !out) return -6;
    return launch_rotation_params(count, app, aqq, apq, tol, out, (cudaStream_t)stream) == cudaSuccess
               ? 0 : JACOBI_ERR_CUDA;
}
