// k_pivot_cluster.cu -- the pivot solves of one step with a thread-block
// cluster of C CTAs per pair, so that a step's few pairs (n/(2b) of them)
// keep all SMs busy: at n = 4096, b = 64 a step has 32 pairs; with C = 4 they
// occupy 128 SMs instead of 32.
//
// Same computation as k_pivot (Algorithm 2 applied with b = 1 to each 2b x 2b
// pivot, rotations in Rutishauser's form, diagonal carried as hi + lo), laid
// out over the cluster's distributed shared memory:
//   * the packed lower triangle of the pivot is split by row ranges over the
//     C CTAs (entry (i, j), i >= j, lives in the CTA that owns row i) and is
//     read and written through DSMEM addresses;
//   * V is split by rows (CTA r owns rows [r k/C, (r+1) k/C)), so rotating
//     its column pairs is local;
//   * every CTA keeps its own copy of the diagonal (hi and lo) and computes
//     every rotation of a round itself from that copy and the (shared) a_pq,
//     so the copies stay identical.  A split cluster barrier (arrive after
//     choosing the rotations, wait before the rotated a_pq entries are
//     zeroed) keeps those zeroes from racing a slower CTA's reads without
//     stalling the rotation work; a full cluster barrier ends each round.
// Quads (2x2 cross-pair blocks) are spread over all C * blockDim threads.
// Every loop runs the same trip count in all CTAs of a cluster, so the
// cluster barriers always match.
//
// Two schedules of the rounds, with the same arithmetic (bit for bit the
// same results):
//   * split (kFused = false): phase A rotates the quads of round g; after a
//     cluster barrier every CTA chooses all rotations of round g + 1 from its
//     own diagonal replica while the other threads rotate V by round g; a
//     split cluster barrier separates that choice from the next zeroing;
//   * fused (kFused = true; the default for k > 128): one phase and one cluster barrier
//     per round.  Round g + 1 pairs every index with one of round g's other
//     pairs, so each of its pivot entries a_p'q' is one entry of one quad of
//     round g.  Those few quads ("leading quads") are rotated first, by the
//     first warp(s) of the CTAs, and the thread that rotates one takes the
//     diagonal of p' and q' through round g and chooses round g + 1's
//     rotation right away, writing its parameters and the two diagonal
//     entries into every CTA of the cluster (double-buffered by round
//     parity).  The other threads rotate the remaining quads and this CTA's
//     rows of V by round g meanwhile.  Each rotation is chosen once per
//     cluster instead of once per CTA, and the choice overlaps the round's
//     bulk FP64 work instead of following it.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include "internal.h"
#include "jacobi_core.cuh"
#include "cluster_common.cuh"
#include "qrcp.cuh"

namespace cg = cooperative_groups;

namespace jac {

constexpr int PC_T = 512;
constexpr int PC_MAXC8 = 8;   // pivot clusters: portable sizes only

__device__ __forceinline__ int pc_pair_map(int I, int J, int b, int x)
{
    return x < b ? I * b + x : J * b + (x - b);
}

size_t pivot_cluster_smem(int k, int C)
{
    const int half = k / 2;
    const size_t chunk = (size_t)split_max_chunk(k, C);
    const size_t vrows = (size_t)(k / C) * k;
    return (chunk + vrows + 4 * (size_t)k + 10 * (size_t)half) * sizeof(double) +
           6 * (size_t)half * sizeof(int) + 64;
}

// The round-robin order over k indices (nr = k - 1 rounds): position 0 holds
// index 0; position pos >= 1 holds index 1 + (pos - 1 + rd) mod nr; pair ee
// joins positions ee and k - 1 - ee (the rule of choose() below).
__device__ __forceinline__ int rr_index_at(int pos, int rd, int nr)
{
    if (pos == 0) return 0;
    int v = pos - 1 + rd;
    if (v >= nr) v -= nr;
    return 1 + v;
}
__device__ __forceinline__ int rr_position_of(int x, int rd, int nr)
{
    if (x == 0) return 0;
    int v = x - 1 - rd;
    if (v < 0) v += nr;
    return 1 + v;
}
__device__ __forceinline__ int rr_pair_of(int x, int rd, int k)
{
    const int pos = rr_position_of(x, rd, k - 1);
    return pos < k - 1 - pos ? pos : k - 1 - pos;
}
__device__ __forceinline__ int rr_partner_of(int x, int rd, int k)
{
    return rr_index_at(k - 1 - rr_position_of(x, rd, k - 1), rd, k - 1);
}

template <bool V32> struct PcVType { using T = double; };
template <> struct PcVType<true> { using T = float; };

// kV32: this CTA's rows of V accumulated in FP32 (rotation parameters rounded
// to FP32 once, when they are chosen), for a V that only feeds the split
// low-precision products
template <bool kFused, bool kV32>
__global__ void __launch_bounds__(PC_T) k_pivot_cluster(PivotArgs a, int C, const unsigned* qtab)
{
    using VT = typename PcVType<kV32>::T;
    extern __shared__ __align__(16) double csm[];
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    const int e = blockIdx.x / C;
    const int tid = threadIdx.x, nt = blockDim.x, gtid = r * nt + tid, gnt = C * nt;
    const int k = a.k, b = a.b, half = k >> 1, nq = half * (half - 1) / 2;
    const int rows = k / C, r_lo = r * rows;
    int I, J;
    {
        const int2 pr = a.pairs[e];
        const bool fz = pr.x < 0;
        I = fz ? -1 - pr.x : pr.x;
        J = fz ? -1 - pr.y : pr.y;
    }
    const bool frozen = a.pairs[e].x < 0;

    DistPacked<double, PC_MAXC8> ap;
    make_split(k, C, ap.sp);
    const int chunk_max = [&] {
        int m = 0;
        for (int u = 0; u < C; ++u) m = max(m, ap.sp.base[u + 1] - ap.sp.base[u]);
        return m;
    }();
    double* my_chunk = csm;
    VT* Vl = reinterpret_cast<VT*>(my_chunk + chunk_max);   // rows x k (ld rows): V(r_lo + i, j) at Vl[i + rows j]
    double* dhi = my_chunk + chunk_max + (size_t)rows * k;  // diagonal replica (fused: round-parity buffer 0)
    double* dlo = dhi + k;
    double* dhi1 = dlo + k;                  // fused: round-parity buffer 1
    double* dlo1 = dhi1 + k;
    double* rtau = dlo1 + k;                 // rotation parameters, two slots of half each
    double* rs = rtau + 2 * half;
    double* rt = rs + 2 * half;
    double* rapq = rt + 2 * half;
    float* rs32 = (float*)(rapq + 2 * half);  // kV32: s and tau rounded to FP32, same slots
    float* rtau32 = rs32 + 2 * half;
    int* rp = (int*)(rtau32 + 2 * half);
    int* rq = rp + 2 * half;
    int* ron = rq + 2 * half;
    __shared__ int s_cnt[2];   // rotations chosen per sweep (by sweep parity)
    __shared__ int s_cntg[4];  // fused: rank 0's copy counts a sweep's rotations (sweep mod 4)
    __shared__ double s_red[PC_T / 32];
    __shared__ double s_part[PC_MAXC8];
    __shared__ int s_dest[256];
    __shared__ int s_pos[256];
    // entry (i, j) of the distributed pivot: a row table (owner rank, offset of
    // the row in the owner's chunk) and mapa addressing of the owner's window
    __shared__ int s_rinfo[256];
    for (int i = tid; i < k; i += nt) {
        int ow = 0;
        for (int u = 1; u < C; ++u)
            if (i >= ap.sp.row0[u]) ow = u;
        s_rinfo[i] = (ow << 20) | (tri(i) - ap.sp.base[ow]);
    }
    const DistRows<double> dr{(uint32_t)__cvta_generic_to_shared(my_chunk), s_rinfo};

    // ---- load: the entries this CTA owns, V rows = identity rows
    const int my_lo = ap.sp.row0[r], my_hi = ap.sp.row0[r + 1];
    if (a.gram == nullptr) {
        for (int idx = tid; idx < k * k; idx += nt) {
            const int ii = idx % k, jj = idx / k;
            if (ii < jj || ii < my_lo || ii >= my_hi) continue;
            const size_t gi = pc_pair_map(I, J, b, ii) + (size_t)a.ld * pc_pair_map(I, J, b, jj);
            my_chunk[tri(ii) + jj - ap.sp.base[r]] = a.Ain32 ? (double)a.Ain32[gi] : a.Ain[gi];
        }
    } else {
        const double* g = a.gram + (size_t)e * a.npanels * k * k;
        for (int idx = tid; idx < k * k; idx += nt) {
            const int ii = idx % k, jj = idx / k;
            if (ii < jj || ii < my_lo || ii >= my_hi) continue;
            double s = 0.0;
            for (int p = 0; p < a.npanels; ++p) s += g[(size_t)p * k * k + idx];  // fixed order
            my_chunk[tri(ii) + jj - ap.sp.base[r]] = s;
        }
    }
    for (int idx = tid; idx < rows * k; idx += nt) {
        const int i = idx % rows, j = idx / rows;
        Vl[idx] = (r_lo + i == j) ? VT(1) : VT(0);
    }
    cluster.sync();
    for (int x = tid; x < k; x += nt) {
        dhi[x] = dsm_ld(dr.addr(x, x), 0.0);
        dlo[x] = 0.0;
    }

    // ---- one-sided stop statistic (Gram pivots), max over the cluster
    if (a.relmax) {
        __syncthreads();
        double mx = 0.0;
        if (!frozen)
            for (int idx = tid; idx < k * k; idx += nt) {
                const int ii = idx % k, jj = idx / k;
                if (ii <= jj || ii < my_lo || ii >= my_hi) continue;
                const double d = sqrt(dhi[ii]) * sqrt(dhi[jj]);
                if (d > 0.0) mx = fmax(mx, fabs(my_chunk[tri(ii) + jj - ap.sp.base[r]]) / d);
            }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0) s_red[tid >> 5] = mx;
        __syncthreads();
        if (tid == 0) {
            double m = 0.0;
            for (int w = 0; w < nt / 32; ++w) m = fmax(m, s_red[w]);
            *cluster.map_shared_rank(&s_part[r], 0) = m;
        }
        cluster.sync();
        if (r == 0 && tid == 0) {
            double m = 0.0;
            for (int u = 0; u < C; ++u) m = fmax(m, s_part[u]);
            a.relmax[e] = m;
        }
    }
    __syncthreads();

    // ---- inner sweeps, software-pipelined over the rounds (global round
    // index g = sweep * (k - 1) + round; parameters of round g in slot g & 1):
    //   phase A(g): rank 0 zeroes the pivot entries a_pq of round g (every
    //     CTA read them while choosing round g), the quads of round g over
    //     the cluster, the diagonal replica (threads < half);
    //   phase B(g): threads < half choose round g + 1 (it reads the a_pq the
    //     quads of round g left and the updated diagonal) while the others
    //     rotate this CTA's rows of V by round g.
    // A full cluster barrier ends phase A; phase B ends with a CTA barrier
    // and a cluster arrive whose wait comes before the next zeroing.
    const double tol = a.tol_rel;
    const int max_sweeps = frozen ? 0 : a.max_sweeps;
    const int nr = k - 1;
    int total_rot = 0, sweeps = 0;
    auto choose = [&](int g, int slot) {
        const int rd = g % nr;
        int* cnt = &s_cnt[(g / nr) & 1];
        for (int ee = tid; ee < half; ee += nt) {
            const int pa = ee, pb = k - 1 - ee;
            const int ia = pa == 0 ? 0 : 1 + (pa - 1 + rd) % (k - 1);
            const int ib = 1 + (pb - 1 + rd) % (k - 1);
            const int p = ia < ib ? ia : ib, q = ia < ib ? ib : ia;
            const double app = dhi[p], aqq = dhi[q], apq = dsm_ld(dr.addr(q, p), 0.0);
            const bool on = rotation_wanted(app, aqq, apq, tol);
            const int o = slot * half + ee;
            rp[o] = p;
            rq[o] = q;
            ron[o] = on;
            if (on) {
                double sv, tv, tauv;
                schur2(app, aqq, apq, sv, tv, tauv);
                rtau[o] = tauv;
                rs[o] = sv;
                rt[o] = tv;
                rapq[o] = apq;
                if (kV32) {
                    rs32[o] = (float)sv;
                    rtau32[o] = (float)tauv;
                }
                atomicAdd(cnt, 1);
            }
        }
    };
    double* dfin = dhi;   // the final diagonal (hi, rounded once with lo)
    if constexpr (!kFused) {
        if (max_sweeps > 0) {
            if (tid == 0) s_cnt[0] = s_cnt[1] = 0;
            __syncthreads();
            if (tid < half) choose(0, 0);
            __syncthreads();
            asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
        }
        for (int sw = 0; sw < max_sweeps; ++sw) {
            for (int rd = 0; rd < nr; ++rd) {
                const int g = sw * nr + rd, so = (g & 1) * half;
                // phase A: quads over the whole cluster
                for (int qi = gtid; qi < nq; qi += gnt) {
                    int e1, e2;
                    quad_of(qtab, qi, e1, e2);
                    const int on1 = ron[so + e1], on2 = ron[so + e2];
                    if (!(on1 | on2)) continue;
                    const int p1 = rp[so + e1], q1 = rq[so + e1], p2 = rp[so + e2], q2 = rq[so + e2];
                    const uint32_t a00 = dr.addr(p1, p2);
                    const uint32_t a01 = dr.addr(p1, q2);
                    const uint32_t a10 = dr.addr(q1, p2);
                    const uint32_t a11 = dr.addr(q1, q2);
                    double x00 = dsm_ld(a00, 0.0), x01 = dsm_ld(a01, 0.0), x10 = dsm_ld(a10, 0.0), x11 = dsm_ld(a11, 0.0);
                    if (on1) {
                        const double sv = rs[so + e1], tauv = rtau[so + e1];
                        rot2(sv, tauv, x00, x10);
                        rot2(sv, tauv, x01, x11);
                    }
                    if (on2) {
                        const double sv = rs[so + e2], tauv = rtau[so + e2];
                        rot2(sv, tauv, x00, x01);
                        rot2(sv, tauv, x10, x11);
                    }
                    dsm_st(a00, x00);
                    dsm_st(a01, x01);
                    dsm_st(a10, x10);
                    dsm_st(a11, x11);
                }
                // diagonal replica (every CTA): the exact 2x2 diagonal form
                for (int ee = tid; ee < half; ee += nt) {
                    if (!ron[so + ee]) continue;
                    const int p = rp[so + ee], q = rq[so + ee];
                    const double tv = rt[so + ee], apq = rapq[so + ee];
                    dd_add_prod(dhi[p], dlo[p], tv, -apq, 1.0);
                    dd_add_prod(dhi[q], dlo[q], tv, apq, 1.0);
                }
                // every CTA has read round g's a_pq: rank 0 zeroes them
                __syncwarp();
                asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
                if (r == 0)
                    for (int ee = tid; ee < half; ee += nt)
                        if (ron[so + ee]) dsm_st(dr.addr(rq[so + ee], rp[so + ee]), 0.0);
                cluster.sync();
                // phase B
                if (tid < half) {
                    if (!(rd == nr - 1 && sw + 1 == max_sweeps)) choose(g + 1, (g + 1) & 1);
                } else {
                    for (int it = tid - half; it < half * rows; it += nt - half) {
                        const int ee = it / rows, i = it - ee * rows;
                        if (!ron[so + ee]) continue;
                        const int p = rp[so + ee], q = rq[so + ee];
                        VT vp = Vl[i + (size_t)rows * p], vq = Vl[i + (size_t)rows * q];
                        if constexpr (kV32) rot2(rs32[so + ee], rtau32[so + ee], vp, vq);
                        else rot2(rs[so + ee], rtau[so + ee], vp, vq);
                        Vl[i + (size_t)rows * p] = vp;
                        Vl[i + (size_t)rows * q] = vq;
                    }
                }
                __syncthreads();
                asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
            }
            const int cnt = s_cnt[sw & 1];
            total_rot += cnt;
            sweeps = sw + 1;
            __syncthreads();
            if (tid == 0) s_cnt[sw & 1] = 0;   // reused by sweep sw + 2 (chosen after further barriers)
            if (cnt == 0) break;
        }
        __syncwarp();
        if (max_sweeps > 0) asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
        for (int x = tid; x < k; x += nt) dhi[x] += dlo[x];  // hi + lo, rounded once
        __syncthreads();
    } else {
        // ---- fused schedule: one phase and one cluster barrier per round
        double* Dh[2] = {dhi, dhi1};
        double* Dl[2] = {dlo, dlo1};
        const int upc = (half + C - 1) / C;            // leading units per CTA (next-round pairs)
        const int lw = (upc + 31) / 32 * 32;           // threads of the leading warps
        const int bt = nt - lw, btid = tid - lw;       // the bulk threads
        int* cnt0 = cluster.map_shared_rank(s_cntg, 0);
        int G = 0;                                     // rounds run
        // rotation of round g + 1 for the pair (x, y) of that round (index epc),
        // x, y already rotated by round g (their entry axy and diagonals given),
        // written with the two diagonal entries into every CTA of the cluster
        auto publish = [&](int sn, int nb, int epc, int x, int y, double axy, double hx, double lx,
                           double hy, double ly, bool want, int cslot) {
            const int p = x < y ? x : y, q = x < y ? y : x;
            const double app = p == x ? hx : hy, aqq = p == x ? hy : hx;
            bool on = false;
            double sv = 0.0, tv = 0.0, tauv = 0.0;
            if (want) {
                on = rotation_wanted(app, aqq, axy, tol);
                if (on) schur2(app, aqq, axy, sv, tv, tauv);
            }
            const int o = sn + epc;
            for (int u = 0; u < C; ++u) {
                *cluster.map_shared_rank(&Dh[nb][x], u) = hx;
                *cluster.map_shared_rank(&Dl[nb][x], u) = lx;
                *cluster.map_shared_rank(&Dh[nb][y], u) = hy;
                *cluster.map_shared_rank(&Dl[nb][y], u) = ly;
                if (!want) continue;
                *cluster.map_shared_rank(&rp[o], u) = p;
                *cluster.map_shared_rank(&rq[o], u) = q;
                *cluster.map_shared_rank(&ron[o], u) = on ? 1 : 0;
                if (on) {
                    *cluster.map_shared_rank(&rtau[o], u) = tauv;
                    *cluster.map_shared_rank(&rs[o], u) = sv;
                    *cluster.map_shared_rank(&rt[o], u) = tv;
                    *cluster.map_shared_rank(&rapq[o], u) = axy;
                    if (kV32) {
                        *cluster.map_shared_rank(&rtau32[o], u) = (float)tauv;
                        *cluster.map_shared_rank(&rs32[o], u) = (float)sv;
                    }
                }
            }
            if (on) atomicAdd(&cnt0[cslot & 3], 1);
        };
        if (max_sweeps > 0) {
            if (tid < 4) s_cntg[tid] = 0;
            __syncthreads();
            // round 0, chosen by every CTA from its own copy (counted by rank 0)
            for (int ee = tid; ee < half; ee += nt) {
                const int pa = ee, pb = k - 1 - ee;
                const int ia = rr_index_at(pa, 0, nr), ib = rr_index_at(pb, 0, nr);
                const int p = ia < ib ? ia : ib, q = ia < ib ? ib : ia;
                const double app = dhi[p], aqq = dhi[q], apq = dsm_ld(dr.addr(q, p), 0.0);
                const bool on = rotation_wanted(app, aqq, apq, tol);
                rp[ee] = p;
                rq[ee] = q;
                ron[ee] = on;
                if (on) {
                    double sv, tv, tauv;
                    schur2(app, aqq, apq, sv, tv, tauv);
                    rtau[ee] = tauv;
                    rs[ee] = sv;
                    rt[ee] = tv;
                    rapq[ee] = apq;
                    if (kV32) {
                        rs32[ee] = (float)sv;
                        rtau32[ee] = (float)tauv;
                    }
                    if (r == 0) atomicAdd(&s_cntg[0], 1);
                }
            }
            cluster.sync();
        }
        for (int sw = 0; sw < max_sweeps; ++sw) {
            // the counter of sweep sw + 2 was last read after sweep sw - 2
            if (r == 0 && tid == 0) s_cntg[(sw + 2) & 3] = 0;
            for (int rd = 0; rd < nr; ++rd) {
                const int g = sw * nr + rd, so = (g & 1) * half, sn = half - so;
                const int cb = g & 1, nb = cb ^ 1;
                const bool last = rd == nr - 1 && sw + 1 == max_sweeps;
                const int rdn = rd + 1 == nr ? 0 : rd + 1;
                const int cslot = rd + 1 == nr ? sw + 1 : sw;
                // diagonal entry x through round g (the exact 2x2 diagonal form)
                auto diag_after = [&](int x, double& h, double& l) {
                    h = Dh[cb][x];
                    l = Dl[cb][x];
                    const int eg = rr_pair_of(x, rd, k);
                    if (ron[so + eg]) {
                        if (x == rp[so + eg]) dd_add_prod(h, l, rt[so + eg], -rapq[so + eg], 1.0);
                        else dd_add_prod(h, l, rt[so + eg], rapq[so + eg], 1.0);
                    }
                };
                if (tid < lw) {
                    const int ep = r + C * tid;   // this unit's pair of round g + 1
                    if (ep < half) {
                        const int x0 = rr_index_at(ep, rdn, nr), y0 = rr_index_at(k - 1 - ep, rdn, nr);
                        if (last) {
                            double hx, lx, hy, ly;
                            diag_after(x0, hx, lx);
                            diag_after(y0, hy, ly);
                            publish(sn, nb, ep, x0, y0, 0.0, hx, lx, hy, ly, false, 0);
                        } else {
                            const int ea = rr_pair_of(x0, rd, k), eb = rr_pair_of(y0, rd, k);
                            const int e1 = ea < eb ? ea : eb, e2 = ea < eb ? eb : ea;
                            const int p1 = rp[so + e1], q1 = rq[so + e1], p2 = rp[so + e2], q2 = rq[so + e2];
                            const int pp1 = rr_partner_of(p1, rdn, k), pq1 = rr_partner_of(q1, rdn, k);
                            const bool h1 = pp1 == p2 || pp1 == q2, h2 = pq1 == p2 || pq1 == q2;
                            const int ep1 = h1 ? rr_pair_of(p1, rdn, k) : half;
                            const int ep2 = h2 ? rr_pair_of(q1, rdn, k) : half;
                            if ((ep1 < ep2 ? ep1 : ep2) == ep) {   // this unit leads quad (e1, e2)
                                const int on1 = ron[so + e1], on2 = ron[so + e2];
                                const uint32_t a00 = dr.addr(p1, p2);
                                const uint32_t a01 = dr.addr(p1, q2);
                                const uint32_t a10 = dr.addr(q1, p2);
                                const uint32_t a11 = dr.addr(q1, q2);
                                double x00 = dsm_ld(a00, 0.0), x01 = dsm_ld(a01, 0.0), x10 = dsm_ld(a10, 0.0), x11 = dsm_ld(a11, 0.0);
                                // the diagonal through round g needs only round g's parameters:
                                // formed while the quad's entries are in flight
                                double hp1 = 0.0, lp1 = 0.0, hpp = 0.0, lpp = 0.0, hq1 = 0.0, lq1 = 0.0, hpq = 0.0, lpq = 0.0;
                                if (h1) {
                                    diag_after(p1, hp1, lp1);
                                    diag_after(pp1, hpp, lpp);
                                }
                                if (h2) {
                                    diag_after(q1, hq1, lq1);
                                    diag_after(pq1, hpq, lpq);
                                }
                                if (on1) {
                                    const double sv = rs[so + e1], tauv = rtau[so + e1];
                                    rot2(sv, tauv, x00, x10);
                                    rot2(sv, tauv, x01, x11);
                                }
                                if (on2) {
                                    const double sv = rs[so + e2], tauv = rtau[so + e2];
                                    rot2(sv, tauv, x00, x01);
                                    rot2(sv, tauv, x10, x11);
                                }
                                if (on1 | on2) {
                                    dsm_st(a00, x00);
                                    dsm_st(a01, x01);
                                    dsm_st(a10, x10);
                                    dsm_st(a11, x11);
                                }
                                if (h1) publish(sn, nb, ep1, p1, pp1, pp1 == p2 ? x00 : x01, hp1, lp1, hpp, lpp, true, cslot);
                                if (h2) publish(sn, nb, ep2, q1, pq1, pq1 == p2 ? x10 : x11, hq1, lq1, hpq, lpq, true, cslot);
                            }
                        }
                    }
                    // round g's pivot entries (read when round g was chosen, before
                    // the last barrier; no quad of round g holds them)
                    if (ep < half && ron[so + ep]) dsm_st(dr.addr(rq[so + ep], rp[so + ep]), 0.0);
                } else {
                    // the other quads of round g over the cluster's bulk threads
                    for (int qi = r * bt + btid; qi < nq; qi += C * bt) {
                        int e1, e2;
                        quad_of(qtab, qi, e1, e2);
                        const int on1 = ron[so + e1], on2 = ron[so + e2];
                        if (!(on1 | on2)) continue;
                        const int p1 = rp[so + e1], q1 = rq[so + e1], p2 = rp[so + e2], q2 = rq[so + e2];
                        if (!last) {   // a leading quad: rotated by its leading unit
                            const int pp1 = rr_partner_of(p1, rdn, k), pq1 = rr_partner_of(q1, rdn, k);
                            if (pp1 == p2 || pp1 == q2 || pq1 == p2 || pq1 == q2) continue;
                        }
                        const uint32_t a00 = dr.addr(p1, p2);
                        const uint32_t a01 = dr.addr(p1, q2);
                        const uint32_t a10 = dr.addr(q1, p2);
                        const uint32_t a11 = dr.addr(q1, q2);
                        double x00 = dsm_ld(a00, 0.0), x01 = dsm_ld(a01, 0.0), x10 = dsm_ld(a10, 0.0), x11 = dsm_ld(a11, 0.0);
                        if (on1) {
                            const double sv = rs[so + e1], tauv = rtau[so + e1];
                            rot2(sv, tauv, x00, x10);
                            rot2(sv, tauv, x01, x11);
                        }
                        if (on2) {
                            const double sv = rs[so + e2], tauv = rtau[so + e2];
                            rot2(sv, tauv, x00, x01);
                            rot2(sv, tauv, x10, x11);
                        }
                        dsm_st(a00, x00);
                        dsm_st(a01, x01);
                        dsm_st(a10, x10);
                        dsm_st(a11, x11);
                    }
                    // this CTA's rows of V by round g
                    for (int it = btid; it < half * rows; it += bt) {
                        const int ee = it / rows, i = it - ee * rows;
                        if (!ron[so + ee]) continue;
                        const int p = rp[so + ee], q = rq[so + ee];
                        VT vp = Vl[i + (size_t)rows * p], vq = Vl[i + (size_t)rows * q];
                        if constexpr (kV32) rot2(rs32[so + ee], rtau32[so + ee], vp, vq);
                        else rot2(rs[so + ee], rtau[so + ee], vp, vq);
                        Vl[i + (size_t)rows * p] = vp;
                        Vl[i + (size_t)rows * q] = vq;
                    }
                }
                cluster.sync();
                ++G;
            }
            const int cnt = *cluster.map_shared_rank(&s_cntg[sw & 3], 0);
            total_rot += cnt;
            sweeps = sw + 1;
            if (cnt == 0) break;
        }
        dfin = Dh[G & 1];
        double* dlfin = Dl[G & 1];
        for (int x = tid; x < k; x += nt) dfin[x] += dlfin[x];  // hi + lo, rounded once
        __syncthreads();
    }

    // ---- permutation (identical in every CTA: same diagonal replica; the
    // QRCP order of Sec. 2.1's pivoting step is computed by rank 0 on the
    // leading rows of Vhat, gathered from the CTAs that own them, and sent
    // to every CTA)
    __shared__ int s_nr, s_r1;
    if (tid == 0) {
        int nr = 0, r1 = 0;
        for (int x = 0; x < k; ++x)
            if (pc_pair_map(I, J, b, x) < a.n_real) {
                r1 += x < b;
                s_pos[nr++] = x;
            }
        s_nr = nr;
        s_r1 = r1;
    }
    __syncthreads();
    if (a.order == 2 && total_rot > 0) {
        __shared__ int s_perm[256];
        __shared__ double s_cn[256], s_vh[128];
        const int nr = s_nr, r1 = s_r1;
        double* M = a.qrws + (size_t)e * b * k;
        for (int idx = tid; idx < r1 * nr; idx += nt) {   // this CTA's leading rows of Vhat
            const int i = idx % r1, j = idx / r1, row = s_pos[i];
            if (row >= r_lo && row < r_lo + rows) M[idx] = Vl[(row - r_lo) + (size_t)rows * s_pos[j]];
        }
        __threadfence();
        cluster.sync();
        if (r == 0) {
            qrcp_order(r1, nr, M, s_perm, s_cn, s_vh);
            for (int x = tid; x < k; x += nt) s_dest[x] = x;
            __syncthreads();
            for (int t = tid; t < nr; t += nt) s_dest[s_pos[s_perm[t]]] = s_pos[t];
            __syncthreads();
            for (int u = 1; u < C; ++u) {
                int* rd = cluster.map_shared_rank(s_dest, u);
                for (int x = tid; x < k; x += nt) rd[x] = s_dest[x];
            }
        }
        cluster.sync();
    } else {
    for (int x = tid; x < k; x += nt) {
        int dest = x;
        if (a.order == 1 && total_rot > 0 && pc_pair_map(I, J, b, x) < a.n_real) {
            const double dx = dfin[x];
            int rr = 0;
            for (int y = 0; y < k; ++y) {
                if (y == x || pc_pair_map(I, J, b, y) >= a.n_real) continue;
                const double dy = dfin[y];
                rr += (dy > dx) || (dy == dx && y < x);
            }
            dest = s_pos[rr];
        }
        s_dest[x] = dest;
    }
    __syncthreads();
    }

    // ---- outputs: this CTA's rows of V (and the matching columns of V^T)
    double* Vo = a.V + (size_t)e * 2 * k * k;
    for (int idx = tid; idx < rows * k; idx += nt) {
        const int i = idx % rows, j = idx / rows;
        const double v = Vl[idx];  // V(r_lo + i, j) -> column s_dest[j]
        Vo[(r_lo + i) + (size_t)k * s_dest[j]] = v;
        Vo[(size_t)k * k + s_dest[j] + (size_t)k * (r_lo + i)] = v;
    }
    if (a.Aout || a.Aout32) {
        for (int idx = tid; idx < k * k; idx += nt) {
            const int ii = idx % k, jj = idx / k;
            const int hi_row = ii >= jj ? ii : jj;
            if (hi_row < my_lo || hi_row >= my_hi) continue;
            const double v = ii == jj ? dfin[ii] : my_chunk[tri(hi_row) + (ii >= jj ? jj : ii) - ap.sp.base[r]];
            const size_t g = pc_pair_map(I, J, b, s_dest[ii]) + (size_t)a.ld * pc_pair_map(I, J, b, s_dest[jj]);
            if (a.Aout32) a.Aout32[g] = (float)v;
            else a.Aout[g] = v;
        }
    }
    if (r == 0 && tid == 0) {
        a.rot[e] = total_rot;
        atomicAdd(&a.cnt->rotations, (unsigned long long)total_rot);
        atomicAdd(&a.cnt->inner_sweeps, (unsigned long long)sweeps);
        if (!frozen) atomicAdd(&a.cnt->pair_solves, 1ull);
        atomicAdd(&a.cnt->flops_fp64, (unsigned long long)total_rot * (unsigned long long)((a.v32 ? 12 : 18) * k));
    }
    // no CTA may leave while others can still read its shared memory
    cluster.sync();
}

// Cluster size for a step with npairs pairs on an sms-SM GPU: the largest
// power of two C <= cmax with npairs * C <= sms whose per-CTA share fits the
// shared-memory limit, or 1 (use the one-CTA kernel).  A round's FP64 work
// per CTA shrinks with C while its cluster barrier does not, so small pivots
// gain nothing from large clusters: k <= 32 uses one CTA, k <= 128 at most 4
// (measured on GB300: n = 256, b = 16: 32 ms with one CTA, 37 ms with
// clusters of 4; the 16 Gram pivots (k = 128) of a step of the 2048-column
// SVD: 524 ms per solve with C = 4, 592 ms with 8, 758 ms with 2).
int pivot_cluster_size(int k, int npairs, int sms, size_t smem_cap)
{
    const int cmax = k <= 32 ? 1 : (k <= 128 ? 4 : PC_MAXC8);
    int best = 1;
    for (int C = 2; C <= cmax; C *= 2) {
        if (k % C || k / C < 8 || npairs * C > sms) break;
        if (pivot_cluster_smem(k, C) + 8192 <= smem_cap) best = C;   // + the static shared memory
    }
    return best;
}

// The fused schedule for pivots of order k > 128, the split one below (the
// same results bit for bit); JACOBI_PIVOT_SCHEDULE=split or =fused forces
// one.
cudaError_t launch_pivot_cluster(const PivotArgs& a, int C, const unsigned* qtab, cudaStream_t s)
{
    if (a.npairs <= 0) return cudaSuccess;
    const char* env = getenv("JACOBI_PIVOT_SCHEDULE");
    bool fused = a.k > 128;   // measured on GB300: fused 7 % faster at k = 256, 26 % slower at k = 128
    if (env && strcmp(env, "split") == 0) fused = false;
    if (env && strcmp(env, "fused") == 0) fused = true;
    void (*kern)(PivotArgs, int, const unsigned*) =
        fused ? (a.v32 ? k_pivot_cluster<true, true> : k_pivot_cluster<true, false>)
              : (a.v32 ? k_pivot_cluster<false, true> : k_pivot_cluster<false, false>);
    const size_t smem = pivot_cluster_smem(a.k, C);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (C > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.npairs * C);
    cfg.blockDim = dim3(PC_T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, C, qtab);
}

}  // namespace jac
