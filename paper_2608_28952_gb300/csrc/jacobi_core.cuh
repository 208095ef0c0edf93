// jacobi_core.cuh -- the scalar parallel-ordered Jacobi solve of one symmetric
// k x k matrix by one CTA, shared by the pivot kernel of the blocked method
// (FP64) and the batched kernels (FP32 and FP64).
//
// The solve is Algorithm 2 applied with block size 1: each sweep is k-1
// rounds of the round-robin order over the k indices; a round computes the
// k/2 textbook 2x2 Schur rotations from the round's starting values, rotates
// every disjoint 2x2 "quad" (rows of pair e1, columns of pair e2) from both
// sides, sets each rotated 2x2 pivot to its exact diagonal form and rotates
// the columns of V.  The symmetric matrix lives in packed lower-triangular
// form; the diagonal is carried as hi (in the packed array) + lo.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace jac {

__device__ __forceinline__ int tri(int i) { return (i * (i + 1)) >> 1; }
__device__ __forceinline__ int sidx(int i, int j) { return i >= j ? tri(i) + j : tri(j) + i; }

// ---------------------------------------------------------------- correctly rounded ops
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double rn_sqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float rn_sqrt(float a) { return __fsqrt_rn(a); }

template <typename T>
struct Lim;
template <>
struct Lim<double> {
    static constexpr double big = 1e150;   // 1 + zeta^2 would overflow beyond this
};
template <>
struct Lim<float> {
    static constexpr float big = 1e18f;
};

// The textbook 2x2 symmetric Schur rotation: zeta = (aqq - app)/(2 apq),
// t = sgn(zeta)/(|zeta| + sqrt(1 + zeta^2)) with sgn(0) = +1, c = 1/sqrt(1+t^2),
// s = t c; J = [[c, s], [-s, c]] makes J^T [[app, apq], [apq, aqq]] J diagonal
// with diagonal (app - t apq, aqq + t apq).  Every operation is rounded
// separately (no contraction).  Returns s, t and tau = s/(1+c).
template <typename T>
__device__ __forceinline__ void schur2(T app, T aqq, T apq, T& s, T& t, T& tau)
{
    const T zeta = rn_div(rn_sub(aqq, app), rn_mul(T(2), apq));
    if (fabs(zeta) > Lim<T>::big) {
        t = rn_div(T(0.5), zeta);
    } else {
        const T r = rn_sqrt(rn_add(T(1), rn_mul(zeta, zeta)));
        t = rn_div(zeta >= T(0) ? T(1) : T(-1), rn_add(fabs(zeta), r));
    }
    const T c = rn_div(T(1), rn_sqrt(rn_add(T(1), rn_mul(t, t))));
    s = rn_mul(t, c);
    tau = rn_div(s, rn_add(T(1), c));
}

template <typename T>
__device__ __forceinline__ bool rotation_wanted(T app, T aqq, T apq, T tol)
{
    if (apq == T(0)) return false;
    return fabs(apq) > rn_mul(rn_mul(tol, rn_sqrt(fabs(app))), rn_sqrt(fabs(aqq)));
}

// (x, y) <- (c x - s y, s x + c y) in Rutishauser's form with tau = s/(1+c):
// x - s (y + tau x), y + s (x - tau y).  Rounding is relative to the
// correction, so vectors keep their length for the small angles of late
// sweeps (where the computed (c, s) have c^2 + s^2 = 1 + u on average).
template <typename T>
__device__ __forceinline__ void rot2(T s, T tau, T& x, T& y)
{
    const T a = x, b = y;
    x = fma(-s, fma(tau, a, b), a);
    y = fma(s, fma(-tau, b, a), b);
}

// (hi, lo) += sgn * t * apq with the product formed exactly (fma) and added
// by an error-free two-sum: the diagonal is carried as hi + lo so that
// rotations whose diagonal change is below half an ulp still move the energy
// of the zeroed entry into the diagonal.
template <typename T>
__device__ __forceinline__ void dd_add_prod(T& hi, T& lo, T t, T apq, T sgn)
{
    T dh = rn_mul(t, apq);
    T dl = fma(t, apq, -dh);
    dh *= sgn;
    dl *= sgn;
    const T a = hi, sum = rn_add(a, dh);
    const T bb = rn_sub(sum, a);
    T err = rn_add(rn_sub(a, rn_sub(sum, bb)), rn_sub(dh, bb));
    err = rn_add(err, rn_add(lo, dl));
    const T h2 = rn_add(sum, err);
    lo = rn_sub(err, rn_sub(h2, sum));
    hi = h2;
}

// Shared scratch of one solve (size k/2 arrays unless noted).
template <typename T>
struct CoreSmem {
    T* tau;
    T* s;
    T* t;
    T* apq;
    T* dlo;        // k entries
    int* p;
    int* q;
    int* on;
    int* cnt;      // one int: rotations of the current sweep
};

// Quad (e1, e2), e1 < e2 < half, of flat index qi = e2 (e2 - 1) / 2 + e1.
__device__ __forceinline__ void quad_of(const unsigned* qtab, int qi, int& e1, int& e2)
{
    const unsigned qq = qtab[qi];
    e1 = qq & 0xffff;
    e2 = qq >> 16;
}

// Solve the packed symmetric k x k matrix Ap (k even) in place by blockDim.x
// threads.  V (k x k, column-major, ld k) accumulates the rotations when not
// null.  Returns the rotations applied; *sweeps_out = sweeps run.  On return
// the diagonal of Ap holds hi + lo rounded once.  Caller: all threads, after
// Ap, V (= I) and sm.dlo (= 0) are initialised and synchronised.
template <typename T>
__device__ int jacobi_solve(T* Ap, T* V, int k, T tol, int max_sweeps, const unsigned* qtab,
                            const CoreSmem<T>& sm, int* sweeps_out)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int half = k >> 1, nq = half * (half - 1) / 2;
    int total_rot = 0, sweeps = 0;
    for (int sw = 0; sw < max_sweeps; ++sw) {
        if (tid == 0) *sm.cnt = 0;
        __syncthreads();
        for (int r = 0; r < k - 1; ++r) {
            for (int ee = tid; ee < half; ee += nt) {
                const int pa = ee, pb = k - 1 - ee;
                const int ia = pa == 0 ? 0 : 1 + (pa - 1 + r) % (k - 1);
                const int ib = 1 + (pb - 1 + r) % (k - 1);
                const int p = ia < ib ? ia : ib, q = ia < ib ? ib : ia;
                const T app = Ap[tri(p) + p], aqq = Ap[tri(q) + q], apq = Ap[tri(q) + p];
                const bool on = rotation_wanted(app, aqq, apq, tol);
                sm.p[ee] = p;
                sm.q[ee] = q;
                sm.on[ee] = on;
                if (on) {
                    T s, t, tau;
                    schur2(app, aqq, apq, s, t, tau);
                    sm.tau[ee] = tau;
                    sm.s[ee] = s;
                    sm.t[ee] = t;
                    sm.apq[ee] = apq;
                    atomicAdd(sm.cnt, 1);
                }
            }
            __syncthreads();
            for (int qi = tid; qi < nq; qi += nt) {  // both-sided rotation of every quad
                int e1, e2;
                quad_of(qtab, qi, e1, e2);
                const int on1 = sm.on[e1], on2 = sm.on[e2];
                if (!(on1 | on2)) continue;
                const int p1 = sm.p[e1], q1 = sm.q[e1], p2 = sm.p[e2], q2 = sm.q[e2];
                const int i00 = sidx(p1, p2), i01 = sidx(p1, q2), i10 = sidx(q1, p2),
                          i11 = sidx(q1, q2);
                T x00 = Ap[i00], x01 = Ap[i01], x10 = Ap[i10], x11 = Ap[i11];
                if (on1) {  // rows: J1^T X
                    const T s = sm.s[e1], tau = sm.tau[e1];
                    rot2(s, tau, x00, x10);
                    rot2(s, tau, x01, x11);
                }
                if (on2) {  // columns: X J2
                    const T s = sm.s[e2], tau = sm.tau[e2];
                    rot2(s, tau, x00, x01);
                    rot2(s, tau, x10, x11);
                }
                Ap[i00] = x00;
                Ap[i01] = x01;
                Ap[i10] = x10;
                Ap[i11] = x11;
            }
            for (int ee = tid; ee < half; ee += nt) {  // exact 2x2 diagonal form
                if (!sm.on[ee]) continue;
                const int p = sm.p[ee], q = sm.q[ee];
                T hp = Ap[tri(p) + p], hq = Ap[tri(q) + q];
                dd_add_prod(hp, sm.dlo[p], sm.t[ee], sm.apq[ee], T(-1));
                dd_add_prod(hq, sm.dlo[q], sm.t[ee], sm.apq[ee], T(1));
                Ap[tri(p) + p] = hp;
                Ap[tri(q) + q] = hq;
                Ap[tri(q) + p] = T(0);
            }
            if (V) {
                for (int it = tid; it < half * k; it += nt) {  // V <- V J
                    const int ee = it / k, row = it - ee * k;
                    if (!sm.on[ee]) continue;
                    const int p = sm.p[ee], q = sm.q[ee];
                    T vp = V[row + (size_t)p * k], vq = V[row + (size_t)q * k];
                    rot2(sm.s[ee], sm.tau[ee], vp, vq);
                    V[row + (size_t)p * k] = vp;
                    V[row + (size_t)q * k] = vq;
                }
            }
            __syncthreads();
        }
        const int cnt = *sm.cnt;
        total_rot += cnt;
        sweeps = sw + 1;
        __syncthreads();
        if (cnt == 0) break;
    }
    for (int x = tid; x < k; x += nt) Ap[tri(x) + x] += sm.dlo[x];  // hi + lo, rounded once
    __syncthreads();
    *sweeps_out = sweeps;
    return total_rot;
}

// Flat quad table for half-size h: entries e1 | e2 << 16 for e1 < e2 < h,
// ordered by e2 then e1 (so a table for h serves every smaller size too).
__device__ __forceinline__ void build_quad_table(unsigned* qtab, int h)
{
    for (int e2 = 1 + threadIdx.x; e2 < h; e2 += blockDim.x)
        for (int e1 = 0; e1 < e2; ++e1) qtab[(e2 * (e2 - 1) >> 1) + e1] = (unsigned)e1 | ((unsigned)e2 << 16);
}

}  // namespace jac
