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
__device__ __forceinline__ void schur2_ref(T app, T aqq, T apq, T& s, T& t, T& tau)
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
__device__ __forceinline__ void schur2(T app, T aqq, T apq, T& s, T& t, T& tau)
{
    schur2_ref(app, aqq, apq, s, t, tau);
}

template <typename T>
__device__ __forceinline__ bool rotation_wanted(T app, T aqq, T apq, T tol)
{
    if (apq == T(0)) return false;
    return fabs(apq) > rn_mul(rn_mul(tol, rn_sqrt(fabs(app))), rn_sqrt(fabs(aqq)));
}

// ---------------------------------------------------------------- FP64 with few FP64 instructions
// On this part FP64 runs at 1/64 of the FP32 rate, and a correctly rounded
// FP64 division or square root is a chain of about ten dependent FP64
// instructions; the textbook rotation has four divisions and two square
// roots in series.  The FP64 overloads below take FP32 seeds (FP32 runs on
// the fast pipe) and refine them with Newton's method in FP64:
//   * t is the root of g(t) = apq t^2 + (aqq - app) t - apq with |t| <= 1
//     (the same root the textbook formula picks); the FP32 seed comes from
//     t = sgn(zeta) |2 apq| / (|d| + sqrt(d^2 + 4 apq^2)), d = aqq - app,
//     evaluated on d and apq scaled by a power of two, and Newton steps
//     t <- t - g(t) r on the scaled g use the seed's r ~ 1/g'(t) (each step
//     squares the relative error, 2^-22 -> 2^-44 -> below 2^-53);
//   * c = 1/sqrt(1 + t^2) from an FP32 reciprocal square root y0 and one
//     second-order step y = y0 (1 + h/2 + 3h^2/8), h = 1 - x y0^2;
//   * tau = s/(1 + c) with 1/(1 + c) from an FP32 reciprocal r0 and one
//     second-order step r = r0 (1 + e + e^2), e = 1 - (1 + c) r0.
// The results agree with the textbook ones to a few units in the last
// place, and c^2 + s^2 = 1 to the same order, so the rotation applied in
// Rutishauser's form stays orthogonal to working precision.
__device__ __forceinline__ int f64_biased_exp(double x) { return (__double2hiint(x) >> 20) & 0x7FF; }

__device__ __forceinline__ void schur2(double app, double aqq, double apq, double& s, double& t, double& tau)
{
    const double d = rn_sub(aqq, app);
    // scale d and apq by 2^(1022 - E'), E' = clamp(max exponent, 2, 2044): the larger lands in [0.5, 4)
    int E = max(f64_biased_exp(d), f64_biased_exp(apq));
    E = min(max(E, 2), 2044);
    // (t depends on the ratio only: the Newton steps run on the scaled values,
    // so 1/g' stays in range even for subnormal apq)
    const double sc = __hiloint2double((2045 - E) << 20, 0);
    const double ds = d * sc, as = apq * sc;
    const float d32 = (float)ds, a2 = 2.0f * (float)as;
    const bool dzero = (__double_as_longlong(d) << 1) == 0;
    const bool dneg = __double2hiint(d) < 0, aneg = __double2hiint(apq) < 0;
    const float R = sqrtf(fmaf(d32, d32, a2 * a2));
    const float sgz = (dzero || dneg == aneg) ? 1.0f : -1.0f;          // sgn(zeta), sgn(0) = +1
    const float t32 = sgz * __fdividef(fabsf(a2), fabsf(d32) + R);
    const float sgg = dzero ? (aneg ? -1.0f : 1.0f) : (dneg ? -1.0f : 1.0f);   // sign of g'(t)
    const double r = (double)__fdividef(sgg, R);                       // ~ 1/g_s'(t), g_s = g sc
    double tt = (double)t32;
    tt = fma(-fma(fma(as, tt, ds), tt, -as), r, tt);
    tt = fma(-fma(fma(as, tt, ds), tt, -as), r, tt);
    if (fabsf(a2) < 1e-30f)   // the seed lost bits (FP32 subnormal range): one more step
        tt = fma(-fma(fma(as, tt, ds), tt, -as), r, tt);
    t = tt;
    const double x = fma(tt, tt, 1.0);                                 // in [1, 2]
    const double y0 = (double)rsqrtf((float)x);
    const double h = fma(-(x * y0), y0, 1.0);
    const double c = fma(y0 * h, fma(0.375, h, 0.5), y0);
    s = tt * c;
    const double u = 1.0 + c;                                          // in (1.7, 2]
    const double r0 = (double)__fdividef(1.0f, (float)u);
    const double e = fma(-u, r0, 1.0);
    tau = s * fma(r0, fma(e, e, e), r0);
}

// |apq| > tol sqrt|app| sqrt|aqq| as apq^2 > tol^2 |app| |aqq| where every
// operand lies in [2^-400, 2^400] (no overflow or underflow in the squares;
// nonnegative doubles compare like their bit patterns), else the square-root
// form.
__device__ __forceinline__ bool rotation_wanted(double app, double aqq, double apq, double tol)
{
    if ((__double_as_longlong(apq) << 1) == 0) return false;
    const int ep = f64_biased_exp(apq), e1 = f64_biased_exp(app), e2 = f64_biased_exp(aqq);
    const bool safe = ep >= 623 && ep <= 1423 && e1 >= 623 && e1 <= 1423 && e2 >= 623 && e2 <= 1423;
    if (safe) {
        const double lhs = apq * apq, rhs = (tol * tol) * (fabs(app) * fabs(aqq));
        return __double_as_longlong(lhs) > __double_as_longlong(rhs);
    }
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
// null, in its own type TV (FP32 for a transform that only feeds the split
// low-precision products: the rotation parameters are rounded to TV once per
// use).  Returns the rotations applied; *sweeps_out = sweeps run.  On return
// the diagonal of Ap holds hi + lo rounded once.  Caller: all threads, after
// Ap, V (= I) and sm.dlo (= 0) are initialised and synchronised.
template <typename T, typename TV = T>
__device__ int jacobi_solve(T* Ap, TV* V, int k, T tol, int max_sweeps, const unsigned* qtab,
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
                    TV vp = V[row + (size_t)p * k], vq = V[row + (size_t)q * k];
                    rot2((TV)sm.s[ee], (TV)sm.tau[ee], vp, vq);
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
