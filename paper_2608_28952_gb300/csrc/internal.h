// internal.h -- declarations shared by the translation units of the GB300
// Jacobi library (kernels, host driver, C ABI).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>

#include "../../include/jacobi.h"

namespace jac {

// ----------------------------------------------------------------- ordering
// A sweep's ordering: steps[s] is a list of disjoint 0-based block pairs
// (I < J).  Round-robin is the default; anti-diagonal is Algorithm 3.
struct Ordering {
    int N = 0;                    // blocks (after padding)
    int S = 0;                    // steps per sweep
    std::vector<int> step_ptr;    // S + 1 offsets into pairs (in pairs)
    std::vector<int> pairs;       // 2 ints per pair
    int max_pairs = 0;            // largest step
    // Device schedule: exactly N/2 entries per step.  Steps of Algorithm 3
    // that leave two blocks out get an extra "frozen" entry holding them
    // (stored as {-1-I, -1-J}); its transform is the identity.
    std::vector<int> dev_pairs;
    int dev_per_step = 0;
};
int padded_blocks(int n, int b, int ordering);
bool make_ordering(int kind, int N, Ordering* out);

// ----------------------------------------------------------------- device data
// Counters accumulated on the device (integers only: deterministic).
struct DevCounters {
    unsigned long long rotations;
    unsigned long long inner_sweeps;
    unsigned long long pair_solves;
    unsigned long long flops_fp64;   // issued update + pivot flops
    unsigned long long flops_update; // of which in the update (and Gram) kernels
    unsigned long long flops_fp32;
    unsigned long long flops_lowp;
    int nonfinite;                   // input scan flag
    int pad_;
};

// ----------------------------------------------------------------- launchers (FP64 path)
// Each returns the cudaError_t of its launch.

// A_w <- mirrored lower triangle of A (n x n, lda), zero padded to np; Q_w <- I
// (or the caller's Q with identity on the pads when warm).  Flags non-finite
// input in cnt->nonfinite.
cudaError_t launch_load_sym(int n, int np, const double* A, int lda, double* Aw,
                            const double* Qin, int ldq, double* Qw, int warm,
                            DevCounters* cnt, cudaStream_t s);

// Sum of squares of the off-diagonal (and, separately, all) entries of the
// np x np matrix Aw, and max_{i!=j}|a_ij|/sqrt(|a_ii a_jj|).  Deterministic
// two-level reduction; result[0] = off^2, result[1] = ||A||_F^2,
// result[2] = relative measure.  partial must hold 3 * reduce_blocks doubles.
int reduce_blocks_for(int np);
cudaError_t launch_offnorm(int np, const double* Aw, double* partial, unsigned int* ticket,
                           double* result, bool want_rel, cudaStream_t s);
// The same reduction on an n x n matrix with leading dimension ld.
cudaError_t launch_offnorm_ld(int n, const double* A, int ld, double* partial, unsigned int* ticket,
                              double* result, bool want_rel, cudaStream_t s);

// Pivot solves of one step (one CTA per pair): reads Ain's pivot blocks
// (EVD) or sums the Gram partials (SVD), runs the FP64 inner Jacobi, writes
// V (and V^T) per pair, D into Aout's pivot blocks (EVD), the rotation count
// per pair and, for the SVD, the pre-rotation max normalised off-diagonal.
struct PivotArgs {
    const double* Ain;         // EVD: working A (np x np, ld np); SVD: null
    double* Aout;              // EVD: next working A (pivot blocks written)
    const float* Ain32;        // mixed form: FP32 working A instead of Ain
    float* Aout32;             // mixed form: FP32 next A instead of Aout
    int ld;                    // np
    const double* gram;        // SVD: Gram partials [pair][panel][k*k] or null
    int npanels;
    const int2* pairs;         // this step's pairs
    int npairs;
    int b, k;
    double* V;                 // [pair][2][k*k]: V then V^T, column-major
    int v32;                   // accumulate V in FP32 (its output values are FP32 numbers):
                               // only for a V consumed by the split low-precision products
    int* rot;                  // [pair] rotations applied (0 => V == I)
    double* relmax;            // [pair] (SVD) pre-rotation max normalised off-diag
    double tol_rel;
    int max_sweeps;
    int order;                 // 1: sort eigenpairs descending over real rows
    int n_real;                // rows/columns >= n_real are zero padding
    double* gscratch;          // k > 128: per-pair global scratch (packed A + V)
    double* qrws;              // order == 2: per-pair QRCP scratch, b x k doubles each
    DevCounters* cnt;
};
cudaError_t launch_pivot(const PivotArgs& a, cudaStream_t s);
// The same pivot solves with a cluster of C CTAs per pair (C from
// pivot_cluster_size; C == 1 means: use launch_pivot).  qtab: quad table
// for half = 128 (device, from launch_quad_table).
int pivot_cluster_size(int k, int npairs, int sms, size_t smem_cap);
size_t pivot_cluster_smem(int k, int C);
cudaError_t launch_pivot_cluster(const PivotArgs& a, int C, const unsigned* qtab, cudaStream_t s);
cudaError_t launch_quad_table(unsigned* qtab, int h, cudaStream_t s);
size_t pivot_gscratch_doubles(int k);   // per pair, 0 when shared memory suffices

// Update of one step (EVD): sandwich items A'_{P1P2} = V1^T A_{P1P2} V2 for
// P1 < P2 (written with their mirror), Q column items Q'(:,P) = Q(:,P) V_P.
struct UpdateArgs {
    const double* Ain; double* Aout; int lda;   // np x np, double-buffered
    const double* Qin; double* Qout; int ldq;   // rows x np, double-buffered (may be null)
    int qrows;                                  // rows of Q (np)
    const int2* pairs; int npairs;
    int b, k;
    const double* V; const int* rot;
    DevCounters* cnt;
};
cudaError_t launch_update_evd(const UpdateArgs& a, cudaStream_t s);

// One-sided update: G'(:,P) = G(:,P) V_P (m rows) and V'(:,P) = V(:,P) V_P.
struct ColUpdateArgs {
    const double* Gin; double* Gout; int ldg; int m;
    const double* Vin; double* Vout; int ldv; int vrows;
    const int2* pairs; int npairs;
    int b, k;
    const double* Vh; const int* rot;
    DevCounters* cnt;
};
cudaError_t launch_update_cols(const ColUpdateArgs& a, cudaStream_t s);

// Gram partials of one step: for each pair P and row panel r,
// part[P][r] = G(rows_r, P)^T G(rows_r, P) (k x k).
int gram_panels_for(int m);
int gram_panel_rows();
cudaError_t launch_gram(const double* G, int ldg, int m, const int2* pairs, int npairs, int b,
                        int k, double* part, DevCounters* cnt, cudaStream_t s);

// Finalisation (EVD): w <- sorted diag(Aw)[0:n] (ascending, stable), Q(:, j)
// <- Qw(0:n, perm j), A <- Aw(0:n, 0:n).
cudaError_t launch_finalize_evd(int n, int np, const double* Aw, const double* Qw, double* w,
                                double* Q, int ldq, double* A, int lda, int* rank_ws,
                                cudaStream_t s);
// Finalisation (SVD): sigma_j = ||G(:,j)||, U = G Sigma^+, sorted descending.
cudaError_t launch_finalize_svd(int m, int n, const double* Gw, int ldgw, const double* Vw,
                                int ldvw, double* U, int ldu, double* sigma, double* V, int ldv,
                                double* norms_ws, int* rank_ws, cudaStream_t s);
// Copy G (m x n, ldg) into Gw (m x np, ld m) with zero pad columns; Vw <- I.
cudaError_t launch_load_svd(int m, int n, int np, const double* G, int ldg, double* Gw,
                            double* Vw, DevCounters* cnt, cudaStream_t s);
// Max over pairs of relmax[0..npairs) into *out (max with its prior value).
cudaError_t launch_max_into(const double* relmax, int npairs, double* out, cudaStream_t s);
// Householder QR (blocked, compact WY; panels of QR_NB columns), see k_qr.cu.
constexpr int QR_NB = 32;
size_t qr_wpart_doubles(int m, int n);
// Panel [j0, j0 + nbp) of A (m rows): reflectors into Y (ld ldy), tau, the
// panel's T and T^T (QR_NB x QR_NB); S: QR_NB x QR_NB scratch.
cudaError_t launch_house_panel(int m, double* A, int lda, int j0, int nbp, double* Y, int ldy, double* tau,
                               double* S, double* T, double* Tt, cudaStream_t s);
// X(j0:m, 0:ncol) <- X - Y_p M (Y_p^T X): M = T^T (trans) or T.  Wpart:
// qr_wpart_doubles(m, ncol); W: QR_NB x ncol; YT: m x QR_NB.
cudaError_t launch_house_update(int m, int j0, int nbp, const double* Y, int ldy, const double* T,
                                const double* Tt, int trans, double* X, int ldx, int ncol, double* Wpart,
                                double* W, double* YT, cudaStream_t s);
// The same with FP64-accurate tensor-core products (xA, xB: m + n ints; err: timeout word).
cudaError_t launch_house_update_emu(int m, int j0, int nbp, const double* Y, int ldy, const double* T,
                                    const double* Tt, int trans, double* X, int ldx, int ncol, double* part,
                                    double* W, double* YT, int* xA, int* xB, int* err, cudaStream_t s);
cudaError_t launch_qr_rt(int n, const double* A, int lda, double* X, cudaStream_t s);
cudaError_t launch_qr_fill(int m, int n, const double* W, double* G, int ldg, cudaStream_t s);
cudaError_t launch_rotation_params(int count, const double* app, const double* aqq, const double* apq, double tol,
                                   double* out, cudaStream_t s);

// ----------------------------------------------------------------- mixed form (tensor cores)
// One low-precision step's updates on FP32 working copies: stage 1
// T_pb = A_{P1P2} V2 (all pair-blocks P1 < P2) and Q'(:,P) = Q(:,P) V_P,
// stage 2 A'_{P1P2} = V1^T T_pb with its mirror; products from bf16 hi/lo
// splits on tcgen05.  The pivot blocks are written by the pivot kernel.
struct TcUpdArgs {
    const float* Ain; float* Aout; int lda;     // np x np FP32, double-buffered
    const float* Qin; float* Qout; int ldq; int qrows;
    float* T;                                   // [npb][k*k] stage-1 products
    const int2* pairs; int npairs; int b, k;
    const double* V; const int* rot;            // pivot kernel outputs (FP64 V, V^T)
    unsigned char* vimg;                        // per pair: V split into hi/lo operand tiles
    unsigned* tmax;                             // FP16x3: per pair-block column maxima of T
    int kind;                                   // 0: bf16 hi/lo, 1: fp16 hi/lo (scaled), 2: tf32 big/small
    int* err;                                   // set on a timed-out tensor-core wait
    DevCounters* cnt;
};
// Launches the V split and the two stages.  T needs tc_update_tbuf_floats,
// vimg tc_update_vimg_bytes (both for the step's entry count and k).
cudaError_t launch_tc_update(const TcUpdArgs& a, cudaStream_t s);
size_t tc_update_tbuf_floats(int npairs, int k);
size_t tc_update_vimg_bytes(int npairs, int k);
size_t tc_update_tmax_words(int npairs, int k);

// FP64-accurate product on the bf16 tensor cores (slices, K <= 256):
// C (M x N) = op(A) B, column-major FP64.
cudaError_t launch_emu_gemm(int M, int N, int K, const double* A, int lda, int transA, const double* B, int ldb,
                            double* C, int ldc, int* err, cudaStream_t s);
// The same product for any K (exact FP32 accumulation per 256 K values,
// 64-bit integer running sums): C = op(A) B, or C += op(A) B when
// accumulate; tiles wholly above the diagonal skipped when lower.  xA, xB:
// int workspace of M and N entries (line exponents).
cudaError_t launch_emu_gemm_big(int M, int N, int K, const double* A, int lda, int transA, const double* B, int ldb,
                                int accumulate, double* C, int ldc, int lower, int* xA, int* xB, int* err,
                                cudaStream_t s);
// The same product with both operands sliced once into images (imgA:
// emu_gemm_img_bytes(M, K) bytes, imgB: emu_gemm_img_bytes(N, K)) that the
// tiles stage by bulk copies, instead of every tile slicing its operands.
size_t emu_gemm_img_bytes(int lines, int K);
cudaError_t launch_emu_gemm_img(int M, int N, int K, const double* A, int lda, int transA, const double* B, int ldb,
                                int accumulate, double* C, int ldc, int lower, int* xA, int* xB,
                                unsigned char* imgA, unsigned char* imgB, int* err, cudaStream_t s);
// W (N x M, ld ldw) = (op(A) B)^T with K split into chunks of kchunk: the
// partials (part: ceil(K / kchunk) x M x N doubles) summed in a fixed order.
cudaError_t launch_emu_gemm_tsplit(int M, int N, int K, const double* A, int lda, int transA, const double* B, int ldb,
                                   double* W, int ldw, int kchunk, double* part, int* xA, int* xB, int* err,
                                   cudaStream_t s);
// The step update of the FP64 path with every product FP64-accurate on the
// tensor cores (stage 1 T = A_{P1P2} V2 and Q V_P, stage 2 V1^T T mirrored).
struct EmuUpdArgs {
    UpdateArgs u;
    double* T;      // [npb][k*k]
    int* err;       // set on a timed-out tensor-core wait
    // 1: balance the pair-blocks' columns by powers of two from the diagonal
    // (graded positive definite inputs under the relative stop criterion)
    int balance = 0;
    // optional: the step's V sliced once into eight bf16 digit images
    // (emu_update_vimg_bytes) and its column scales (emu_update_vexp_ints);
    // the update tiles then stage V's slices by bulk copies instead of
    // slicing V themselves
    unsigned char* vimg = nullptr;
    int* vexp = nullptr;
    // optional (with vimg, without balance): the step's stage-1 operands
    // sliced once as well -- every off-diagonal pair-block A_{P1P2} with its
    // row scales over P2 (aimg, atab), every column pair Q(:, P) with its row
    // scales over P (qimg, qtab) -- so the stage-1 tiles slice nothing
    unsigned char* aimg = nullptr;
    int* atab = nullptr;
    unsigned char* qimg = nullptr;
    int* qexp = nullptr;
};
cudaError_t launch_emu_update(const EmuUpdArgs& a, cudaStream_t s);
size_t emu_update_vimg_bytes(int npairs, int k);
size_t emu_update_vexp_ints(int npairs, int k);
size_t emu_update_aimg_bytes(int npairs, int k);
size_t emu_update_qimg_bytes(int npairs, int k, int qrows);
// The one-sided step's products FP64-accurate on the tensor cores: Gram
// partials per pair and row panel (the layout the pivot kernel reads), and
// the column update of G and V.
struct EmuSvdArgs {
    const double* Gin; double* Gout; int ldg; int m;
    const double* Vin; double* Vout; int ldv; int vrows;
    const int2* pairs; int npairs;
    int b, k;
    const double* Vh; const int* rot;
    double* part; int npanels; int panel_rows;
    int* err;
    DevCounters* cnt;
};
cudaError_t launch_emu_gram(const EmuSvdArgs& a, cudaStream_t s);
cudaError_t launch_emu_cols(const EmuSvdArgs& a, cudaStream_t s);
size_t emu_update_tbuf_doubles(int npairs, int k);
cudaError_t launch_offnorm32(int np, const float* Aw, double* partial, unsigned int* ticket,
                             double* result, cudaStream_t s);
// C = alpha op(A) B + beta C (FP64, column-major); lower = 1 computes only
// the tiles that meet the lower triangle (for a symmetric product; mirror
// afterwards with launch_mirror_lower).
cudaError_t launch_gemm64(int M, int N, int K, double alpha, const double* A, int lda, int transA,
                          const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t s,
                          int lower = 0);
cudaError_t launch_mirror_lower(int n, double* C, int ldc, cudaStream_t s);
cudaError_t launch_load_sym32(int n, int np, const double* A, int lda, float* A32, float* Q32,
                              DevCounters* cnt, cudaStream_t s);
cudaError_t launch_pad_sym64(int n, int np, const double* A, int lda, double* A0p, cudaStream_t s);
cudaError_t launch_f32_to_f64(long long count, const float* x, double* y, cudaStream_t s);
cudaError_t launch_oa_step_elementwise(int np, const double* S, double* G, double* lam, double eta,
                                       cudaStream_t s);
cudaError_t launch_symmetrize(int np, const double* S, double* B, cudaStream_t s);
cudaError_t launch_ns_halfres(int np, double* G, cudaStream_t s);

}  // namespace jac
