/*
 * jacobi.h -- C ABI of the GB300 (sm_103a) blocked Jacobi library.
 *
 * The method is the blocked Jacobi algorithm for the symmetric eigenvalue
 * problem A = Q D Q^T and the one-sided Jacobi SVD G = U Sigma V^T analysed in
 * Demmel, Luo, Schneider & Wang, "Minimizing the Arithmetic and Communication
 * Complexity of Jacobi's Method for Eigenvalues and Singular Values: Part Two
 * -- Parallel Algorithms".  Each step of a sweep pairs the N = n/b blocks into
 * N/2 disjoint pairs (Sec. 3, item 1), solves every 2b x 2b pivot subproblem,
 * and applies the orthogonal transforms to A and Q (Algorithms 1 and 2) or to
 * the column pairs of G and V (Algorithm 6).
 *
 * Conventions (all entry points):
 *   - matrices are column-major with a leading dimension (lda, ldq, ...);
 *   - pointers are DEVICE pointers unless the entry point name ends in "_h"
 *     (host pointers) or the argument is named h_*;
 *   - the caller owns every buffer; the library allocates its workspace with
 *     cudaMallocAsync on the given stream and frees it before returning;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); the calls return only after the work is complete;
 *   - nothing is printed, nothing throws, nothing exits;
 *   - return value: 0 converged, >0 the sweep count when max_sweeps ran out
 *     (outputs then hold the current iterate), <0 an error (JACOBI_ERR_* or
 *     -k for an invalid k-th argument);
 *   - the pivot solves of a step with few pairs run with a thread-block
 *     cluster of up to 8 CTAs per pair (chosen automatically); the
 *     environment variable JACOBI_PIVOT_CLUSTER=1 forces one CTA per pair,
 *     =2/4/8 that cluster size where it fits.
 *
 * Environment switches (read at each call; none is needed):
 *   JACOBI_PIVOT_CLUSTER=1|2|4|8   pivot cluster size (above);
 *   JACOBI_BATCHED_LARGE=blocked|cluster|l2   route of the batched EVD
 *                                  orders above the shared-memory size
 *                                  (default blocked);
 *   JACOBI_BATCHED_SVD=rowwise     the batched one-sided SVD with one Gram
 *                                  entry per thread instead of staged row
 *                                  tiles (same results bit for bit);
 *   JACOBI_PIVOT_SCHEDULE=split|fused  round schedule of the cluster pivot
 *                                  solves (default: fused for 2b > 128,
 *                                  split below; the same results bit for
 *                                  bit);
 *   JACOBI_EMU_IMAGE=0             the emulated FP64 products slice their
 *                                  operands in every tile instead of once
 *                                  into an image (V per step in the update,
 *                                  both operands of a refinement product;
 *                                  the same results bit for bit);
 *   JACOBI_TUNE_CACHE=<path>       file of the batched autotuner's cache;
 *   JACOBI_WORKSPACE_LIMIT=<bytes> cap on one call's workspace (fault
 *                                  injection: JACOBI_ERR_ALLOC before any
 *                                  launch).
 */
#ifndef JACOBI_GB300_H
#define JACOBI_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ codes */
#define JACOBI_OK 0
#define JACOBI_ERR_NONFINITE (-100) /* NaN or Inf in the input                     */
#define JACOBI_ERR_CUDA (-101)      /* a CUDA runtime call failed                  */
#define JACOBI_ERR_ALLOC (-102)     /* workspace allocation failed                 */
#define JACOBI_ERR_TIMEOUT (-103)   /* a bounded device wait ran out               */
#define JACOBI_ERR_UNSUPPORTED (-104) /* valid but not supported (e.g. b > 128)    */

/* Orderings of the pairs within a sweep (Sec. 3).
 *  ROUND_ROBIN: tournament; block 0 fixed, positions 1..N-1 rotate by one per
 *               step, step s pairs position j with position N-1-j (N even).
 *  ANTI_DIAGONAL: Algorithm 3, group K = {(I,J): I<J, (I+J) mod N = K}
 *               (1-based I,J), groups emitted for K = 0..N-1. */
#define JACOBI_ORDER_ROUND_ROBIN 0
#define JACOBI_ORDER_ANTI_DIAGONAL 1

/* Arithmetic of the update GEMMs.  Pivot solves, the off-norm test and the
 * closing sweeps are FP64 in every mode.
 *  FP64:          DFMA throughout.
 *  FP32:          the batched forms' FP32 storage and arithmetic.
 *  MIXED_BF16X3:  low-precision sweeps on FP32 working copies, products on the
 *                 tensor cores from bf16 hi/lo splits (three products), then
 *                 the FP64 refinement and closing sweeps (jacobi_syev).  In
 *                 the low-precision sweeps the pivot solves (matrix, diagonal,
 *                 rotation parameters) stay FP64 and accumulate each pivot's
 *                 transform V in FP32, the precision the products take it in.
 *  MIXED_FP16X3:  the same with fp16 hi/lo splits (22 bits per operand), the
 *                 FP32 operands scaled by powers of two per row / column.
 *  MIXED_TF32:    the same with tf32 big/small splits (x = big + small, big =
 *                 x with its low 13 mantissa bits cleared; kind::tf32).
 *  FP64_EMU:      the plain FP64 method with every update product formed
 *                 FP64-accurately on the bf16 tensor cores (eight 7-bit slices
 *                 per operand, see jacobi_f64emu_gemm); pivots, off-norm and
 *                 everything else as FP64.  jacobi_syev and jacobi_syev_step. */
#define JACOBI_PREC_FP64 0
#define JACOBI_PREC_FP32 1
#define JACOBI_PREC_MIXED_BF16X3 2
#define JACOBI_PREC_MIXED_FP16X3 3
#define JACOBI_PREC_MIXED_TF32 4
#define JACOBI_PREC_FP64_EMU 5

/* Stop criteria.
 *  OFF_ABS: Xi(A) = sqrt(sum_{i!=j} a_ij^2) <= tol * ||A||_F (Sec. 2.1,
 *           eq. (Omega_A)); ||A||_F is taken once from the input.
 *  REL:     max_{i!=j} |a_ij| / sqrt(|a_ii| |a_jj|) <= tol. */
#define JACOBI_CONV_OFF_ABS 0
#define JACOBI_CONV_REL 1

typedef struct {
    int b;                /* block size, 1 <= b <= 128; n need not be a multiple
                             (zero padding, exact: a zero row and column is
                             never rotated)                                    */
    int ordering;         /* JACOBI_ORDER_*                                     */
    int max_sweeps;       /* outer sweep cap (default 60: graded spectra with
                             closely spaced eigenvalues converge linearly for
                             many sweeps, e.g. 30 at n = 4096, b = 64 with
                             lambda_i = +-10^(-12 i/(n-1)))                     */
    int inner_max_sweeps; /* cap on the sweeps of one pivot solve; a small cap
                             gives the approximate solve the paper allows
                             (Sec. 3, after Algorithm 3).  0 (default) =
                             automatic: 1 for the two-sided EVD (same outer
                             sweep count, half the time at n = 4096), 30 for
                             the one-sided SVD on G (a cap there costs
                             sweeps), 2 for the SVD on R^T (svd_qr: the same
                             sweeps with half the inner sweeps)              */
    double tol;           /* outer tolerance (default 1e-14; SVD: see gesvd)    */
    double inner_tol;     /* a scalar rotation inside a pivot solve is skipped
                             when |a_pq| <= inner_tol sqrt|a_pp| sqrt|a_qq|
                             (default 4 * 2^-53)                                */
    int precision;        /* JACOBI_PREC_* (default FP64)                       */
    int conv;             /* JACOBI_CONV_* (default OFF_ABS)                    */
    int want_vectors;     /* 1: accumulate Q / V (default 1)                    */
    int warm_start;       /* 1: Q (or V) holds an orthogonal start: resume
                             from the caller's (A, Q); 0: start from Q = I      */
    double switch_tol;    /* mixed forms: leave the low-precision sweeps when
                             off(A_w) <= switch_tol ||A||_F (0 = default)        */
    int refine_steps;     /* mixed forms: FP64 refinement steps (default 1)     */
    int pivot_order;      /* permutation after each pivot solve, Qhat <- Qhat P
                             (the slot of the pivoting step, Sec. 2.1):
                             0 = eigenpairs as solved (the pseudocode of
                             Algorithms 1, 2 and 6); 1 = sorted by descending
                             eigenvalue over the pivot's non-padding rows
                             (default; far fewer sweeps on graded spectra);
                             2 = the order column-pivoted QR picks on the
                             leading rows of Qhat (the pivoting step of
                             Sec. 2.1, the condition of Drmac's convergence
                             proof)                                            */
    int fp64_products;    /* how the FP64 sweeps form their update products:
                             0 = FP64 FMA (default); 1 = FP64-accurate products
                             on the bf16 tensor cores as in
                             JACOBI_PREC_FP64_EMU (b <= 128).  Applies to the
                             plain FP64 solve and to the closing sweeps of the
                             mixed forms                                       */
    int svd_qr;           /* jacobi_gesvd: 1 = factor G = QR first (Householder,
                             blocked) and run the one-sided method on R^T,
                             U = Q times its rotations, V = its normalised
                             columns (Sec. 6, "Preprocessing with QR");
                             0 = directly on G (default)                       */
} jacobi_params;

typedef struct {
    int status;              /* the return code                                */
    int sweeps;              /* outer sweeps run (all precisions)              */
    int sweeps_lowp;         /* of which in the low-precision phase (mixed)    */
    int stalled;             /* stopped by the stall rule                      */
    long long steps;         /* parallel steps run                             */
    long long pair_solves;   /* 2b x 2b pivot solves                           */
    long long rotations;     /* scalar rotations applied inside pivot solves   */
    long long inner_sweeps;  /* sum over pivot solves of their sweeps          */
    double norm_fro;         /* ||A||_F of the input (EVD)                      */
    double off_initial;      /* Xi(A) of the input (EVD) / first sweep's max
                                normalised Gram off-diagonal (SVD)              */
    double off_final;        /* same measure at exit                           */
    double off_hist[64];     /* per sweep                                      */
    double ms_total;         /* device time of the call (CUDA events)          */
    double ms_pivot;         /* device time in the pivot-solve kernels         */
    double ms_update;        /* device time in the update kernels (A and Q /
                                G and V; for the SVD including the Gram)        */
    long long launches;      /* kernels this call launched                     */
    long long pivot_launches;  /* of which pivot-solve kernels                 */
    long long update_launches; /* of which update kernels                      */
    double flops_fp64;       /* FP64 flops issued (updates + pivot solves; a
                                V accumulated in FP32 is not counted)          */
    double flops_update;     /* of which in the update / Gram kernels          */
    double flops_fp32;       /* FP32 flops issued                              */
    double flops_lowp;       /* bf16 / fp16 / tf32 tensor flops issued         */
    double ms_lowp;          /* mixed forms: device time of the low-precision
                                sweeps (pivot solves included)                 */
    double ms_refine;        /* mixed forms: device time of the return to FP64
                                (re-orthogonalisation, refinement, S = X^T A X) */
    double ms_pivot_lowp;    /* mixed forms: of ms_pivot, in the low-precision
                                sweeps                                         */
    double ms_update_lowp;   /* mixed forms: of ms_update, in the low-precision
                                sweeps (tensor-core update kernels)            */
    double flops_refine;     /* mixed forms: of flops_fp64, in the refinement
                                GEMMs                                          */
    double ms_precond;       /* gesvd with svd_qr: device time of the QR
                                factorisation and of forming U = Q W           */
    double flops_precond;    /* the FP64 flops issued there (also counted in
                                flops_fp64)                                    */
    double rel_final;        /* EVD under JACOBI_CONV_REL: the relative
                                measure max_{i!=j}|a_ij|/sqrt(|a_ii a_jj|) of
                                the stop test at exit (0 under OFF_ABS)        */
    double rel_hist[64];     /* the same measure after each sweep             */
} jacobi_stats;

/*
 * jacobi_off_norm -- the stop statistic of the two-sided method on an
 * arbitrary matrix: the off-diagonal norm Xi(A) = sqrt(sum_{i != j} a_ij^2)
 * (Sec. 2.1, eq. (Omega_A); the quantity Algorithm 1's stop test compares
 * with tol ||A||_F), ||A||_F, and, when want_rel != 0, the relative measure
 * max_{i != j} |a_ij| / sqrt(|a_ii| |a_jj|) of JACOBI_CONV_REL (an entry
 * with a_ii a_jj = 0 counts as 0 when it is 0 and as +inf otherwise).
 * Computed by the same kernel and reduction order the sweeps use (sums of
 * squares in FP64, never as ||A||_F^2 - sum a_ii^2).
 *   n      order (n >= 1)
 *   A      device, n x n, leading dimension lda >= n; every entry is read
 *   h_out  host, 3 doubles: Xi(A), ||A||_F, the relative measure (0 when
 *          want_rel = 0)
 * Allocates a small workspace stream-ordered and blocks until done.
 * Returns 0, -k for an invalid argument k, JACOBI_ERR_ALLOC, JACOBI_ERR_CUDA.
 */
int jacobi_off_norm(int n, const double* A, int lda, int want_rel, double* h_out, void* stream);

/* Fill *p with the defaults above.  Returns 0. */
int jacobi_params_default(jacobi_params* p);

/* Static text for a return code. */
const char* jacobi_status_string(int status);

/*
 * jacobi_syev -- eigen-decomposition of a real symmetric n x n matrix by
 * blocked two-sided Jacobi (Algorithm 1, swept in the parallel order of
 * Algorithm 2; ordering from Algorithm 3 or round-robin).
 *
 *   n        order of A (n >= 1)
 *   A        device, n x n, leading dimension lda >= n.  Only the lower
 *            triangle is read (it is mirrored).  On exit A holds the final,
 *            nearly diagonal iterate D (Algorithm 1, Ensure).
 *   w        device, n doubles: the eigenvalues, ascending (the diagonal of D)
 *   Q        device, n x n, ldq >= n (may be NULL if p->want_vectors == 0):
 *            on exit the orthonormal eigenvectors, column j belonging to w[j].
 *            With p->warm_start, on entry an orthogonal start (resume): the
 *            call then continues from the caller's A and Q.
 *   p        parameters (NULL = defaults)
 *   st       statistics out (may be NULL)
 *   stream   cudaStream_t as void*
 * FP64 throughout for precision == JACOBI_PREC_FP64; the MIXED_* values run
 * the early sweeps' update GEMMs on the tensor cores from FP32 working copies
 * and return to FP64 for the closing sweeps and the refinement.
 */
int jacobi_syev(int n, double* A, int lda, double* w, double* Q, int ldq,
                const jacobi_params* p, jacobi_stats* st, void* stream);

/* Same as jacobi_syev with HOST buffers: the library copies A (and Q for a
 * warm start) to the device, runs, and copies A, w and Q back. */
int jacobi_syev_h(int n, double* h_A, int lda, double* h_w, double* h_Q, int ldq,
                  const jacobi_params* p, jacobi_stats* st, void* stream);

/*
 * jacobi_syev_f32 -- jacobi_syev for a matrix stored in FP32: A (n x n, lda
 * >= n, lower triangle read), w (n floats) and Q (n x n, ldq >= n, or NULL
 * when p->want_vectors == 0) are device FP32 buffers with the meaning, the
 * ownership and the return codes of jacobi_syev.  The input is widened
 * exactly to FP64 in library workspace, solved by jacobi_syev with the same
 * parameters (p->precision FP64, a mixed form or FP64_EMU), and D, w and Q
 * are rounded to FP32 once at the end (also when the sweep cap ends the
 * call); on a negative return the caller's buffers are left as they were.
 * With p->warm_start the FP32 Q is the (widened) start.  p->tol keeps its
 * FP64 meaning: a value near 2^-24 stops at FP32 accuracy sooner.
 */
int jacobi_syev_f32(int n, float* A, int lda, float* w, float* Q, int ldq,
                    const jacobi_params* p, jacobi_stats* st, void* stream);

/*
 * jacobi_gesvd -- one-sided blocked Jacobi SVD of an m x n matrix, m >= n
 * (Algorithm 6 in the parallel order): the pivot of block-column pair (I,J)
 * is the Gram block G(:,[I,J])^T G(:,[I,J]) (Sec. 6, eq. (SVD_subproblem)),
 * its eigenvectors rotate the column pair of G and of V; at exit
 * sigma_i = ||G(:,i)||_2 and U = G Sigma^+ (the output step of Algorithm 6),
 * sorted descending.
 *
 *   G      device, m x n, ldg >= m; in: G, out: U (zero column for sigma = 0)
 *   sigma  device, n doubles, descending
 *   V      device, n x n, ldv >= n (NULL if p->want_vectors == 0)
 * The stop test and the inner rotation threshold both use
 * tol_eff = max(p->tol, sqrt(m) * 2^-53): a sweep whose largest normalised
 * Gram off-diagonal |a_ij| / sqrt(a_ii a_jj) is <= tol_eff ends the
 * iteration.  p->conv is ignored.
 * p->precision: JACOBI_PREC_FP64, or JACOBI_PREC_FP64_EMU (or
 * p->fp64_products = 1) for the Gram blocks and the column updates formed
 * FP64-accurately on the bf16 tensor cores; the mixed precisions return
 * JACOBI_ERR_UNSUPPORTED.
 * With p->svd_qr = 1 (Sec. 6, "Preprocessing with QR"): G = QR by blocked
 * Householder QR (FP64), the method above on X = R^T (n x n, so tol_eff uses
 * sqrt(n)), X W = U_X Sigma, and G = (Q W) Sigma U_X^T: U = Q W (always
 * computed), V = U_X.  An exactly zero singular value then gives a zero
 * column of V instead of U.  st->ms_precond holds the QR time.
 */
int jacobi_gesvd(int m, int n, double* G, int ldg, double* sigma, double* V, int ldv,
                 const jacobi_params* p, jacobi_stats* st, void* stream);

/* Same as jacobi_gesvd with HOST buffers. */
int jacobi_gesvd_h(int m, int n, double* h_G, int ldg, double* h_sigma, double* h_V, int ldv,
                   const jacobi_params* p, jacobi_stats* st, void* stream);

/*
 * jacobi_syev_step -- exactly one parallel step of Algorithm 2: the pivot
 * solves of step `step` (0-based) of the sweep schedule, then the block-row
 * and block-column updates of A and the column updates of Q, then the pivot
 * blocks overwritten by D.  Operates in place on a full symmetric np x np
 * matrix (both triangles read; it must be exactly symmetric) with np = N * p->b
 * and N the block count (even for round-robin).  No sorting, no stop test.
 *   A  device, np x np, lda >= np;   Q  device, np x np, ldq >= np, or NULL.
 * p->precision: JACOBI_PREC_FP64 or JACOBI_PREC_FP64_EMU (the update
 * products on the tensor cores, FP64-accurate); others return
 * JACOBI_ERR_UNSUPPORTED.
 * Returns 0, or <0 on an invalid argument / CUDA error.
 */
int jacobi_syev_step(int np, double* A, int lda, double* Q, int ldq, const jacobi_params* p,
                     int step, void* stream);

/*
 * jacobi_gesvd_step -- exactly one step of the one-sided method (Algorithm
 * 6): for every column-block pair of step `step`, the Gram block (Sec. 6,
 * eq. (SVD_subproblem)), its FP64 Jacobi solve with the relative threshold
 * tol_eff (as in jacobi_gesvd), and G(:,[I,J]) <- G(:,[I,J]) Vhat,
 * V(:,[I,J]) <- V(:,[I,J]) Vhat.  G is m x np (np = N * p->b), V np x np or
 * NULL.  *relmax_out (host, may be NULL) receives the step's largest
 * normalised Gram off-diagonal before rotation.
 */
int jacobi_gesvd_step(int m, int np, double* G, int ldg, double* V, int ldv,
                      const jacobi_params* p, int step, double* relmax_out, void* stream);

/* ------------------------------------------------------------ batched forms
 * Thousands of independent matrices in one persistent launch (not in the
 * paper, whose subject is one matrix on P processors; the per-matrix method is
 * the same Jacobi iteration).  Each matrix is solved by one CTA with the
 * scalar parallel-ordered Jacobi of the pivot solve (Algorithm 2 applied with
 * b = 1, i.e. the blocked method with a single pair covering the matrix);
 * the matrices are taken longest first from an atomic queue.  A matrix of
 * order n (1 <= n <= 512) is solved in shared memory when it fits, else in a
 * per-CTA slot of global scratch.  Stop: a sweep applies no rotation
 * (relative threshold p->inner_tol; the default becomes 4 * 2^-24 for FP32),
 * or p->max_sweeps.
 *
 * Pointer arguments named without h_ are HOST arrays of DEVICE pointers, one
 * per matrix; h_* arrays are host arrays of sizes / leading dimensions (NULL
 * = tight).  info: DEVICE array of batch ints: 0 converged, >0 sweeps run
 * without converging, -100 non-finite input.  A is read only (lower
 * triangle); w ascending; Q (or NULL when p->want_vectors == 0) eigenvectors.
 * Argument errors carry jacobi_plan_create_batched's codes: -4 batch < 1,
 * -6 h_n (NULL, or some n outside 1..512), -7 a leading dimension too small.
 */
int jacobi_syev_batched(int batch, const int* h_n, double* const* A, const int* h_lda,
                        double* const* w, double* const* Q, const int* h_ldq,
                        const jacobi_params* p, int* info, jacobi_stats* st, void* stream);
int jacobi_syev_batched_f32(int batch, const int* h_n, float* const* A, const int* h_lda,
                            float* const* w, float* const* Q, const int* h_ldq,
                            const jacobi_params* p, int* info, jacobi_stats* st, void* stream);

/* Batched one-sided SVD (Algorithm 6 with a single column-block pair): each
 * sweep forms the n x n Gram block of G (m x n, m >= n, m n < 2^31; the
 * Gram, V-hat and the accumulated V live in shared memory, which bounds n at
 * 124 on GB300: larger n returns JACOBI_ERR_UNSUPPORTED), solves it with the
 * FP32 Jacobi core, sorts its eigenpairs descending and rotates G's columns
 * and V.  Stop: the Gram's largest normalised off-diagonal <= max(p->tol,
 * sqrt(m) 2^-24), or a sweep without rotation.  G is overwritten by U; sigma
 * descending.  Argument errors carry jacobi_plan_create_batched's codes:
 * -4 batch < 1, -5 h_m (NULL, or some m n >= 2^31), -6 h_n (some n < 1,
 * n > 512 or n > m), -7 a leading dimension too small. */
int jacobi_gesvd_batched_f32(int batch, const int* h_m, const int* h_n, float* const* G,
                             const int* h_ldg, float* const* sigma, float* const* V,
                             const int* h_ldv, const jacobi_params* p, int* info,
                             jacobi_stats* st, void* stream);

/* Plan API: validation, longest-first order, workspace and the launch shape
 * are set up once; the first execute captures [pointer upload, queue reset,
 * persistent kernel] into a CUDA graph that later executes replay.
 *   kind: 0 = symmetric EVD, 1 = one-sided SVD;  precision: JACOBI_PREC_FP64
 *   or JACOBI_PREC_FP32 (kind 1: FP32 only).  h_m may be NULL for kind 0.
 * jacobi_plan_autotune times each candidate launch shape (threads per CTA,
 * largest order kept in shared memory), then each candidate order above
 * which the blocked method takes over (jacobi_plan_blocking), on a sample of
 * the batch, keeps the fastest, and records it in an in-process cache keyed
 * by kind, precision,
 * vectors and the size mix (also written to the file named by the
 * environment variable JACOBI_TUNE_CACHE, if set, and read back by later
 * plans).  Plans are not thread-safe; one plan per stream. */
typedef struct jacobi_plan jacobi_plan;
int jacobi_plan_create_batched(jacobi_plan** out, int kind, int precision, int batch,
                               const int* h_m, const int* h_n, const int* h_lda,
                               const int* h_ldq, const jacobi_params* p, void* stream);
int jacobi_plan_autotune(jacobi_plan* plan, void* const* A_or_G, void* const* w_or_sigma,
                         void* const* Q_or_V, int* info, void* stream);
int jacobi_plan_execute(jacobi_plan* plan, void* const* A_or_G, void* const* w_or_sigma,
                        void* const* Q_or_V, int* info, jacobi_stats* st, void* stream);
int jacobi_plan_shape(const jacobi_plan* plan, int* threads, int* smem_kmax, int* grid);
/* The block size a symmetric-EVD plan uses per size class: orders up to
 * *min_order are solved unblocked (the whole matrix is one pivot, in shared
 * memory or spread over a cluster), orders above it by the blocked method of
 * Algorithm 1 with block size *b (16).  jacobi_plan_autotune chooses
 * min_order (with the launch shape) by timing candidates on a sample of the
 * batch; *b = *min_order = 0 for a plan without the blocked route (one-sided
 * plans, JACOBI_BATCHED_LARGE=l2|cluster).  Returns 0, -1 (plan NULL). */
int jacobi_plan_blocking(const jacobi_plan* plan, int* b, int* min_order);
void jacobi_plan_destroy(jacobi_plan* plan);

/*
 * jacobi_syev_step_noalloc -- jacobi_syev_step without any allocation.  The
 * paper has no counterpart: it exists for callers that cannot allocate, such
 * as code inside a framework that owns all device memory through its own pool
 * (a cudaMalloc from outside the pool fails or fragments it) and
 * latency-critical loops that cannot take an allocation's implicit
 * synchronisation.  Same arguments and the same step as jacobi_syev_step;
 * every buffer besides A and Q lives in a fixed array in device global
 * memory, so the call makes no cudaMalloc / cudaFree and no host heap
 * allocation.
 *   Limits: np <= 768 and 1 <= p->b <= 128, else JACOBI_ERR_UNSUPPORTED.
 *   Plain FP64 products only: p->precision other than JACOBI_PREC_FP64,
 *   p->fp64_products = 1, or p->pivot_order = 2 (the QRCP pivoting step)
 *   return JACOBI_ERR_UNSUPPORTED; the other parameters are checked as in
 *   jacobi_syev_step (-6 when invalid).  The array (about 24 MB) stays
 *   resident on every GPU the process uses until the process exits.
 *   Results: the pivot solves always run one CTA per pair, so A and Q agree
 *   with jacobi_syev_step to rounding, and bit for bit when that call also
 *   runs one CTA per pair (JACOBI_PIVOT_CLUSTER=1).
 *   The first call on a device looks up the array's address on that device;
 *   make that first call before any stream capture.  The address is kept for
 *   the life of the process: after cudaDeviceReset on a device, do not call
 *   this entry point on that device again.
 *   All calls share the array: calls whose work overlaps on the GPU (other
 *   streams, other host threads) race and must be serialised by the caller.
 *   Returns 0, -k for an invalid argument k, -7 for a step outside the
 *   schedule, JACOBI_ERR_UNSUPPORTED, JACOBI_ERR_CUDA.
 */
int jacobi_syev_step_noalloc(int np, double* A, int lda, double* Q, int ldq,
                             const jacobi_params* p, int step, void* stream);

/*
 * jacobi_rotation_params -- diagnostic: the 2x2 symmetric Schur rotation of
 * the scalar Jacobi solves inside every FP64 pivot solve (Sec. 2.1,
 * Algorithm 1 applied with b = 1), for `count` triples (app[i], aqq[i],
 * apq[i]) in device memory.  For each i, out[8 i .. 8 i + 7] (device) gets
 * t, s, tau and the rotation test (1.0 rotate, 0.0 skip) as the pivot solves
 * compute them (FP32 seeds refined by Newton steps in FP64), then t, s, tau
 * and the test by the textbook formulas in correctly rounded FP64 operations
 * (zeta = (aqq - app)/(2 apq), t = sgn(zeta)/(|zeta| + sqrt(1 + zeta^2)),
 * c = 1/sqrt(1 + t^2), s = t c, tau = s/(1 + c); rotate when
 * |apq| > tol sqrt|app| sqrt|aqq|).  Returns 0, -k for an invalid
 * argument k, JACOBI_ERR_CUDA.
 */
int jacobi_rotation_params(int count, const double* app, const double* aqq, const double* apq, double tol,
                           double* out, void* stream);

/*
 * jacobi_lowp_gemm -- the split-precision tensor-core product used by the
 * mixed-precision sweeps, as a primitive: C = op(A) B in FP32 where every
 * operand value x enters as hi = bf16(x), lo = bf16(x - hi) and each product
 * as hi*hi + hi*lo + lo*hi, accumulated in FP32 by tcgen05.mma (kind::f16)
 * in tensor memory.  All matrices column-major FP32 on the device: A is
 * M x K (transA = 0, lda >= M) or K x M (transA = 1, lda >= K), B K x N
 * (ldb >= K), C M x N (ldc >= M).  Returns 0, -k for an invalid argument,
 * JACOBI_ERR_TIMEOUT if a bounded wait on the tensor cores ran out.
 * (The paper names variable precision as future work, Sec. 7.)
 */
int jacobi_lowp_gemm(int M, int N, int K, const float* A, int lda, int transA, const float* B,
                     int ldb, float* C, int ldc, void* stream);

/*
 * jacobi_f64emu_gemm -- an FP64-accurate product on the bf16 tensor cores:
 * C = op(A) B with every row of op(A) and column of B scaled by a power of two
 * and cut into eight 7-bit integer slices (bf16), the 36 slice products with
 * p + q <= 9 accumulated exactly in FP32 per significance level (tcgen05,
 * TMEM) and combined in FP64 (the error-free splitting of Ozaki et al.,
 * applied with bf16 slices).  Error below about (9 K + 64) 2^-56 2^{E_m + F_n}
 * per entry, where 2^{E_m} > max |op(A)(m, :)| and 2^{F_n} > max |B(:, n)|.
 * Column-major FP64 on the device: A is M x K (transA = 0, lda >= M) or
 * K x M (transA = 1, lda >= K), B K x N (ldb >= K), C M x N (ldc >= M).
 * Beyond K = 256 the exact FP32 level sums are drained every 256 K values
 * into 64-bit integer running sums (the scales then cover whole rows and
 * columns); K <= 2^20 (JACOBI_ERR_UNSUPPORTED above).  Returns 0, -k for
 * an invalid argument, JACOBI_ERR_ALLOC, JACOBI_ERR_TIMEOUT if a bounded
 * tensor-core wait ran out.
 */
int jacobi_f64emu_gemm(int M, int N, int K, const double* A, int lda, int transA, const double* B,
                       int ldb, double* C, int ldc, void* stream);

/*
 * jacobi_syev_step_lowp -- one step of the mixed form's low-precision phase
 * (Algorithm 2's step with the updates on the tensor cores): the pivot
 * blocks of step `step` are promoted to FP64 and solved in FP64 (as in
 * jacobi_syev_step), D is written back rounded to FP32, and every
 * block-row/column update of A (A'_{P1P2} = V1^T A_{P1P2} V2, mirrored) and
 * column update of Q (Q'(:,P) = Q(:,P) V_P) is formed from V (accumulated in
 * FP32 by the pivot solve: |dV| <= 6 k u32 entry-wise inside each pair's
 * k x k block, k = 2b) by the split-precision product of jacobi_lowp_gemm (bf16 splits; fp16
 * splits with power-of-two row/column scaling for MIXED_FP16X3).  A is a full
 * symmetric np x np FP32 matrix (exactly symmetric), np = N * p->b with N
 * even for round-robin; Q is np x np FP32 or NULL; both device, column-major,
 * updated in place.  p->precision must be JACOBI_PREC_MIXED_BF16X3,
 * JACOBI_PREC_MIXED_FP16X3 or JACOBI_PREC_MIXED_TF32 (tf32 big/small splits).
 * Returns 0, -k for an invalid argument, JACOBI_ERR_UNSUPPORTED for another
 * precision, JACOBI_ERR_TIMEOUT if a bounded tensor-core wait ran out,
 * JACOBI_ERR_CUDA / JACOBI_ERR_ALLOC.  Allocates its workspace
 * stream-ordered and blocks until done.
 */
int jacobi_syev_step_lowp(int np, float* A, int lda, float* Q, int ldq, const jacobi_params* p,
                          int step, void* stream);

/*
 * jacobi_wait_selftest -- failure detection on the tensor cores, exercised:
 * the paper has no counterpart.  The tcgen05 kernels (the mixed forms'
 * updates, the emulated FP64 products, jacobi_lowp_gemm, jacobi_f64emu_gemm)
 * wait on mbarriers that their own MMAs arrive at; every such wait is
 * bounded (about 2 s by the global timer, and a cap on the polls), and a
 * wait that runs out sets the call's error word, skips the rest of the
 * tile, frees the CTA's tensor memory and returns, so the call returns
 * JACOBI_ERR_TIMEOUT and the CUDA context stays usable.  This entry point
 * runs one CTA through the same steps: allocate tensor memory, initialise an
 * mbarrier, wait on it with the bound limit_ms (1 .. 2000 ms), free the
 * tensor memory.  arrive = 1: one thread arrives, the wait completes,
 * returns 0.  arrive = 0: nothing arrives, the wait runs out after about
 * limit_ms, returns JACOBI_ERR_TIMEOUT.  Blocks until done.
 * Returns 0, JACOBI_ERR_TIMEOUT, -1 (arrive not 0 or 1), -2 (limit_ms out
 * of range), JACOBI_ERR_ALLOC, JACOBI_ERR_CUDA.
 */
int jacobi_wait_selftest(int arrive, double limit_ms, void* stream);

/*
 * jacobi_ordering_table -- the library's pair schedule for N blocks
 * (host-side logic, no GPU needed): kind is JACOBI_ORDER_*; pairs receives
 * 2 ints (I < J, 0-based) per pair, step after step (room for N*(N-1) ints);
 * step_ptr (N+1 ints) the offset of each step in pairs.  Returns the number of
 * steps, or -1 for an invalid (kind, N) (N < 2, or odd N for round-robin).
 */
int jacobi_ordering_table(int kind, int N, int* pairs, int* step_ptr);

#ifdef __cplusplus
}
#endif
#endif /* JACOBI_GB300_H */
