/*
 * jacobi_oracle.c -- plain, slow CPU reference of blocked Jacobi (EVD and
 * one-sided SVD) in IEEE FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * (the CUDA library) never calls it, and it shares no code, header, table or
 * constant generator with the product.
 *
 * Every public function is pinned against facts from outside this file
 * (closed forms, printed tables, constructed spectra, exact roots, LAPACK,
 * mpmath) in tests/test_oracle_pins.py, and tests/test_oracle_mutants.py
 * plants plausible mistakes in copies of this file to show the pins catch
 * them; no function is parity-unpinned.
 *
 * What is computed, and where the paper defines it
 * (Demmel, Luo, Schneider, Wang, "Minimizing the Arithmetic and Communication
 *  Complexity of Jacobi's Method ... Part Two -- Parallel Algorithms"):
 *
 *   - Block partition A_IJ = A((I-1)b+1:Ib, (J-1)b+1:Jb)           Sec. 2.1, eq. (A_subblock)
 *   - Off-diagonal "norm" Xi(A) = sqrt(sum_{i!=j} A(i,j)^2)          Sec. 2.1, eq. (Omega_A)
 *   - Block Jacobi sweep: diagonalise the 2b x 2b pivot, multiply
 *     block rows I,J by Qhat^T, block columns I,J by Qhat, and Q by Qhat
 *                                                                     Algorithm 1
 *   - One parallel step over a group of disjoint pairs: every pivot of
 *     the group is solved, then the block-row update, then the
 *     block-column update of A and Q, then the pivot blocks are
 *     overwritten by D (including the D12 / D21 of an approximate solve)
 *                                                                     Algorithm 2, Sec. 3
 *   - Orderings: "cyclic by anti-diagonals"                           Algorithm 3
 *                round-robin tournament (standard; the paper allows
 *                any grouping into disjoint pairs)                    Sec. 3 (item 2)
 *   - The 2b x 2b pivot solve is itself Jacobi on 1 x 1 blocks with
 *     the same parallel ordering (the recursive use of 2D Jacobi on
 *     a subproblem, Sec. 4); the 1x1-block "pivot" is the textbook
 *     2 x 2 symmetric Schur rotation (Sec. 1: one rotation zeroes
 *     A(i,j) and lowers off^2 by 2 A(i,j)^2).  The solve may be
 *     approximate (Sec. 3, after Algorithm 3).
 *   - One-sided Jacobi SVD: Gram pivot Ahat = G(:,[I,J])^T G(:,[I,J]),
 *     G(:,[I,J]) <- G(:,[I,J]) Vhat, V likewise; Sigma = column norms,
 *     U = G Sigma^+                                                    Algorithm 6, Sec. 6
 *
 * Readings where the paper is silent:
 *   - round-robin: block 0 fixed, positions 1..N-1 rotate by one per step;
 *     step s pairs position k with position N-1-k;
 *   - anti-diagonal groups are emitted in the order K = 0..N-1;
 *   - b that does not divide n: pad with zero rows/columns; N is raised to
 *     at least 2 and to an even number (for both orderings);
 *   - a scalar rotation is skipped when |a_pq| <= tol_rel*sqrt|a_pp|*sqrt|a_qq|;
 *   - the inner solve stops after a sweep with no rotation, or after
 *     inner_max_sweeps sweeps;
 *   - after a pivot solve its eigenpairs may be permuted, Qhat <- Qhat P (the
 *     slot of the pivoting step of Sec. 2.1, items 1-2 after Algorithm 1); the
 *     permutation used here sorts the pivot's eigenvalues in descending order
 *     (ties keep their index order) over the pivot's real rows, leaving the
 *     zero padding rows where they are (pivot_order 1); pivot_order 2 is the
 *     pivoting step itself: the column order that column-pivoted QR
 *     (Businger-Golub, norms recomputed, ties to the smaller index) picks on
 *     the leading real rows of Vhat; the GPU path applies the same rules;
 *   - the outer loop stops when off(A) <= tol*||A||_F (or, for the relative
 *     criterion, max |a_ij|/sqrt|a_ii a_jj| <= tol), or when the measure is
 *     already <= 100*tol and did not halve over the last sweep (stall).
 *
 * Applying a rotation: with tau = s/(1+c) the pair (x, y) becomes
 * (x - s(y + tau x), y + s(x - tau y)), algebraically (c x - s y, s x + c y).
 * This is Rutishauser's form of the update; its rounding error is relative to
 * the correction s(...), so the rotated vectors keep their length even for
 * the small angles of late sweeps, where the computed (c, s) satisfy
 * c^2 + s^2 = 1 + u on average and the plain form would let every column
 * grow by about one unit roundoff per rotation.
 *
 * Diagonal of a pivot during its solve: each entry is carried as an unevaluated
 * sum hi + lo (hi is what the rotation tests read).  A rotation's diagonal
 * change -/+ t a_pq is formed exactly (fma) and added with an error-free
 * two-sum, and the output Dhat gets hi + lo rounded once.  In the last inner
 * sweeps t a_pq is below half an ulp of a_pp while the zeroed a_pq is not
 * negligible; without the lo part that energy is lost on every rotation, in
 * the same direction, and the spectrum shrinks by O(n u) over a solve.
 *
 * Numbers: everything is IEEE binary64, round-to-nearest, built with
 * -ffp-contract=off so that no fused multiply-add changes a rounding, which
 * makes x86-64 and AArch64 builds give identical bits.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_ORDER_ROUND_ROBIN 0
#define ORC_ORDER_ANTI_DIAGONAL 1
#define ORC_CONV_OFF_ABS 0
#define ORC_CONV_REL 1

typedef struct {
    int b;                /* block size b (>= 1)                                  */
    int ordering;         /* 0 round-robin, 1 anti-diagonal (Algorithm 3)         */
    int max_sweeps;       /* outer sweep cap                                      */
    int inner_max_sweeps; /* inner (pivot) sweep cap                              */
    int conv;             /* 0: off(A) <= tol ||A||_F; 1: relative criterion      */
    double tol;           /* outer tolerance                                      */
    double inner_tol;     /* relative threshold of one scalar rotation            */
    int want_vectors;     /* accumulate Q (EVD) / V (SVD)                         */
    int threads;          /* OpenMP threads (0 = runtime default)                 */
    int pivot_order;      /* 0: as solved; 1: sorted descending; 2: QRCP (Sec. 2.1) */
} orc_params;

typedef struct {
    int status;           /* 0 converged, >0 sweeps done without converging       */
    int sweeps;
    int stalled;          /* stopped by the stall rule                            */
    long long steps;
    long long pair_solves;
    long long rotations;      /* scalar rotations applied (inner + scalar paths)  */
    long long inner_sweeps;
    double off_initial;
    double off_final;
    double norm_fro;
    double off_hist[64];
    double rel_hist[64];      /* under ORC_CONV_REL: the relative measure per sweep */
} orc_stats;

/* ------------------------------------------------------------------ */
/* Orderings                                                           */
/* ------------------------------------------------------------------ */

/* Round-robin tournament on N (even) blocks, 0-based.  Writes N-1 steps of
 * N/2 pairs (I<J) into pairs[2*(s*N/2+k)+{0,1}].  Returns the step count. */
static int rr_table(int N, int *pairs)
{
    int half = N / 2, S = N - 1;
    for (int s = 0; s < S; s++) {
        for (int k = 0; k < half; k++) {
            int pa = k, pb = N - 1 - k;
            /* block sitting at a position: position 0 holds block 0; position
             * p>=1 holds block 1 + ((p - 1 + s) mod (N-1)). */
            int ba = (pa == 0) ? 0 : 1 + ((pa - 1 + s) % (N - 1));
            int bb = (pb == 0) ? 0 : 1 + ((pb - 1 + s) % (N - 1));
            int I = ba < bb ? ba : bb, J = ba < bb ? bb : ba;
            pairs[2 * (s * half + k) + 0] = I;
            pairs[2 * (s * half + k) + 1] = J;
        }
    }
    return S;
}

/* Algorithm 3: group K (K = 0..N-1) holds the 1-based pairs I<J with
 * (I+J) mod N == K.  Output is 0-based.  step_ptr[s]..step_ptr[s+1] index the
 * pairs of step s.  Returns N (the step count). */
static int ad_table(int N, int *pairs, int *step_ptr)
{
    int cnt = 0;
    for (int K = 0; K < N; K++) {
        step_ptr[K] = cnt;
        for (int I = 1; I <= N - 1; I++)
            for (int J = I + 1; J <= N; J++)
                if ((I + J) % N == K) {
                    pairs[2 * cnt + 0] = I - 1;
                    pairs[2 * cnt + 1] = J - 1;
                    cnt++;
                }
    }
    step_ptr[N] = cnt;
    return N;
}

/* Public: ordering table.  kind 0 round-robin (N must be even), 1 Algorithm 3.
 * pairs needs room for N*(N-1)/2 pairs, step_ptr for N+1 entries.
 * Returns the number of steps, or -1 on a bad argument. */
int oracle_ordering(int kind, int N, int *pairs, int *step_ptr)
{
    if (N < 2) return -1;
    if (kind == ORC_ORDER_ROUND_ROBIN) {
        if (N % 2) return -1;
        int S = rr_table(N, pairs);
        for (int s = 0; s <= S; s++) step_ptr[s] = s * (N / 2);
        return S;
    }
    if (kind == ORC_ORDER_ANTI_DIAGONAL) return ad_table(N, pairs, step_ptr);
    return -1;
}

/* ------------------------------------------------------------------ */
/* The textbook 2x2 symmetric Schur rotation                           */
/* ------------------------------------------------------------------ */

/* For [[app, apq],[apq, aqq]] with apq != 0: zeta = (aqq-app)/(2 apq),
 * t = sgn(zeta)/(|zeta| + sqrt(1+zeta^2)) (sgn(0)=+1, so |angle| <= pi/4),
 * c = 1/sqrt(1+t^2), s = t c.  With J = [[c, s],[-s, c]],
 * J^T [[app,apq],[apq,aqq]] J = diag(app - t apq, aqq + t apq). */
void oracle_rotation(double app, double aqq, double apq, double *c, double *s, double *t)
{
    double zeta = (aqq - app) / (2.0 * apq);
    double tt;
    if (fabs(zeta) > 1e150) {
        tt = 0.5 / zeta;                       /* 1 + zeta^2 would overflow */
    } else {
        double r = sqrt(1.0 + zeta * zeta);
        tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + r);
    }
    double cc = 1.0 / sqrt(1.0 + tt * tt);
    *t = tt;
    *c = cc;
    *s = tt * cc;
}

/* (hi, lo) <- (hi, lo) + d * sgn for the diagonal update, with d = t * apq
 * formed exactly as dh + dl (fma) and the sum by an error-free two-sum. */
static void dd_add_prod(double *hi, double *lo, double t, double apq, double sgn)
{
    double dh = t * apq;
    double dl = fma(t, apq, -dh);
    dh *= sgn;
    dl *= sgn;
    double a = *hi, sum = a + dh;
    double bb = sum - a;
    double err = (a - (sum - bb)) + (dh - bb);
    err += *lo + dl;
    double h2 = sum + err;
    *lo = err - (h2 - sum);
    *hi = h2;
}

/* The pair (x, y) <- (c x - s y, s x + c y) in Rutishauser's form. */
static void rot_apply(double s, double tau, double *x, double *y)
{
    double a = *x, b = *y;
    *x = a - s * (b + tau * a);
    *y = b + s * (a - tau * b);
}

static int rotation_wanted(double app, double aqq, double apq, double tol_rel)
{
    if (apq == 0.0) return 0;
    return fabs(apq) > tol_rel * sqrt(fabs(app)) * sqrt(fabs(aqq));
}

/* ------------------------------------------------------------------ */
/* Small helpers                                                        */
/* ------------------------------------------------------------------ */

#define AT(M, ld, i, j) ((M)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

static double off_norm(int n, const double *A, int lda)
{
    double s = 0.0;
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++)
            if (i != j) s += AT(A, lda, i, j) * AT(A, lda, i, j);
    return sqrt(s);
}

static double fro_norm(int n, const double *A, int lda)
{
    double s = 0.0;
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) s += AT(A, lda, i, j) * AT(A, lda, i, j);
    return sqrt(s);
}

/* max_{i != j} |a_ij| / sqrt(|a_ii| |a_jj|); an entry whose diagonal product
 * is zero counts as 0 when it is itself zero and as +inf otherwise. */
static double rel_off(int n, const double *A, int lda)
{
    double m = 0.0;
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            if (i == j) continue;
            double a = fabs(AT(A, lda, i, j));
            if (a == 0.0) continue;
            double d = sqrt(fabs(AT(A, lda, i, i))) * sqrt(fabs(AT(A, lda, j, j)));
            double r = d > 0.0 ? a / d : INFINITY;
            if (r > m) m = r;
        }
    return m;
}

/* Public: off(A) as defined in Sec. 2.1. */
double oracle_off_norm(int n, const double *A, int lda) { return off_norm(n, A, lda); }
double oracle_rel_off(int n, const double *A, int lda) { return rel_off(n, A, lda); }

/* ------------------------------------------------------------------ */
/* One textbook rotation (used by the scalar path and the pins)          */
/* ------------------------------------------------------------------ */

/* Apply the rotation that annihilates A(p,q) to rows/columns p,q of the full
 * symmetric A and to columns p,q of Q (if Q != NULL).  Returns 1 if applied,
 * 0 if A(p,q) == 0. */
int oracle_rotate(int n, double *A, int lda, double *Q, int ldq, int p, int q)
{
    double apq = AT(A, lda, p, q);
    if (apq == 0.0) return 0;
    double app = AT(A, lda, p, p), aqq = AT(A, lda, q, q);
    double c, s, t;
    oracle_rotation(app, aqq, apq, &c, &s, &t);
    double tau = s / (1.0 + c);
    for (int j = 0; j < n; j++)            /* rows: A <- J^T A */
        rot_apply(s, tau, &AT(A, lda, p, j), &AT(A, lda, q, j));
    for (int i = 0; i < n; i++)            /* columns: A <- A J */
        rot_apply(s, tau, &AT(A, lda, i, p), &AT(A, lda, i, q));
    AT(A, lda, p, p) = app - t * apq;
    AT(A, lda, q, q) = aqq + t * apq;
    AT(A, lda, p, q) = 0.0;
    AT(A, lda, q, p) = 0.0;
    if (Q)
        for (int i = 0; i < n; i++) rot_apply(s, tau, &AT(Q, ldq, i, p), &AT(Q, ldq, i, q));
    return 1;
}

/* ------------------------------------------------------------------ */
/* Finalisation                                                         */
/* ------------------------------------------------------------------ */

/* Stable sort of idx[0..n) by key (ascending if asc, else descending);
 * ties keep the original order.  Insertion sort: slow and obvious. */
static void stable_argsort(int n, const double *key, int *idx, int asc)
{
    for (int i = 0; i < n; i++) idx[i] = i;
    for (int i = 1; i < n; i++) {
        int v = idx[i], j = i - 1;
        while (j >= 0) {
            double a = key[idx[j]], b = key[v];
            int after = asc ? (a > b) : (a < b);
            if (!after) break;
            idx[j + 1] = idx[j];
            j--;
        }
        idx[j + 1] = v;
    }
}

/* EVD: w = diag(A) ascending; Q's columns permuted alike (Algorithm 1, Ensure). */
static void finalize_evd(int n, const double *A, int lda, double *w, double *Qw, int ldqw,
                         double *Q, int ldq)
{
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    int *idx = (int *)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; i++) d[i] = AT(A, lda, i, i);
    stable_argsort(n, d, idx, 1);
    for (int i = 0; i < n; i++) w[i] = d[idx[i]];
    if (Q && Qw)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) AT(Q, ldq, i, j) = AT(Qw, ldqw, i, idx[j]);
    free(d);
    free(idx);
}

/* ------------------------------------------------------------------ */
/* Pivot solve: Jacobi on 1x1 blocks with the round-robin parallel order  */
/* ------------------------------------------------------------------ */

/* Diagonalise the k x k symmetric Ahat (k even, column-major, ld k) in place.
 * On return Ahat holds Dhat and V (k x k, ld k) the product of the rotations.
 * Each round: every pair (p,q) of the round computes its rotation from the
 * round's starting values; then all rows are rotated (A <- J^T A), then all
 * columns (A <- A J) and V <- V J; then every rotated 2x2 pivot is set to
 * its exact diagonal form (Algorithm 2 applied with b = 1).
 * Returns the number of rotations applied; *sweeps_out = inner sweeps run. */
int oracle_pivot_solve(int k, double *Ah, double *V, double tol_rel, int max_sweeps,
                       int *sweeps_out)
{
    int half = k / 2, S = k - 1;
    int *tab = (int *)malloc(sizeof(int) * (size_t)(2 * half * (S > 0 ? S : 1)));
    double *cs = (double *)malloc(sizeof(double) * (size_t)(4 * half));
    int *on = (int *)malloc(sizeof(int) * (size_t)half);
    double *dlo = (double *)calloc((size_t)k, sizeof(double)); /* low parts of the diagonal */
    double *diag0 = (double *)malloc(sizeof(double) * (size_t)k); /* hi parts at round start */
    if (S > 0) rr_table(k, tab);
    for (int j = 0; j < k; j++)
        for (int i = 0; i < k; i++) AT(V, k, i, j) = (i == j) ? 1.0 : 0.0;
    int total = 0, sw = 0;
    for (sw = 0; sw < max_sweeps; sw++) {
        int in_sweep = 0;
        for (int r = 0; r < S; r++) {
            const int *pr = tab + 2 * half * r;
            for (int e = 0; e < half; e++) {
                int p = pr[2 * e], q = pr[2 * e + 1];
                double app = AT(Ah, k, p, p), aqq = AT(Ah, k, q, q), apq = AT(Ah, k, p, q);
                diag0[p] = app;
                diag0[q] = aqq;
                on[e] = rotation_wanted(app, aqq, apq, tol_rel);
                if (on[e]) {
                    double c, s, t;
                    oracle_rotation(app, aqq, apq, &c, &s, &t);
                    cs[4 * e + 0] = c;
                    cs[4 * e + 1] = s;
                    cs[4 * e + 2] = t;
                    cs[4 * e + 3] = apq;
                }
            }
            for (int e = 0; e < half; e++) { /* rows */
                if (!on[e]) continue;
                int p = pr[2 * e], q = pr[2 * e + 1];
                double s = cs[4 * e + 1], tau = s / (1.0 + cs[4 * e]);
                for (int j = 0; j < k; j++) rot_apply(s, tau, &AT(Ah, k, p, j), &AT(Ah, k, q, j));
            }
            for (int e = 0; e < half; e++) { /* columns of A and V */
                if (!on[e]) continue;
                int p = pr[2 * e], q = pr[2 * e + 1];
                double s = cs[4 * e + 1], tau = s / (1.0 + cs[4 * e]);
                for (int i = 0; i < k; i++) {
                    rot_apply(s, tau, &AT(Ah, k, i, p), &AT(Ah, k, i, q));
                    rot_apply(s, tau, &AT(V, k, i, p), &AT(V, k, i, q));
                }
            }
            for (int e = 0; e < half; e++) { /* exact 2x2 diagonal form */
                if (!on[e]) continue;
                int p = pr[2 * e], q = pr[2 * e + 1];
                double t = cs[4 * e + 2], apq = cs[4 * e + 3];
                double hp = diag0[p], hq = diag0[q];
                dd_add_prod(&hp, &dlo[p], t, apq, -1.0);
                dd_add_prod(&hq, &dlo[q], t, apq, +1.0);
                AT(Ah, k, p, p) = hp;
                AT(Ah, k, q, q) = hq;
                AT(Ah, k, p, q) = 0.0;
                AT(Ah, k, q, p) = 0.0;
                in_sweep++;
            }
        }
        total += in_sweep;
        if (in_sweep == 0) { sw++; break; }
    }
    for (int i = 0; i < k; i++) AT(Ah, k, i, i) += dlo[i]; /* hi + lo, rounded once */
    if (sweeps_out) *sweeps_out = sw;
    free(tab);
    free(cs);
    free(on);
    free(dlo);
    free(diag0);
    return total;
}

/* Permutation step after a pivot solve: reorder the eigenpairs (Dhat's
 * rows/columns and Vhat's columns) so that diag(Dhat) is descending over the
 * pivot's real positions (global index < n_real); padding positions stay put;
 * ties keep their index order.  Dhat <- P^T Dhat P, Vhat <- Vhat P. */
static void sort_pivot_desc(int k, double *Ah, double *V, double *tmp, int *idx, int I, int J,
                            int b, int n_real)
{
    double *d = tmp;
    int *pos = (int *)malloc(sizeof(int) * (size_t)k);
    int *ord = (int *)malloc(sizeof(int) * (size_t)k);
    int nr = 0;
    for (int x = 0; x < k; x++) {
        int g = x < b ? I * b + x : J * b + (x - b);
        idx[x] = x;
        if (g < n_real) pos[nr++] = x;
    }
    for (int t = 0; t < nr; t++) d[t] = AT(Ah, k, pos[t], pos[t]);
    stable_argsort(nr, d, ord, 0);
    for (int t = 0; t < nr; t++) idx[pos[t]] = pos[ord[t]];
    free(pos);
    free(ord);
    double *B = tmp + k;
    for (int j = 0; j < k; j++)
        for (int i = 0; i < k; i++) AT(B, k, i, j) = AT(Ah, k, idx[i], idx[j]);
    memcpy(Ah, B, sizeof(double) * (size_t)k * k);
    for (int j = 0; j < k; j++)
        for (int i = 0; i < k; i++) AT(B, k, i, j) = AT(V, k, i, idx[j]);
    memcpy(V, B, sizeof(double) * (size_t)k * k);
}

/* Column-pivoted QR (Businger-Golub) of the r x c matrix M (column-major, ld
 * r, overwritten): at step t the remaining column of largest norm over rows
 * t.. (recomputed, not downdated; ties to the smaller index) is swapped to
 * position t, and a Householder reflection clears it below row t.  perm
 * (c entries, in: identity) records the column order. */
static void qrcp_steps(int r, int c, double *M, int *perm)
{
    double *v = (double *)malloc(sizeof(double) * (size_t)(r > 0 ? r : 1));
    int steps = r < c ? r : c;
    for (int t = 0; t < steps; t++) {
        int best = t;
        double bn = -1.0;
        for (int j = t; j < c; j++) {
            double s = 0.0;
            for (int i = t; i < r; i++) s += M[i + (size_t)r * j] * M[i + (size_t)r * j];
            if (s > bn) { bn = s; best = j; }
        }
        if (best != t) {
            int ti = perm[t]; perm[t] = perm[best]; perm[best] = ti;
            for (int i = 0; i < r; i++) {
                double tv = M[i + (size_t)r * t];
                M[i + (size_t)r * t] = M[i + (size_t)r * best];
                M[i + (size_t)r * best] = tv;
            }
        }
        double alpha = M[t + (size_t)r * t], xn = 0.0;
        for (int i = t + 1; i < r; i++) xn += M[i + (size_t)r * t] * M[i + (size_t)r * t];
        xn = sqrt(xn);
        if (xn == 0.0) continue; /* H = I */
        double beta = -copysign(hypot(alpha, xn), alpha);
        double tau = (beta - alpha) / beta, sc = 1.0 / (alpha - beta);
        v[t] = 1.0;
        for (int i = t + 1; i < r; i++) v[i] = M[i + (size_t)r * t] * sc;
        for (int j = t + 1; j < c; j++) {
            double w = 0.0;
            for (int i = t; i < r; i++) w += v[i] * M[i + (size_t)r * j];
            w *= tau;
            for (int i = t; i < r; i++) M[i + (size_t)r * j] -= w * v[i];
        }
        M[t + (size_t)r * t] = beta;
        for (int i = t + 1; i < r; i++) M[i + (size_t)r * t] = 0.0;
    }
    free(v);
}

/* The QRCP column order of the r x c matrix X alone (for the pins). */
int oracle_qrcp_perm(int r, int c, const double *X, int *perm_out)
{
    if (r < 0 || c < 0 || !X || !perm_out) return -1;
    double *M = (double *)malloc(sizeof(double) * (size_t)(r > 0 ? r : 1) * (c > 0 ? c : 1));
    for (int j = 0; j < c; j++) {
        perm_out[j] = j;
        for (int i = 0; i < r; i++) M[i + (size_t)r * j] = X[i + (size_t)r * j];
    }
    qrcp_steps(r, c, M, perm_out);
    free(M);
    return 0;
}

/* The pivoting step of Sec. 2.1 (the condition of Drmac's convergence
 * proof): QRCP of the leading rows of Vhat -- its rows at the real positions
 * of block I -- over the real positions.  The chosen columns take the front
 * real positions in the order chosen, the others follow in the order QRCP
 * left them; padding positions stay put.  Vhat <- Vhat P, Dhat <- P^T Dhat P. */
static void qrcp_pivot(int k, double *Ah, double *V, int I, int J, int b, int n_real)
{
    int *pos = (int *)malloc(sizeof(int) * (size_t)k);
    int *perm = (int *)malloc(sizeof(int) * (size_t)k);
    int *idx = (int *)malloc(sizeof(int) * (size_t)k);
    int nr = 0, r1 = 0;
    for (int x = 0; x < k; x++) {
        int g = x < b ? I * b + x : J * b + (x - b);
        idx[x] = x;
        if (g < n_real) {
            if (x < b) r1++;
            pos[nr++] = x;
        }
    }
    double *M = (double *)malloc(sizeof(double) * (size_t)(r1 > 0 ? r1 : 1) * (nr > 0 ? nr : 1));
    for (int j = 0; j < nr; j++) {
        perm[j] = j;
        for (int i = 0; i < r1; i++) M[i + (size_t)r1 * j] = AT(V, k, pos[i], pos[j]);
    }
    qrcp_steps(r1, nr, M, perm);
    for (int t = 0; t < nr; t++) idx[pos[t]] = pos[perm[t]];
    double *B = (double *)malloc(sizeof(double) * (size_t)k * k);
    for (int j = 0; j < k; j++)
        for (int i = 0; i < k; i++) AT(B, k, i, j) = AT(Ah, k, idx[i], idx[j]);
    memcpy(Ah, B, sizeof(double) * (size_t)k * k);
    for (int j = 0; j < k; j++)
        for (int i = 0; i < k; i++) AT(B, k, i, j) = AT(V, k, i, idx[j]);
    memcpy(V, B, sizeof(double) * (size_t)k * k);
    free(B);
    free(M);
    free(idx);
    free(perm);
    free(pos);
}

/* ------------------------------------------------------------------ */
/* Blocked two-sided step (Algorithm 2 structure, one group of pairs)      */
/* ------------------------------------------------------------------ */

typedef struct {
    double *Ah, *V;  /* per pair: k x k pivot and eigenvector matrix */
    int rot, sw;
} pair_ws;

/* One parallel step on the np x np working matrix (ld np) with np = N*b.
 * pairs[2*e], pairs[2*e+1] (0-based I<J), npairs of them.  Q may be NULL.
 * Rows, then columns, then the pivot blocks <- Dhat. */
static void evd_step(int np, int n_real, int b, double *A, double *Q, int npairs,
                     const int *pairs, double tol_rel, int inner_max, int order, pair_ws *ws,
                     double *tmp_all, long long *rot_acc, long long *isw_acc)
{
    int k = 2 * b;
    long long rot = 0, isw = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : rot, isw)
    for (int e = 0; e < npairs; e++) {
        int I = pairs[2 * e], J = pairs[2 * e + 1];
        double *Ah = ws[e].Ah;
        for (int jj = 0; jj < k; jj++) {
            int gj = (jj < b) ? I * b + jj : J * b + (jj - b);
            for (int ii = 0; ii < k; ii++) {
                int gi = (ii < b) ? I * b + ii : J * b + (ii - b);
                AT(Ah, k, ii, jj) = AT(A, np, gi, gj);
            }
        }
        int sw = 0;
        ws[e].rot = oracle_pivot_solve(k, Ah, ws[e].V, tol_rel, inner_max, &sw);
        ws[e].sw = sw;
        if (order == 1 && ws[e].rot > 0) {
            double *t = (double *)malloc(sizeof(double) * (size_t)(k + k * k));
            int *ix = (int *)malloc(sizeof(int) * (size_t)k);
            sort_pivot_desc(k, Ah, ws[e].V, t, ix, I, J, b, n_real);
            free(t);
            free(ix);
        } else if (order == 2 && ws[e].rot > 0) {
            qrcp_pivot(k, Ah, ws[e].V, I, J, b, n_real);
        }
        rot += ws[e].rot;
        isw += sw;
    }
    /* rows:  A([I,J], :) <- Vhat^T A([I,J], :)  (Algorithm 2, block-row update) */
#pragma omp parallel for schedule(dynamic, 1)
    for (int e = 0; e < npairs; e++) {
        if (ws[e].rot == 0) continue; /* Vhat == I exactly */
        int I = pairs[2 * e], J = pairs[2 * e + 1];
        const double *V = ws[e].V;
        double *x = tmp_all + (size_t)e * 2 * k, *y = x + k;
        for (int c = 0; c < np; c++) {
            for (int ii = 0; ii < k; ii++) {
                int gi = (ii < b) ? I * b + ii : J * b + (ii - b);
                x[ii] = AT(A, np, gi, c);
            }
            for (int jj = 0; jj < k; jj++) {
                double s = 0.0;
                for (int ii = 0; ii < k; ii++) s += AT(V, k, ii, jj) * x[ii];
                y[jj] = s;
            }
            for (int ii = 0; ii < k; ii++) {
                int gi = (ii < b) ? I * b + ii : J * b + (ii - b);
                AT(A, np, gi, c) = y[ii];
            }
        }
    }
    /* columns: A(:, [I,J]) <- A(:, [I,J]) Vhat, Q likewise */
#pragma omp parallel for schedule(dynamic, 1)
    for (int e = 0; e < npairs; e++) {
        if (ws[e].rot == 0) continue;
        int I = pairs[2 * e], J = pairs[2 * e + 1];
        const double *V = ws[e].V;
        double *x = tmp_all + (size_t)e * 2 * k, *y = x + k;
        for (int m = 0; m < 2; m++) {
            double *M = m == 0 ? A : Q;
            if (!M) continue;
            for (int r = 0; r < np; r++) {
                for (int jj = 0; jj < k; jj++) {
                    int gj = (jj < b) ? I * b + jj : J * b + (jj - b);
                    x[jj] = AT(M, np, r, gj);
                }
                for (int jj = 0; jj < k; jj++) {
                    double s = 0.0;
                    for (int ii = 0; ii < k; ii++) s += x[ii] * AT(V, k, ii, jj);
                    y[jj] = s;
                }
                for (int jj = 0; jj < k; jj++) {
                    int gj = (jj < b) ? I * b + jj : J * b + (jj - b);
                    AT(M, np, r, gj) = y[jj];
                }
            }
        }
    }
    /* pivot blocks <- Dhat (Algorithm 2: A([I,J],[I,J]) <- D) */
    for (int e = 0; e < npairs; e++) {
        if (ws[e].rot == 0) continue;
        int I = pairs[2 * e], J = pairs[2 * e + 1];
        const double *Ah = ws[e].Ah;
        for (int jj = 0; jj < k; jj++) {
            int gj = (jj < b) ? I * b + jj : J * b + (jj - b);
            for (int ii = 0; ii < k; ii++) {
                int gi = (ii < b) ? I * b + ii : J * b + (ii - b);
                AT(A, np, gi, gj) = AT(Ah, k, ii, jj);
            }
        }
    }
    *rot_acc += rot;
    *isw_acc += isw;
}

/* Padded block count for n, b and the ordering (see the readings above). */
int oracle_padded_blocks(int n, int b, int ordering)
{
    int N = (n + b - 1) / b;
    if (N < 2) N = 2;
    if (N % 2) N++;
    (void)ordering;
    return N;
}

static void set_threads(const orc_params *p)
{
#ifdef _OPENMP
    if (p->threads > 0) omp_set_num_threads(p->threads);
#else
    (void)p;
#endif
}

/* Public: one parallel step on an np x np matrix (np = N*b, ld np) with the
 * given pairs; Q may be NULL.  Returns the rotations applied. */
long long oracle_syev_step(int np, int b, double *A, double *Q, int npairs, const int *pairs,
                           double tol_rel, int inner_max, int order)
{
    int k = 2 * b;
    pair_ws *ws = (pair_ws *)calloc((size_t)npairs, sizeof(pair_ws));
    double *buf = (double *)malloc(sizeof(double) * (size_t)npairs * (size_t)(2 * k * k + 2 * k));
    for (int e = 0; e < npairs; e++) {
        ws[e].Ah = buf + (size_t)e * 2 * k * k;
        ws[e].V = ws[e].Ah + (size_t)k * k;
    }
    double *tmp = buf + (size_t)npairs * 2 * k * k;
    long long rot = 0, isw = 0;
    evd_step(np, np, b, A, Q, npairs, pairs, tol_rel, inner_max, order, ws, tmp, &rot, &isw);
    free(ws);
    free(buf);
    return rot;
}

/* Public: blocked two-sided Jacobi (Algorithm 1 swept in the parallel order of
 * Algorithm 2).  Reads the lower triangle of A (n x n, lda) and mirrors it.
 * Outputs: A <- the final (nearly diagonal) iterate, w ascending eigenvalues,
 * Q (if want_vectors) the eigenvectors in the order of w.
 * Return: 0 converged, >0 sweep count when max_sweeps ran out, <0 bad argument. */
int oracle_syev_blocked(int n, double *A, int lda, double *w, double *Q, int ldq,
                        const orc_params *p, orc_stats *st)
{
    if (n < 1 || lda < n || p->b < 1 || (p->want_vectors && ldq < n)) return -1;
    if (p->ordering != ORC_ORDER_ROUND_ROBIN && p->ordering != ORC_ORDER_ANTI_DIAGONAL) return -2;
    set_threads(p);
    int b = p->b, N = oracle_padded_blocks(n, b, p->ordering), np = N * b, k = 2 * b;
    double *Aw = (double *)calloc((size_t)np * np, sizeof(double));
    double *Qw = p->want_vectors ? (double *)calloc((size_t)np * np, sizeof(double)) : NULL;
    for (int j = 0; j < n; j++)
        for (int i = j; i < n; i++) {
            double v = AT(A, lda, i, j);
            AT(Aw, np, i, j) = v;
            AT(Aw, np, j, i) = v;
        }
    if (Qw)
        for (int i = 0; i < np; i++) AT(Qw, np, i, i) = 1.0;
    int maxp = N * (N - 1) / 2;
    int *pairs = (int *)malloc(sizeof(int) * (size_t)(2 * maxp));
    int *sptr = (int *)malloc(sizeof(int) * (size_t)(N + 1));
    int S = oracle_ordering(p->ordering, N, pairs, sptr);
    int maxpp = N / 2;
    pair_ws *ws = (pair_ws *)calloc((size_t)maxpp, sizeof(pair_ws));
    double *buf = (double *)malloc(sizeof(double) * (size_t)maxpp * (size_t)(2 * k * k + 2 * k));
    for (int e = 0; e < maxpp; e++) {
        ws[e].Ah = buf + (size_t)e * 2 * k * k;
        ws[e].V = ws[e].Ah + (size_t)k * k;
    }
    double *tmp = buf + (size_t)maxpp * 2 * k * k;

    orc_stats s;
    memset(&s, 0, sizeof(s));
    s.norm_fro = fro_norm(np, Aw, np);
    double meas = p->conv == ORC_CONV_REL ? rel_off(np, Aw, np) : off_norm(np, Aw, np);
    double target = p->conv == ORC_CONV_REL ? p->tol : p->tol * s.norm_fro;
    s.off_initial = off_norm(np, Aw, np);
    int status = 0, sw = 0;
    double prev = meas;
    if (!(meas <= target)) {
        status = -999;
        for (sw = 0; sw < p->max_sweeps; sw++) {
            for (int st_i = 0; st_i < S; st_i++) {
                int np_st = sptr[st_i + 1] - sptr[st_i];
                evd_step(np, n, b, Aw, Qw, np_st, pairs + 2 * sptr[st_i], p->inner_tol,
                         p->inner_max_sweeps, p->pivot_order, ws, tmp, &s.rotations,
                         &s.inner_sweeps);
                s.steps++;
                s.pair_solves += np_st;
            }
            meas = p->conv == ORC_CONV_REL ? rel_off(np, Aw, np) : off_norm(np, Aw, np);
            if (sw < 64) s.off_hist[sw] = off_norm(np, Aw, np);
            if (sw < 64 && p->conv == ORC_CONV_REL) s.rel_hist[sw] = meas;
            if (meas <= target) { status = 0; sw++; break; }
            if (meas <= 100.0 * target && meas > 0.5 * prev) { status = 0; s.stalled = 1; sw++; break; }
            prev = meas;
        }
        if (status != 0) status = sw;
    }
    s.sweeps = sw;
    s.status = status;
    s.off_final = off_norm(np, Aw, np);
    finalize_evd(n, Aw, np, w, Qw, np, Q, ldq);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) AT(A, lda, i, j) = AT(Aw, np, i, j);
    if (st) *st = s;
    free(Aw);
    free(Qw);
    free(pairs);
    free(sptr);
    free(ws);
    free(buf);
    return status;
}

/* Public: scalar cyclic Jacobi (Algorithm 1 with b = 1, row-cyclic order
 * p < q, one rotation at a time).  Same I/O contract as the blocked form;
 * a rotation is applied when |a_pq| > inner_tol * sqrt|a_pp| sqrt|a_qq|. */
int oracle_syev_scalar(int n, double *A, int lda, double *w, double *Q, int ldq,
                       const orc_params *p, orc_stats *st)
{
    if (n < 1 || lda < n || (p->want_vectors && ldq < n)) return -1;
    double *Aw = (double *)calloc((size_t)n * n, sizeof(double));
    double *Qw = p->want_vectors ? (double *)calloc((size_t)n * n, sizeof(double)) : NULL;
    for (int j = 0; j < n; j++)
        for (int i = j; i < n; i++) {
            AT(Aw, n, i, j) = AT(A, lda, i, j);
            AT(Aw, n, j, i) = AT(A, lda, i, j);
        }
    if (Qw)
        for (int i = 0; i < n; i++) AT(Qw, n, i, i) = 1.0;
    orc_stats s;
    memset(&s, 0, sizeof(s));
    s.norm_fro = fro_norm(n, Aw, n);
    s.off_initial = off_norm(n, Aw, n);
    double meas = p->conv == ORC_CONV_REL ? rel_off(n, Aw, n) : s.off_initial;
    double target = p->conv == ORC_CONV_REL ? p->tol : p->tol * s.norm_fro;
    int status = 0, sw = 0;
    double prev = meas;
    if (!(meas <= target)) {
        status = -999;
        for (sw = 0; sw < p->max_sweeps; sw++) {
            long long in_sweep = 0;
            for (int pp = 0; pp < n - 1; pp++)
                for (int q = pp + 1; q < n; q++) {
                    if (!rotation_wanted(AT(Aw, n, pp, pp), AT(Aw, n, q, q), AT(Aw, n, pp, q),
                                         p->inner_tol))
                        continue;
                    in_sweep += oracle_rotate(n, Aw, n, Qw, n, pp, q);
                }
            s.rotations += in_sweep;
            meas = p->conv == ORC_CONV_REL ? rel_off(n, Aw, n) : off_norm(n, Aw, n);
            if (sw < 64) s.off_hist[sw] = off_norm(n, Aw, n);
            if (sw < 64 && p->conv == ORC_CONV_REL) s.rel_hist[sw] = meas;
            if (meas <= target || in_sweep == 0) { status = 0; sw++; break; }
            if (meas <= 100.0 * target && meas > 0.5 * prev) { status = 0; s.stalled = 1; sw++; break; }
            prev = meas;
        }
        if (status != 0) status = sw;
    }
    s.sweeps = sw;
    s.status = status;
    s.off_final = off_norm(n, Aw, n);
    finalize_evd(n, Aw, n, w, Qw, n, Q, ldq);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) AT(A, lda, i, j) = AT(Aw, n, i, j);
    if (st) *st = s;
    free(Aw);
    free(Qw);
    return status;
}

/* ------------------------------------------------------------------ */
/* One-sided Jacobi SVD (Algorithm 6)                                   */
/* ------------------------------------------------------------------ */

/* Normalised off-diagonal measure of a Gram block: max_{i!=j}
 * |a_ij| / (sqrt(a_ii) sqrt(a_jj)); a pair with a zero column counts as 0. */
static double gram_rel_off(int k, const double *Ah)
{
    double m = 0.0;
    for (int j = 0; j < k; j++)
        for (int i = 0; i < k; i++) {
            if (i == j) continue;
            double d = sqrt(AT(Ah, k, i, i)) * sqrt(AT(Ah, k, j, j));
            if (d == 0.0) continue;
            double r = fabs(AT(Ah, k, i, j)) / d;
            if (r > m) m = r;
        }
    return m;
}

/* Public: Gram block Ahat = G(:,[I,J])^T G(:,[I,J]) of an m x np matrix
 * (ld ldg), eq. (SVD_subproblem): a plain dot product per entry. */
void oracle_gram_pair(int m, int b, const double *G, int ldg, int I, int J, double *Ah)
{
    int k = 2 * b;
    for (int jj = 0; jj < k; jj++) {
        int gj = (jj < b) ? I * b + jj : J * b + (jj - b);
        for (int ii = 0; ii < k; ii++) {
            int gi = (ii < b) ? I * b + ii : J * b + (ii - b);
            double s = 0.0;
            for (int r = 0; r < m; r++) s += AT(G, ldg, r, gi) * AT(G, ldg, r, gj);
            AT(Ah, k, ii, jj) = s;
        }
    }
}

/* One step of the one-sided method over disjoint column pairs.  Returns the
 * step's maximum normalised Gram off-diagonal (before rotation). */
static double svd_step(int m, int np, int n_real, int b, double *G, int ldg, double *V,
                       int npairs, const int *pairs, double tol_rel, int inner_max, int order,
                       pair_ws *ws, double *tmp_all, long long *rot_acc, long long *isw_acc)
{
    int k = 2 * b;
    long long rot = 0, isw = 0;
    double mx = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : rot, isw) reduction(max : mx)
    for (int e = 0; e < npairs; e++) {
        int I = pairs[2 * e], J = pairs[2 * e + 1];
        oracle_gram_pair(m, b, G, ldg, I, J, ws[e].Ah);
        double r = gram_rel_off(k, ws[e].Ah);
        if (r > mx) mx = r;
        int sw = 0;
        ws[e].rot = oracle_pivot_solve(k, ws[e].Ah, ws[e].V, tol_rel, inner_max, &sw);
        ws[e].sw = sw;
        if (order == 1 && ws[e].rot > 0) {
            double *t = (double *)malloc(sizeof(double) * (size_t)(k + k * k));
            int *ix = (int *)malloc(sizeof(int) * (size_t)k);
            sort_pivot_desc(k, ws[e].Ah, ws[e].V, t, ix, I, J, b, n_real);
            free(t);
            free(ix);
        } else if (order == 2 && ws[e].rot > 0) {
            qrcp_pivot(k, ws[e].Ah, ws[e].V, I, J, b, n_real);
        }
        rot += ws[e].rot;
        isw += sw;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int e = 0; e < npairs; e++) {
        if (ws[e].rot == 0) continue;
        int I = pairs[2 * e], J = pairs[2 * e + 1];
        const double *Vh = ws[e].V;
        double *x = tmp_all + (size_t)e * 2 * k, *y = x + k;
        for (int mm = 0; mm < 2; mm++) {
            double *M = mm == 0 ? G : V;
            if (!M) continue;
            int rows = mm == 0 ? m : np, ld = mm == 0 ? ldg : np;
            for (int r = 0; r < rows; r++) {
                for (int jj = 0; jj < k; jj++) {
                    int gj = (jj < b) ? I * b + jj : J * b + (jj - b);
                    x[jj] = AT(M, ld, r, gj);
                }
                for (int jj = 0; jj < k; jj++) {
                    double s = 0.0;
                    for (int ii = 0; ii < k; ii++) s += x[ii] * AT(Vh, k, ii, jj);
                    y[jj] = s;
                }
                for (int jj = 0; jj < k; jj++) {
                    int gj = (jj < b) ? I * b + jj : J * b + (jj - b);
                    AT(M, ld, r, gj) = y[jj];
                }
            }
        }
    }
    *rot_acc += rot;
    *isw_acc += isw;
    return mx;
}

/* SVD finalisation (the output step of Algorithm 6): sigma_i = ||g_i||_2,
 * u_i = g_i / sigma_i (0 when sigma_i == 0), sorted descending (stable). */
static void finalize_svd(int m, int n, double *Gw, int ldgw, double *G, int ldg,
                         double *sigma, double *Vw, int ldvw, double *V, int ldv)
{
    double *sg = (double *)malloc(sizeof(double) * (size_t)n);
    int *idx = (int *)malloc(sizeof(int) * (size_t)n);
    for (int j = 0; j < n; j++) {
        double s = 0.0;
        for (int r = 0; r < m; r++) s += AT(Gw, ldgw, r, j) * AT(Gw, ldgw, r, j);
        sg[j] = sqrt(s);
    }
    stable_argsort(n, sg, idx, 0);
    for (int j = 0; j < n; j++) {
        int c = idx[j];
        sigma[j] = sg[c];
        for (int r = 0; r < m; r++)
            AT(G, ldg, r, j) = sg[c] > 0.0 ? AT(Gw, ldgw, r, c) / sg[c] : 0.0;
        if (V && Vw)
            for (int r = 0; r < n; r++) AT(V, ldv, r, j) = AT(Vw, ldvw, r, c);
    }
    free(sg);
    free(idx);
}

/* Public: one step of the one-sided method on G (m x np, ld ldg) and V
 * (np x np, ld np, may be NULL).  Returns the max normalised Gram off-diagonal. */
double oracle_gesvd_step(int m, int np, int b, double *G, int ldg, double *V, int npairs,
                         const int *pairs, double tol_rel, int inner_max, int order)
{
    int k = 2 * b;
    pair_ws *ws = (pair_ws *)calloc((size_t)npairs, sizeof(pair_ws));
    double *buf = (double *)malloc(sizeof(double) * (size_t)npairs * (size_t)(2 * k * k + 2 * k));
    for (int e = 0; e < npairs; e++) {
        ws[e].Ah = buf + (size_t)e * 2 * k * k;
        ws[e].V = ws[e].Ah + (size_t)k * k;
    }
    long long rot = 0, isw = 0;
    double mx = svd_step(m, np, np, b, G, ldg, V, npairs, pairs, tol_rel, inner_max, order, ws,
                         buf + (size_t)npairs * 2 * k * k, &rot, &isw);
    free(ws);
    free(buf);
    return mx;
}

/* Public: blocked one-sided Jacobi SVD (Algorithm 6 in the parallel order).
 * G (m x n, ldg, m >= n) is overwritten by U; sigma (n) descending; V (n x n,
 * ldv) if want_vectors.  The inner threshold and the stop test both use
 * p->tol: stop when a sweep's maximum normalised Gram off-diagonal <= tol
 * (or the stall rule).  Return as for oracle_syev_blocked. */
int oracle_gesvd_blocked(int m, int n, double *G, int ldg, double *sigma, double *V, int ldv,
                         const orc_params *p, orc_stats *st)
{
    if (n < 1 || m < n || ldg < m || p->b < 1 || (p->want_vectors && ldv < n)) return -1;
    set_threads(p);
    int b = p->b, N = oracle_padded_blocks(n, b, p->ordering), np = N * b, k = 2 * b;
    double *Gw = (double *)calloc((size_t)m * np, sizeof(double));
    double *Vw = p->want_vectors ? (double *)calloc((size_t)np * np, sizeof(double)) : NULL;
    for (int j = 0; j < n; j++)
        for (int r = 0; r < m; r++) AT(Gw, m, r, j) = AT(G, ldg, r, j);
    if (Vw)
        for (int i = 0; i < np; i++) AT(Vw, np, i, i) = 1.0;
    int maxp = N * (N - 1) / 2;
    int *pairs = (int *)malloc(sizeof(int) * (size_t)(2 * maxp));
    int *sptr = (int *)malloc(sizeof(int) * (size_t)(N + 1));
    int S = oracle_ordering(p->ordering, N, pairs, sptr);
    int maxpp = N / 2;
    pair_ws *ws = (pair_ws *)calloc((size_t)maxpp, sizeof(pair_ws));
    double *buf = (double *)malloc(sizeof(double) * (size_t)maxpp * (size_t)(2 * k * k + 2 * k));
    for (int e = 0; e < maxpp; e++) {
        ws[e].Ah = buf + (size_t)e * 2 * k * k;
        ws[e].V = ws[e].Ah + (size_t)k * k;
    }
    double *tmp = buf + (size_t)maxpp * 2 * k * k;
    orc_stats s;
    memset(&s, 0, sizeof(s));
    int status = -999, sw = 0;
    double prev = INFINITY;
    for (sw = 0; sw < p->max_sweeps; sw++) {
        double mx = 0.0;
        long long rot_before = s.rotations;
        for (int st_i = 0; st_i < S; st_i++) {
            int np_st = sptr[st_i + 1] - sptr[st_i];
            double r = svd_step(m, np, n, b, Gw, m, Vw, np_st, pairs + 2 * sptr[st_i], p->tol,
                                p->inner_max_sweeps, p->pivot_order, ws, tmp, &s.rotations,
                                &s.inner_sweeps);
            if (r > mx) mx = r;
            s.steps++;
            s.pair_solves += np_st;
        }
        if (sw < 64) s.off_hist[sw] = mx;
        if (sw == 0) s.off_initial = mx;
        s.off_final = mx;
        if (mx <= p->tol || s.rotations == rot_before) { status = 0; sw++; break; }
        if (mx <= 100.0 * p->tol && mx > 0.5 * prev) { status = 0; s.stalled = 1; sw++; break; }
        prev = mx;
    }
    if (status != 0) status = sw;
    s.sweeps = sw;
    s.status = status;
    finalize_svd(m, n, Gw, m, G, ldg, sigma, Vw, np, V, ldv);
    if (st) *st = s;
    free(Gw);
    free(Vw);
    free(pairs);
    free(sptr);
    free(ws);
    free(buf);
    return status;
}

/* Public: scalar one-sided (Hestenes) Jacobi, row-cyclic p < q:
 * alpha = ||g_p||^2, beta = ||g_q||^2, gamma = g_p^T g_q; rotate when
 * |gamma| > tol sqrt(alpha) sqrt(beta) with the 2x2 rotation of
 * [[alpha, gamma],[gamma, beta]].  Stop after a sweep with no rotation. */
int oracle_gesvd_scalar(int m, int n, double *G, int ldg, double *sigma, double *V, int ldv,
                        const orc_params *p, orc_stats *st)
{
    if (n < 1 || m < n || ldg < m || (p->want_vectors && ldv < n)) return -1;
    double *Gw = (double *)malloc(sizeof(double) * (size_t)m * n);
    double *Vw = p->want_vectors ? (double *)calloc((size_t)n * n, sizeof(double)) : NULL;
    for (int j = 0; j < n; j++)
        for (int r = 0; r < m; r++) AT(Gw, m, r, j) = AT(G, ldg, r, j);
    if (Vw)
        for (int i = 0; i < n; i++) AT(Vw, n, i, i) = 1.0;
    orc_stats s;
    memset(&s, 0, sizeof(s));
    int status = -999, sw = 0;
    for (sw = 0; sw < p->max_sweeps; sw++) {
        long long in_sweep = 0;
        double mx = 0.0;
        for (int pp = 0; pp < n - 1; pp++)
            for (int q = pp + 1; q < n; q++) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int r = 0; r < m; r++) {
                    double x = AT(Gw, m, r, pp), y = AT(Gw, m, r, q);
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                double d = sqrt(al) * sqrt(be);
                if (d > 0.0 && fabs(ga) / d > mx) mx = fabs(ga) / d;
                if (!rotation_wanted(al, be, ga, p->tol)) continue;
                double c, sn, t;
                oracle_rotation(al, be, ga, &c, &sn, &t);
                double tau = sn / (1.0 + c);
                for (int r = 0; r < m; r++) rot_apply(sn, tau, &AT(Gw, m, r, pp), &AT(Gw, m, r, q));
                if (Vw)
                    for (int r = 0; r < n; r++)
                        rot_apply(sn, tau, &AT(Vw, n, r, pp), &AT(Vw, n, r, q));
                in_sweep++;
            }
        s.rotations += in_sweep;
        if (sw < 64) s.off_hist[sw] = mx;
        s.off_final = mx;
        if (in_sweep == 0) { status = 0; sw++; break; }
    }
    if (status != 0) status = sw;
    s.sweeps = sw;
    s.status = status;
    finalize_svd(m, n, Gw, m, G, ldg, sigma, Vw, n, V, ldv);
    if (st) *st = s;
    free(Gw);
    free(Vw);
    return status;
}

/* ------------------------------------------------------------------ */
/* Split-precision operand model for the mixed-precision form             */
/* ------------------------------------------------------------------ */

/* Round an IEEE binary32 to the nearest bfloat16 (ties to even), returned as
 * the binary32 holding that value.  Written from the formats' definitions:
 * bfloat16 keeps the top 16 bits of a binary32. */
static float bf16_round(float x)
{
    unsigned int u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) { /* inf / nan: truncate, keep nan quiet */
        if (u & 0x007fffffu) u |= 0x00400000u;
        u &= 0xffff0000u;
    } else {
        unsigned int lsb = (u >> 16) & 1u;
        u += 0x7fffu + lsb;
        u &= 0xffff0000u;
    }
    float r;
    memcpy(&r, &u, 4);
    return r;
}

/* hi = bf16(x), lo = bf16(x - hi); x - hi is exact in binary32. */
void oracle_split_bf16(int n, const float *x, float *hi, float *lo)
{
    for (int i = 0; i < n; i++) {
        float h = bf16_round(x[i]);
        hi[i] = h;
        lo[i] = bf16_round(x[i] - h);
    }
}
