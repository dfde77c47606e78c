/*
 * spamm_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 CPU statement of what the library computes, written
 * from the paper (Bock, Challacombe, Kale, "Solvers for O(N) Electronic
 * Structure in the Strong Scaling Limit", arXiv:1403.7458) and from the
 * cited second-order spectral projection (SP2) method.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the CUDA
 * library shares no code, header or helper with it.
 *
 * Contents
 *   - leaf Frobenius norms, squared (Sec. 2, Eq. 2), accumulated exactly in
 *     double-double and rounded once;
 *   - the norm quadtree (Sec. 2, Eqs. 1 and 3), each parent the once-rounded
 *     sum of its four children's squared norms;
 *   - SpAMM as the recursive octree walk of Algorithm 1 (Sec. 3.1) with the
 *     culling rule of Eq. 4, applied to squared norms;
 *   - a brute-force flat enumeration of the surviving leaf triples;
 *   - a dense triple-loop product;
 *   - Gershgorin spectral bounds and the SP2 iteration.
 *
 * Readings where the paper is silent (stated again in the repository's design
 * notes):
 *   - "||A|| ||B|| > tau" is evaluated as  n2A * n2B > tau * tau  in FP64 on
 *     squared norms; equality is culled (strict ">");
 *   - the root node is tested like every other node;
 *   - children are visited in (i, j, k) order with k innermost, so each
 *     output leaf receives its products in increasing k;
 *   - padding to a power of two is virtual: missing leaves have norm 0 and
 *     are never multiplied;
 *   - SP2 chooses X^2 when |tr X^2 - Ne| < |2 tr X - tr X^2 - Ne|, else
 *     2X - X^2 (ties go to 2X - X^2); rule 1 is the simpler "tr X > Ne".
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fused
 * multiply-add is introduced except the explicit fma() of TwoProd).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------- */
/* Double-double accumulation (Knuth's TwoSum, Dekker/FMA TwoProd).        */
/* ---------------------------------------------------------------------- */

typedef struct { double hi, lo; } ora_dd;

static void ora_two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}

static void ora_fast_two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    *s = x;
    *e = b - (x - a);
}

/* (hi, lo) + (p, q), accurate double-double addition. */
static ora_dd ora_dd_add(ora_dd x, double p, double q)
{
    double s, e, t, f;
    ora_two_sum(x.hi, p, &s, &e);
    ora_two_sum(x.lo, q, &t, &f);
    e += t;
    ora_fast_two_sum(s, e, &s, &e);
    e += f;
    ora_dd r;
    ora_fast_two_sum(s, e, &r.hi, &r.lo);
    return r;
}

static ora_dd ora_dd_add_sq(ora_dd x, double a)
{
    double p = a * a;
    double q = fma(a, a, -p);
    return ora_dd_add(x, p, q);
}

static double ora_dd_round(ora_dd x) { return x.hi + x.lo; }

/* ---------------------------------------------------------------------- */
/* Norm quadtree (Sec. 2, Eqs. 1-3).                                       */
/* ---------------------------------------------------------------------- */

static int64_t ora_ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

/* Depth d of the quadtree: the smallest d with 2^d >= nb. */
int ora_depth(int64_t nb)
{
    int d = 0;
    while (((int64_t)1 << d) < nb) d++;
    return d;
}

/* Squared Frobenius norm of every leaf (Eq. 2 squared).  a is n x n row-major
 * with leading dimension lda; the leaf tier is written as a P x P row-major
 * grid, P = 2^depth, padding leaves zero.  Each value is the exact sum of the
 * exact squares, rounded once to FP64 (double-double accumulation). */
void ora_leaf_norms2(const double *a, int64_t n, int64_t lda, int b, double *n2)
{
    int64_t nb = ora_ceil_div(n, b);
    int64_t P = (int64_t)1 << ora_depth(nb);
    for (int64_t I = 0; I < P; I++) {
        for (int64_t K = 0; K < P; K++) {
            ora_dd s = {0.0, 0.0};
            if (I < nb && K < nb) {
                for (int64_t r = I * b; r < (I + 1) * b && r < n; r++)
                    for (int64_t c = K * b; c < (K + 1) * b && c < n; c++)
                        s = ora_dd_add_sq(s, a[r * lda + c]);
            }
            n2[I * P + K] = ora_dd_round(s);
        }
    }
}

/* Offset of tier t inside the concatenated pyramid: sum_{s<t} 4^s. */
int64_t ora_tier_offset(int t)
{
    return (((int64_t)1 << (2 * t)) - 1) / 3;
}

/* Squared norms of all tiers t = 0..depth, concatenated, tier t a 2^t x 2^t
 * row-major grid.  Tier `depth` is copied from leaf_n2; a parent is the sum of
 * its four children (Eq. 3 squared), accumulated exactly and rounded once. */
void ora_norm_pyramid(const double *leaf_n2, int depth, double *tiers)
{
    int64_t P = (int64_t)1 << depth;
    memcpy(tiers + ora_tier_offset(depth), leaf_n2, sizeof(double) * P * P);
    for (int t = depth - 1; t >= 0; t--) {
        int64_t W = (int64_t)1 << t;
        const double *child = tiers + ora_tier_offset(t + 1);
        double *par = tiers + ora_tier_offset(t);
        for (int64_t I = 0; I < W; I++) {
            for (int64_t J = 0; J < W; J++) {
                ora_dd s = {0.0, 0.0};
                for (int i = 0; i < 2; i++)
                    for (int j = 0; j < 2; j++)
                        s = ora_dd_add(s, child[(2 * I + i) * (2 * W) + (2 * J + j)], 0.0);
                par[I * W + J] = ora_dd_round(s);
            }
        }
    }
}

/* The culling predicate of Eq. 4 on squared norms: keep iff n2a*n2b > tau^2. */
static int ora_keep(double n2a, double n2b, double tau2)
{
    return n2a * n2b > tau2;
}

/* ---------------------------------------------------------------------- */
/* SpAMM, recursive (Algorithm 1).                                          */
/* ---------------------------------------------------------------------- */

typedef struct {
    const double *A, *B;
    double *C;
    int64_t n, lda, ldb, ldc;
    int b, depth;
    const double *tA, *tB; /* norm pyramids */
    double tau2;
    int32_t *tasks;        /* optional (i, k, j) triples, in visit order */
    int64_t cap, ntask;
    int par_tiers;         /* spawn OpenMP tasks per (i, j) child above this tier */
} ora_ctx;

/* Dense leaf product C_IJ += A_IK B_KJ over the rows and columns that exist
 * (three nested loops, Algorithm 1's leaf branch). */
static void ora_leaf_product(const ora_ctx *x, int64_t I, int64_t K, int64_t J)
{
    int64_t r0 = I * x->b, r1 = r0 + x->b < x->n ? r0 + x->b : x->n;
    int64_t l0 = K * x->b, l1 = l0 + x->b < x->n ? l0 + x->b : x->n;
    int64_t c0 = J * x->b, c1 = c0 + x->b < x->n ? c0 + x->b : x->n;
    for (int64_t r = r0; r < r1; r++) {
        double *crow = x->C + r * x->ldc;
        for (int64_t l = l0; l < l1; l++) {
            double arl = x->A[r * x->lda + l];
            const double *brow = x->B + l * x->ldb;
            for (int64_t c = c0; c < c1; c++)
                crow[c] = crow[c] + arl * brow[c];
        }
    }
}

static double ora_node(const double *tiers, int t, int64_t I, int64_t J)
{
    return tiers[ora_tier_offset(t) + I * ((int64_t)1 << t) + J];
}

/* SpAMM_omp(tau, t, A^t_IK, B^t_KJ, C^t_IJ) of Algorithm 1, without the lock:
 * the OpenMP variant below gives every (i, j) child to one task, so no two
 * tasks write the same C leaf. */
static void ora_spamm_rec(ora_ctx *x, int t, int64_t I, int64_t K, int64_t J)
{
    if (t < x->depth) {
        int spawn = t < x->par_tiers;
        for (int i = 0; i < 2; i++) {
            for (int j = 0; j < 2; j++) {
                int64_t cI = 2 * I + i, cJ = 2 * J + j;
                if (spawn) {
#pragma omp task firstprivate(cI, cJ) untied
                    for (int k = 0; k < 2; k++) {
                        int64_t cK = 2 * K + k;
                        if (ora_keep(ora_node(x->tA, t + 1, cI, cK),
                                     ora_node(x->tB, t + 1, cK, cJ), x->tau2))
                            ora_spamm_rec(x, t + 1, cI, cK, cJ);
                    }
                } else {
                    for (int k = 0; k < 2; k++) {
                        int64_t cK = 2 * K + k;
                        if (ora_keep(ora_node(x->tA, t + 1, cI, cK),
                                     ora_node(x->tB, t + 1, cK, cJ), x->tau2))
                            ora_spamm_rec(x, t + 1, cI, cK, cJ);
                    }
                }
            }
        }
        if (spawn) {
#pragma omp taskwait
        }
    } else {
        if (x->tasks) {
            if (x->ntask < x->cap) {
                x->tasks[3 * x->ntask + 0] = (int32_t)I;
                x->tasks[3 * x->ntask + 1] = (int32_t)K;
                x->tasks[3 * x->ntask + 2] = (int32_t)J;
            }
            x->ntask++;
        }
        ora_leaf_product(x, I, K, J);
    }
}

static double *ora_pyramid_of(const double *a, int64_t n, int64_t lda, int b, int depth)
{
    int64_t P = (int64_t)1 << depth;
    double *leaf = (double *)malloc(sizeof(double) * P * P);
    double *tiers = (double *)malloc(sizeof(double) * ora_tier_offset(depth + 1));
    if (!leaf || !tiers) { free(leaf); free(tiers); return NULL; }
    ora_leaf_norms2(a, n, lda, b, leaf);
    ora_norm_pyramid(leaf, depth, tiers);
    free(leaf);
    return tiers;
}

/* C = SpAMM(A, B, tau) for n x n row-major matrices (C is overwritten).
 * If tasks != NULL the surviving (i, k, j) leaf triples are recorded in visit
 * order (up to cap of them) and the walk runs on one thread; *ntask receives
 * the total.  nthreads <= 0 uses the OpenMP default.  Returns 0, or -2 when
 * memory runs out. */
int ora_spamm(const double *A, int64_t lda, const double *B, int64_t ldb,
              double *C, int64_t ldc, int64_t n, int b, double tau,
              int32_t *tasks, int64_t cap, int64_t *ntask, int nthreads)
{
    int64_t nb = ora_ceil_div(n, b);
    int depth = ora_depth(nb);
    ora_ctx x;
    memset(&x, 0, sizeof(x));
    x.A = A; x.B = B; x.C = C;
    x.n = n; x.lda = lda; x.ldb = ldb; x.ldc = ldc;
    x.b = b; x.depth = depth;
    x.tau2 = tau * tau;
    x.tasks = tasks; x.cap = cap; x.ntask = 0;
    x.tA = ora_pyramid_of(A, n, lda, b, depth);
    x.tB = ora_pyramid_of(B, n, ldb, b, depth);
    if (!x.tA || !x.tB) {
        free((void *)x.tA); free((void *)x.tB);
        return -2;
    }
    for (int64_t r = 0; r < n; r++)
        memset(C + r * ldc, 0, sizeof(double) * n);
    if (ora_keep(ora_node(x.tA, 0, 0, 0), ora_node(x.tB, 0, 0, 0), x.tau2)) {
        if (tasks) {
            x.par_tiers = 0;
            ora_spamm_rec(&x, 0, 0, 0, 0);
        } else {
            x.par_tiers = 3;
#ifdef _OPENMP
            int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
#pragma omp single
#endif
            ora_spamm_rec(&x, 0, 0, 0, 0);
        }
    }
    (void)nthreads;
    if (ntask) *ntask = x.ntask;
    free((void *)x.tA);
    free((void *)x.tB);
    return 0;
}

/* Every leaf triple (i, k, j), i, k, j < nb, with n2A[i,k] * n2B[k,j] > tau^2,
 * in (i, j, k) lexicographic order: the brute-force O(nb^3) statement of the
 * culled product set.  Leaf grids are P x P row-major, P = 2^depth. */
int64_t ora_flat_tasks(const double *n2A, const double *n2B, int64_t nb, int64_t P,
                       double tau, int32_t *tasks, int64_t cap)
{
    double tau2 = tau * tau;
    int64_t cnt = 0;
    for (int64_t i = 0; i < nb; i++)
        for (int64_t j = 0; j < nb; j++)
            for (int64_t k = 0; k < nb; k++)
                if (ora_keep(n2A[i * P + k], n2B[k * P + j], tau2)) {
                    if (tasks && cnt < cap) {
                        tasks[3 * cnt + 0] = (int32_t)i;
                        tasks[3 * cnt + 1] = (int32_t)k;
                        tasks[3 * cnt + 2] = (int32_t)j;
                    }
                    cnt++;
                }
    return cnt;
}

/* Dense C = A B, three loops, FP64. */
void ora_gemm(const double *A, const double *B, double *C, int64_t n)
{
    memset(C, 0, sizeof(double) * n * n);
    for (int64_t r = 0; r < n; r++)
        for (int64_t l = 0; l < n; l++) {
            double arl = A[r * n + l];
            for (int64_t c = 0; c < n; c++)
                C[r * n + c] = C[r * n + c] + arl * B[l * n + c];
        }
}

/* ---------------------------------------------------------------------- */
/* SP2 (second-order spectral projection, Niklasson 2002, cited in Sec. 4). */
/* ---------------------------------------------------------------------- */

/* Gershgorin bounds: emin = min_i (f_ii - sum_{j!=i} |f_ij|),
 *                    emax = max_i (f_ii + sum_{j!=i} |f_ij|). */
void ora_gershgorin(const double *F, int64_t n, double *emin, double *emax)
{
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t j = 0; j < n; j++)
            if (j != i) s += fabs(F[i * n + j]);
        double d = F[i * n + i];
        if (d - s < lo) lo = d - s;
        if (d + s > hi) hi = d + s;
    }
    *emin = lo;
    *emax = hi;
}

static double ora_trace(const double *X, int64_t n)
{
    double t = 0.0;
    for (int64_t i = 0; i < n; i++) t += X[i * n + i];
    return t;
}

/* SP2 history row layout (per iteration). */
enum { ORA_H_TR = 0, ORA_H_TR2 = 1, ORA_H_IDEM = 2, ORA_H_BRANCH = 3,
       ORA_H_TASKS = 4, ORA_H_TRNEW = 5, ORA_H_COLS = 6 };

/* Stop reasons. */
enum { ORA_STOP_CONVERGED = 0, ORA_STOP_STAGNATED = 1, ORA_STOP_FIXED = 2,
       ORA_STOP_MAXITER = 3 };

/*
 * P = SP2(F, Ne, tau).  X0 = (emax I - F) / (emax - emin); each iteration
 * forms X2 = SpAMM(X, X, tau), t1 = tr X, t2 = tr X2, e = ||X2 - X||_F, picks
 * the branch (rule 0: X2 iff |t2 - Ne| < |2 t1 - t2 - Ne|; rule 1: X2 iff
 * t1 > Ne) and replaces X by X2 or 2X - X2.
 *
 * Stopping (checked after each update): fixed_iters > 0 runs exactly that
 * many iterations; otherwise stop when |tr X_new - Ne| < trace_tol and
 * e < idem_tol (converged), or when e < 1e-3 and e > 0.5 e_{n-2}
 * (stagnated: the SpAMM error floor is reached), or after max_iter.
 *
 * hist receives ORA_H_COLS doubles per iteration: tr X, tr X2, e, branch
 * (1 = X2, 0 = 2X - X2), surviving leaf triples, tr X_new.  Returns the
 * number of iterations; *stop gets the stop reason.  -2 when memory runs out.
 */
int ora_sp2(const double *F, int64_t n, int b, double Ne, double tau,
            int max_iter, int rule, double trace_tol, double idem_tol,
            int fixed_iters, double *P, double *hist, int *stop, int nthreads)
{
    double emin, emax;
    ora_gershgorin(F, n, &emin, &emax);
    double *X = P;
    double *X2 = (double *)malloc(sizeof(double) * n * n);
    if (!X2) return -2;
    double range = emax - emin;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++)
            X[i * n + j] = ((i == j ? emax : 0.0) - F[i * n + j]) / range;

    int it = 0;
    int reason = ORA_STOP_MAXITER;
    int limit = fixed_iters > 0 ? fixed_iters : max_iter;
    double ehist[3] = {INFINITY, INFINITY, INFINITY};
    while (it < limit) {
        int64_t nt = 0;
        int rc;
        /* The task count is only needed for the history; count it with the
         * flat enumeration of the same predicate (equal sets, see tests). */
        rc = ora_spamm(X, n, X, n, X2, n, n, b, tau, NULL, 0, NULL, nthreads);
        if (rc) { free(X2); return rc; }
        {
            int64_t nb = ora_ceil_div(n, b);
            int depth = ora_depth(nb);
            int64_t PP = (int64_t)1 << depth;
            double *lx = (double *)malloc(sizeof(double) * PP * PP);
            if (!lx) { free(X2); return -2; }
            ora_leaf_norms2(X, n, n, b, lx);
            nt = ora_flat_tasks(lx, lx, nb, PP, tau, NULL, 0);
            free(lx);
        }
        double t1 = ora_trace(X, n);
        double t2 = ora_trace(X2, n);
        double e2 = 0.0;
        for (int64_t q = 0; q < n * n; q++) {
            double d = X2[q] - X[q];
            e2 += d * d;
        }
        double e = sqrt(e2);
        int take_sq;
        if (rule == 1)
            take_sq = t1 > Ne;
        else
            take_sq = fabs(t2 - Ne) < fabs(2.0 * t1 - t2 - Ne);
        if (take_sq) {
            memcpy(X, X2, sizeof(double) * n * n);
        } else {
            for (int64_t q = 0; q < n * n; q++) X[q] = 2.0 * X[q] - X2[q];
        }
        double tn = ora_trace(X, n);
        if (hist) {
            double *h = hist + (int64_t)it * ORA_H_COLS;
            h[ORA_H_TR] = t1;
            h[ORA_H_TR2] = t2;
            h[ORA_H_IDEM] = e;
            h[ORA_H_BRANCH] = take_sq ? 1.0 : 0.0;
            h[ORA_H_TASKS] = (double)nt;
            h[ORA_H_TRNEW] = tn;
        }
        ehist[0] = ehist[1];
        ehist[1] = ehist[2];
        ehist[2] = e;
        it++;
        if (fixed_iters > 0) {
            if (it == fixed_iters) reason = ORA_STOP_FIXED;
            continue;
        }
        if (fabs(tn - Ne) < trace_tol && e < idem_tol) {
            reason = ORA_STOP_CONVERGED;
            break;
        }
        if (it >= 3 && e < 1e-3 && e > 0.5 * ehist[0]) {
            reason = ORA_STOP_STAGNATED;
            break;
        }
    }
    free(X2);
    if (stop) *stop = reason;
    return it;
}

int ora_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
