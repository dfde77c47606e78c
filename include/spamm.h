/*
 * spamm.h -- C ABI of the GB300 (sm_103a) SpAMM / SP2 library.
 *
 * The library implements the Sparse Approximate Matrix Multiply (SpAMM) of
 * Bock, Challacombe and Kale, "Solvers for O(N) Electronic Structure in the
 * Strong Scaling Limit" (arXiv:1403.7458), Sec. 2, Eqs. 1-4 and Algorithm 1,
 * and the second-order spectral projection (SP2) loop that the paper drives
 * with it (Sec. 4).  All arithmetic runs in the library's own CUDA kernels.
 *
 * Conventions shared by every entry point
 *   - Return value: SPAMM_OK (0) or a negative SPAMM_E_* code.  A short text
 *     for the last failure on the calling thread is in spamm_last_error().
 *   - Matrices are square, n x n, FP64, row-major with a leading dimension
 *     (elements, >= n).  Pointers passed as matrix data may be host or device
 *     memory; the library asks the CUDA runtime which one it is.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *     device work is enqueued on it; only the calls documented as blocking
 *     wait for it.
 *   - Handles (spamm_mat_t) own their device memory, are created by the
 *     library and released with spamm_free().  Inputs are never modified.
 *     Device memory is drawn from the library's own stream-ordered pool,
 *     which keeps freed memory cached until spamm_trim().
 *   - Matrices are cut into b x b leaves (b = 16, 32 or 64).  The leaf grid
 *     is nb x nb, nb = ceil(n / b); the norm quadtree has depth d with
 *     2^d >= nb, tier 0 the root, tier d the leaves.  Padding up to 2^d is
 *     virtual: padding leaves have norm 0 and are never multiplied.  The
 *     ragged last leaf row and column are zero-filled.
 */
#ifndef SPAMM_H
#define SPAMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SPAMM_OK 0
#define SPAMM_E_INVAL (-1)    /* bad argument (size, leaf, tau, pointer)        */
#define SPAMM_E_NOMEM (-2)    /* device or host allocation failed               */
#define SPAMM_E_CUDA (-3)     /* a CUDA runtime call failed                     */
#define SPAMM_E_CAPACITY (-4) /* a caller-sized buffer is too small             */
#define SPAMM_E_TIMEOUT (-5)  /* a bounded device-side wait gave up             */
#define SPAMM_E_NOCONV (-6)   /* SP2 reached max_iter; the iterate is returned  */
#define SPAMM_E_NOTSUP (-7)   /* option combination not built                   */

/* ---- leaf-product precision ------------------------------------------- */
typedef enum {
    /* FP64 operands, FP64 fused multiply-add accumulation. */
    SPAMM_FP64 = 0,
    /* Exact-slice mixed precision on the tcgen05 tensor cores: each matrix
     * gets one power-of-two scale 2^sigma with max|x| < 2^sigma (SP2 fixes
     * sigma = 1 for its iterates, |x| < 2); every element is rounded to
     * 7 s bits below 2^sigma and cut into s = `slices` base-128 digits with
     * the element's sign, held exactly in BF16.  Elements below about
     * 2^(sigma - 7 s) keep no digits, so accuracy is absolute, relative to
     * the largest element.  Slice pairs (p, q) with p + q < s are multiplied
     * (exact products) and summed per diagonal d = p + q in FP32 in tensor
     * memory; the diagonals are combined exactly (integer arithmetic,
     * 128-bit when needed) and rounded once to FP64.  A diagonal's sum is
     * exact while the absolute values of its terms add up to less than 2^24
     * per output element (then the result is the exact product of the
     * sliced operands, rounded once); beyond that FP32 rounds it, by at most
     * about 2^-23 of the running sum per accumulation step (leading
     * diagonal: FP32-level relative accuracy).  The library does not prove
     * that condition; it counts the output elements whose final diagonal sum
     * reached 2^24 (spamm_stats_t.sums_rounded, sp2_report_t.sums_rounded),
     * a lower bound on the inexact ones.  Splitting after Ozaki, Ogita,
     * Oishi and Rump (2012). */
    SPAMM_OZAKI_BF16 = 1,
    /* One BF16 term per operand (x rounded to BF16), FP32 accumulation on the
     * tensor cores: the plain low-precision product of the precision study. */
    SPAMM_BF16 = 2,
    /* Split-BF16, 3 terms: hi = bf16(x), lo = bf16(x - hi);
     * hi*hi + hi*lo + lo*hi with FP32 accumulation, combined in FP64. */
    SPAMM_BF16X3 = 3,
    /* One TF32 term per operand (x rounded to nearest TF32, 10 fraction
     * bits), FP32 accumulation on the tensor cores (tcgen05 kind::tf32). */
    SPAMM_TF32 = 4,
    /* Split-TF32, 3 terms: hi = tf32(x), lo = tf32(x - hi);
     * hi*hi + hi*lo + lo*hi with FP32 accumulation, combined in FP64. */
    SPAMM_TF32X3 = 5
} spamm_prec_t;

/* ---- options ---------------------------------------------------------- */
#define SPAMM_F_TIMING 1 /* record per-stage device times into spamm_stats_t */
#define SPAMM_F_NOSYM 2  /* SP2: form every leaf of X^2 even when F is symmetric */
#define SPAMM_F_NOGRAPH 8 /* SP2: enqueue every iteration's launches directly
                             instead of replaying a captured CUDA graph */
#define SPAMM_F_HEAVIEST 4 /* tensor path: hand tiles out heaviest first
                              (longest-processing-time order) instead of
                              row-major (a schedule the autotuner tries) */

typedef struct {
    int32_t leaf;   /* leaf edge b: 16, 32 or 64; 0 selects 32            */
    int32_t prec;   /* spamm_prec_t                                       */
    int32_t slices; /* slices per operand for SPAMM_OZAKI_BF16 (0 = 7)    */
    int32_t flags;  /* SPAMM_F_* bits                                     */
} spamm_opts_t;

typedef struct {
    int64_t tasks;       /* surviving leaf triples (i, k, j)                 */
    int64_t candidates;  /* nb^3                                             */
    double flops_useful; /* 2 b^3 per surviving triple                       */
    double flops_issued; /* arithmetic issued, incl. slice pairs             */
    float ms_cull;       /* device time of the cull (+ slicing, mixed path)  */
    float ms_gemm;       /* device time of the leaf products                 */
    float ms_norm;       /* device time of the output norms                  */
    int32_t sums_rounded; /* SPAMM_OZAKI_BF16: output elements for which some
                             diagonal sum S_d ended at or beyond 2^24 in its
                             FP32 accumulator, i.e. was certainly rounded
                             (a lower bound on the elements whose result is
                             not exact; saturates at 2^31 - 1); else 0     */
} spamm_stats_t;

/* ---- matrices --------------------------------------------------------- */
typedef struct spamm_mat *spamm_mat_t;

/*
 * Build a matrix handle: leaf storage plus the norm quadtree.
 *   Eq. 1 (Sec. 2): the quadtree A^t = [[A^{t+1}_11, A^{t+1}_12],
 *   [A^{t+1}_21, A^{t+1}_22]]; Eq. 2: the leaf Frobenius norms; Eq. 3: a
 *   parent's norm from its four children.
 * a      : n x n FP64, row-major, leading dimension lda >= n (host or device).
 * drop   : sparse storage: leaf (i, k) is stored iff ||A_ik||_F > drop
 *          (squared norm > drop * drop in FP64); a leaf not stored is zero
 *          in every later use.  drop = 0 stores the nonzero leaves; drop < 0
 *          stores every leaf (dense).  Stored leaves are packed in row-major
 *          leaf order.  Handles with absent leaves serve as inputs only.
 * opts   : leaf size (others ignored here); NULL = defaults.
 * out    : receives the new handle (caller frees it with spamm_free).
 * Squared norms are stored.  Each is the exact sum of the exact squares
 * (resp. of the four children) rounded once to FP64, so its value does not
 * depend on the order of summation.  Device work is enqueued on `stream`;
 * a host `a` is copied before the call returns (in blocks of up to 2048
 * rows on a copy stream the library owns, overlapped with the packing into
 * leaves; two blocks of device staging; pinned host memory copies fastest).
 * Errors: E_INVAL (n < 1, lda < n, bad leaf, NULL a/out), E_NOMEM, E_CUDA.
 */
int spamm_tree_build(const double *a, int64_t n, int64_t lda, double drop,
                     const spamm_opts_t *opts, void *stream, spamm_mat_t *out);

/*
 * C = SpAMM(A, B, tau)  (Eq. 4, Algorithm 1 of Sec. 3.1).
 * Keeps the leaf triple (i, k, j) iff ||A_ik||^2 ||B_kj||^2 > tau^2, which
 * is the set the recursive walk of Algorithm 1 reaches (a parent's norm is
 * never below a child's), and sets C_ij = sum over kept k of A_ik B_kj with
 * k increasing.  C's norm quadtree is built too.
 * A, B   : handles of equal n and leaf size.
 * tau    : >= 0 and finite.
 * C      : *C == NULL creates a new handle; otherwise *C must have A's shape
 *          and is overwritten.  C may not alias A or B; a reused C must
 *          store every leaf (built by this library as an output, or by
 *          spamm_tree_build with drop < 0).
 * opts   : precision (spamm_prec_t), slices, flags.  The tensor-core modes
 *          take leaf 16, 32 or 64 with slices x leaf <= 256 (so leaf 64
 *          allows at most 4 exact slices).
 * stats  : optional; when given the call waits for the stream and fills it.
 * Errors: E_INVAL, E_NOTSUP, E_NOMEM, E_CUDA, E_CAPACITY (internal list
 *         overflow, never expected).
 */
int spamm_multiply(spamm_mat_t A, spamm_mat_t B, double tau, spamm_mat_t *C,
                   const spamm_opts_t *opts, spamm_stats_t *stats, void *stream);

/*
 * Many independent products C[m] = SpAMM(A[m], B[m], tau[m]), m < count, of
 * any sizes (each as in spamm_multiply, Eq. 4 and Algorithm 1), with the leaf
 * products of all of them in ONE persistent kernel launch (per group of at
 * most 64 products): tiles of every product are handed out from one device
 * counter, larger products first, each product's tiles in row-major order
 * (SPAMM_F_HEAVIEST: heaviest first).  The
 * paper has no batched form; this is the deployment batching of many small
 * SpAMMs onto one GPU.
 * A, B   : count handles each; A[m] and B[m] of equal n; one leaf size for
 *          all (the kernel is compiled per leaf size).
 * tau    : count thresholds (>= 0, finite).
 * C      : count handle slots; NULL entries are created (A[m]'s shape),
 *          others reused (must match A[m] and alias neither A[m] nor B[m];
 *          two slots may not share a handle).
 * opts   : one precision / slices / flags for the whole batch.
 * stats  : optional, ONE struct: totals over the batch (tasks, candidates,
 *          flops); the call then waits for the stream.  With SPAMM_F_TIMING,
 *          ms_cull covers slicing and culling of all products, ms_gemm the
 *          batched leaf-product launch(es), ms_norm the output norms.
 * Graph capture: without stats the call never waits for the stream.  Once a
 * batch has run with given handles, a repeat of it allocates nothing, so the
 * repeat may be captured into a CUDA graph on `stream`.
 * Errors: E_INVAL (count < 0, NULL arrays, shapes, aliasing, tau), E_NOTSUP,
 *         E_NOMEM, E_CUDA, E_CAPACITY.
 */
int spamm_multiply_batched(int32_t count, const spamm_mat_t *A, const spamm_mat_t *B,
                           const double *tau, spamm_mat_t *C, const spamm_opts_t *opts,
                           spamm_stats_t *stats, void *stream);

/* ---- autotuner --------------------------------------------------------- */
#define SPAMM_TUNE_MAX 6

typedef struct {
    int32_t leaf;                      /* chosen leaf edge                      */
    int32_t flags;                     /* chosen schedule (0 or SPAMM_F_HEAVIEST) */
    float ms;                          /* its device time for the batch          */
    int32_t tried;                     /* candidates timed                       */
    int32_t cand_leaf[SPAMM_TUNE_MAX];
    int32_t cand_flags[SPAMM_TUNE_MAX];
    float cand_ms[SPAMM_TUNE_MAX];     /* median over reps; -1 = mode not built  */
    int64_t cand_tasks[SPAMM_TUNE_MAX]; /* surviving triples at that leaf       */
} spamm_tune_t;

/*
 * Pick the leaf size (16, 32, 64) and the tile schedule (heaviest first or
 * row-major) for a batch of products C[m] = SpAMM(A[m], B[m], tau[m]) by
 * timing spamm_multiply_batched on the caller's own data.  The paper's task
 * granularity is fixed (Sec. 3); this is the GPU's counterpart of choosing
 * it.  For each leaf size the precision mode supports, handles are built
 * from the dense inputs, the batch is run once to warm up and then `reps`
 * times per schedule (CUDA events on `stream`); the smallest median wins.
 * a, b   : count dense n[m] x n[m] FP64 row-major matrices (host or device),
 *          leading dimension n[m].
 * tau    : count thresholds.  opts: precision and slices (leaf ignored).
 * reps   : timed runs per candidate (>= 1).
 * out    : receives the choice and every candidate's time.
 * Blocking.  Allocates and frees its trial handles.
 * Errors: E_INVAL, E_NOTSUP (no leaf size supports the mode), E_NOMEM,
 *         E_CUDA.
 */
int spamm_autotune_batched(int32_t count, const double *const *a, const double *const *b,
                           const int64_t *n, const double *tau, const spamm_opts_t *opts,
                           int32_t reps, spamm_tune_t *out, void *stream);

/*
 * Write the matrix to dense row-major storage (host or device), n x n with
 * leading dimension ld >= n.  Blocking when dst is host memory (then the
 * rows are unpacked and copied out in blocks, the copies on a copy stream
 * the library owns, overlapped with the unpacking of the next block).
 */
int spamm_to_dense(spamm_mat_t M, double *dst, int64_t ld, void *stream);

/*
 * Copy the squared norms of quadtree tier t (0 = root ... depth = leaves)
 * to dst (host or device): a 2^t x 2^t row-major grid.  Blocking when dst
 * is host memory.
 */
int spamm_norms(spamm_mat_t M, int32_t tier, double *dst, void *stream);

/* Shape of a handle: n, leaf edge b, leaf grid nb, quadtree depth d, and the
 * number of stored leaves (nb * nb for dense handles).  Any pointer may be
 * NULL. */
int spamm_info(spamm_mat_t M, int64_t *n, int32_t *leaf, int64_t *nb,
               int32_t *depth, int64_t *stored);

/*
 * The culled task list of SpAMM(A, B, tau), grouped by output leaf (Eq. 4):
 * for output leaf g = i * nb + j, the surviving k are k_host[off_host[g] ..
 * off_host[g + 1]) in increasing order.  off_host has nb*nb + 1 entries;
 * k_host has room for cap entries.  *ntasks receives the total; when it is
 * larger than cap the call returns E_CAPACITY and k_host is untouched.
 * Blocking (waits for the stream).  Host buffers.
 */
int spamm_task_list(spamm_mat_t A, spamm_mat_t B, double tau, int64_t *off_host,
                    uint32_t *k_host, int64_t cap, int64_t *ntasks, void *stream);

/*
 * The culled task list of SpAMM(A, B, tau), like spamm_task_list, for callers
 * that cannot allocate device memory (codes that give all of HBM to their own
 * memory pool, and latency-critical loops that cannot afford the implicit
 * synchronisation of cudaMalloc / cudaFree).  The paper has no counterpart:
 * this is a deployment variant of the culling pass.  It allocates nothing;
 * its only scratch is a fixed file-scope device array of
 * 1024 x 1024 int32 counts (4 MiB, held by every GPU that loads the library
 * until the process exits).
 * n2A    : device, leaf-tier squared norms of A, nb rows, row stride lda >= nb
 *          (e.g. spamm_norms(A, depth, ...) with lda = 2^depth).
 * n2B    : device, the same for B (row-major, stride ldb >= nb).
 * nb     : leaf grid, 1 <= nb <= 1024 (larger: SPAMM_E_CAPACITY).
 * off    : device, nb*nb + 1 int64; off[g] .. off[g+1] are the surviving k of
 *          output leaf g = i * nb + j; off[nb*nb] is the total.
 * klist  : device, room for cap uint32 (may be NULL when cap = 0).  When the
 *          total exceeds cap, groups that do not fit are not written: compare
 *          off[nb*nb] with cap after the stream reaches this work.
 * Asynchronous on `stream`.  Every call looks up the scratch array's device
 * address in the current context; the first call on a device may load the
 * library's device code, so make it before any stream capture.  All calls
 * share the scratch: calls whose GPU work overlaps (unordered streams) race
 * on it.
 */
int spamm_cull_noalloc(const double *n2A, int64_t lda, const double *n2B, int64_t ldb,
                       int64_t nb, double tau, int64_t *off, uint32_t *klist, int64_t cap,
                       void *stream);

/* Release a handle (its device memory is freed in stream order). */
void spamm_free(spamm_mat_t M);

/*
 * Free the scratch a handle keeps for later products: its tensor-core slices
 * (the largest buffers of the mixed path: e s bytes per stored element and
 * layout for s slices of e-byte elements; one layout when the handle was only
 * used in symmetric products, such as the SP2 iterate, two otherwise) and the
 * task lists of the product it was the output of.  The matrix, its norms and its shape are
 * untouched; the next product that needs the scratch allocates it again.
 * Stream-ordered on `stream`.  No-op for NULL.
 */
void spamm_release_scratch(spamm_mat_t M, void *stream);

/*
 * Return the device memory the library keeps cached to the driver.  Device
 * memory comes from a pool owned by the library (one per device, created on
 * first use) that keeps freed memory for the library's later allocations:
 * repeated products and SP2 solves then reuse it instead of mapping it anew.
 * This call waits for the current device (cudaDeviceSynchronize), then
 * releases every byte of that pool that no live handle uses; the next
 * allocation maps memory again.  Blocking.  Errors: E_CUDA.  The paper has
 * no counterpart.
 */
int spamm_trim(void);

/*
 * Self-test of the device watchdog that bounds every wait inside the
 * library's kernels: one GPU thread waits, through the same bounded wait, on
 * a barrier that nothing completes; after about `ms` milliseconds (1..10000)
 * the wait gives up and the call returns SPAMM_E_TIMEOUT (the expected
 * result), with the device context still usable.  Blocking.  No fault, no
 * trap: the kernel simply returns.  The paper has no counterpart.
 */
int spamm_watchdog_selftest(int32_t ms, void *stream);

/* Static text for a status code. */
const char *spamm_strerror(int status);

/* Detail of the last failure on the calling thread ("" if none). */
const char *spamm_last_error(void);

/* ---- SP2 spectral projection ------------------------------------------ */
#define SP2_RULE_TRACE_DISTANCE 0 /* X^2 iff |tr X^2 - Ne| < |2trX - trX^2 - Ne| */
#define SP2_RULE_TRACE_ABOVE 1    /* X^2 iff tr X > Ne                          */

#define SP2_STOP_CONVERGED 0 /* |tr X - Ne| < trace_tol and e < idem_tol       */
#define SP2_STOP_STAGNATED 1 /* e < 1e-3 and e > 0.5 e(two iterations before)  */
#define SP2_STOP_FIXED 2     /* fixed_iters iterations done                    */
#define SP2_STOP_MAXITER 3   /* max_iter reached without a stop                */

typedef struct {
    int32_t max_iter;    /* 0 selects 100                                    */
    int32_t rule;        /* SP2_RULE_*                                       */
    double trace_tol;    /* 0 selects 1e-10                                  */
    double idem_tol;     /* 0 selects 1e-8                                   */
    int32_t fixed_iters; /* > 0: run exactly this many iterations            */
    int32_t leaf;        /* 0 selects 32                                     */
    int32_t prec;        /* spamm_prec_t of the X^2 products                 */
    int32_t slices;      /* for SPAMM_OZAKI_BF16 (0 = 7)                     */
    int32_t flags;       /* SPAMM_F_TIMING: per-stage device times;
                            SPAMM_F_NOSYM, SPAMM_F_HEAVIEST as for products */
    int32_t reserved;
} sp2_opts_t;

/* History columns, one row of SP2_H_COLS doubles per iteration. */
#define SP2_H_TR 0     /* tr X                                  */
#define SP2_H_TR2 1    /* tr X^2                                */
#define SP2_H_IDEM 2   /* e = ||X^2 - X||_F                     */
#define SP2_H_BRANCH 3 /* 1: X <- X^2, 0: X <- 2X - X^2         */
#define SP2_H_TASKS 4  /* surviving leaf triples of the product */
#define SP2_H_TRNEW 5  /* tr of the updated X                   */
#define SP2_H_FILL 6   /* fraction of the updated X's leaves that are nonzero */
#define SP2_H_COLS 7

typedef struct {
    int32_t iters;        /* iterations run                               */
    int32_t stop_reason;  /* SP2_STOP_*                                    */
    double trace_err;     /* |tr P - Ne|                                   */
    double idem_err;      /* e of the last iteration                       */
    double emin, emax;    /* Gershgorin bounds of F                        */
    int64_t tasks_total;  /* surviving leaf triples over all iterations    */
    double flops_useful;  /* 2 b^3 tasks_total                             */
    double flops_tensor;  /* arithmetic of the leaf products formed:
                             tensor path: 2 b^3 per slice pair of a
                             surviving product that is not identically
                             zero (leading zero slices skipped); FP64:
                             2 b^3 per leaf product formed; both exclude
                             the mirrored half of a symmetric product */
    double ms_total;      /* device time of the whole solve                */
    double ms_cull;       /* SPAMM_F_TIMING: summed time of cull (+ slicing) */
    double ms_gemm;       /*   ... of the leaf products                     */
    double ms_update;     /*   ... of the SP2 decide + update passes        */
    int64_t launches;     /* kernels the solve launched                     */
    int32_t symmetric;    /* 1: upper block triangle of X^2 formed + mirrored */
    int32_t graphed;      /* iterations run by replaying a captured CUDA graph */
    double *history;      /* in: optional host buffer of history_cap rows  */
    int32_t history_cap;  /* in: rows available in history                 */
    int32_t sums_rounded; /* spamm_stats_t.sums_rounded summed over the
                             solve's products (saturates at 2^31 - 1)      */
} sp2_report_t;

/*
 * P = SP2(F, Ne, tau): second-order spectral projection (Niklasson 2002,
 * the solver of Sec. 4) with every X^2 formed by SpAMM at threshold tau.
 * X0 = (emax I - F) / (emax - emin) from Gershgorin bounds; each iteration
 * forms X^2 = SpAMM(X, X, tau), picks X^2 or 2X - X^2 by `rule` on the
 * device, and updates X.  Stops as in SP2_STOP_*.
 * With SPAMM_OZAKI_BF16 and an exactly symmetric F, every iterate is exactly
 * symmetric (the slice arithmetic is exact), so only the upper block triangle
 * of X^2 is formed and mirrored; the result is bit-identical to forming all
 * leaves (SPAMM_F_NOSYM in flags forces the full product).
 * F      : symmetric handle (checked on the leaf norms: mirror leaves whose
 *          norms differ beyond 1e-12 relative give E_INVAL); Ne in (0, n)
 *          is the trace of the projector.
 * P      : *P == NULL creates a new handle; otherwise reused (F's shape,
 *          every leaf stored).  F may have absent leaves.
 * report : optional; filled when given.
 * Iterations are enqueued four at a time and the state is read once per
 * four (blocking).  After the first four, the launches of four iterations
 * are captured once into a CUDA graph (on an internal stream) and replayed
 * for the rest of the solve, unless SPAMM_F_NOGRAPH is set or a product
 * could need to wait for a task count (FP64 lists above 512 MB); the results
 * are the same either way.
 * Errors: E_INVAL, E_NOTSUP, E_NOMEM, E_CUDA; E_NOCONV when max_iter is
 *         reached (P holds the last iterate).
 */
int sp2_solve(spamm_mat_t F, double Ne, double tau, const sp2_opts_t *opts,
              spamm_mat_t *P, sp2_report_t *report, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SPAMM_H */
