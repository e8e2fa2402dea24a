/*
 * rsf.h -- C ABI of the GB300 recursive skeletonization factorization (RSF)
 * library for Gaussian-process log-likelihoods and scores on 2-D points.
 *
 * Method: Minden, Damle, Ho, Ying, "Fast spatial Gaussian process maximum
 * likelihood estimation via skeletonization factorizations".
 *   - model and objective: Sec. 1, Eqs. (normaldist), (loglikelihood),
 *     (gradient);
 *   - factorization F ~ Sigma: Sec. 2, Def. (ID), Sec. 2.1 block equations,
 *     Eq. (rskelf), Sec. 2.3.1 Eq. (proxyid) (modified proxy trick);
 *   - apply / solve / square root / log-determinant: Sec. 2.3.2, Table 1;
 *   - trace by weak peeling: Sec. 3, Eq. (lowrankapprox);
 *   - log-likelihood and score: Sec. 4, Algorithm 1.
 *
 * Conventions shared by every entry point:
 *   - points: DEVICE pointer, n x 2 row-major fp64 (x0 y0 x1 y1 ...),
 *     caller-owned, read only during the call;
 *   - vectors (z, B, alpha): DEVICE pointers in the caller's original point
 *     order; B is column-major n x nrhs with leading dimension ldb >= n;
 *   - theta = {l, s2, nug}: host array of 3 doubles; the covariance is
 *     K(x_i, x_j) = s2 * k(|x_i - x_j| / l) + nug * delta_ij (nugget on equal
 *     indices);
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream);
 *     all work of a handle runs on the stream it was built with;
 *   - every call returns an rsf_status and never aborts, traps or prints
 *     (unless the environment variable RSF_VERBOSE is set: then a few
 *     diagnostics go to stderr, for debugging).
 *     On error the outputs are left unchanged, handles stay valid (or NULL),
 *     and rsf_last_error() returns a message (thread-local, valid until the
 *     next call on that thread).  Device-side failures (non-positive pivot,
 *     NaN/Inf) are recorded in a device status word and reported by the
 *     call that synchronises next.
 *   - memory: handles own all device memory they allocate (stream-ordered
 *     cudaMallocAsync on the handle's stream, or the hook installed with
 *     rsf_set_allocator) and release it in rsf_destroy / rsf_tree_destroy;
 *   - every device-side wait is bounded (RSF_ETIMEOUT, see
 *     rsf_selftest_wait_limit).
 */
#ifndef RSF_H
#define RSF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RSF_OK = 0,
  RSF_EINVAL = 1,    /* bad argument or unsupported combination */
  RSF_ENOMEM = 2,    /* device allocation failed */
  RSF_ENOTPD = 3,    /* Cholesky of a diagonal block met a non-positive pivot */
  RSF_ENUMERIC = 4,  /* NaN / Inf produced */
  RSF_ETIMEOUT = 5,  /* a bounded device wait gave up */
  RSF_ECUDA = 6      /* a CUDA runtime call failed */
} rsf_status;

/* Kernel families (Sec. 1 Eqs. (matern), (rationalquadratic); Sec. 5.5
 * Eq. (diffkernels)). */
typedef enum {
  RSF_MATERN12 = 0,  /* s2 exp(-r/l) */
  RSF_MATERN32 = 1,  /* s2 (1 + a) exp(-a), a = sqrt(3) r / l */
  RSF_MATERN52 = 2,  /* s2 (1 + a + a^2/3) exp(-a), a = sqrt(5) r / l */
  RSF_MATERN1 = 3,   /* s2 x K_1(x), x = sqrt(2) r / l (K_0, K_1: ascending
                        series for x < 1, trapezoid rule on the integral
                        representation otherwise) */
  RSF_RQ = 4         /* s2 (1 + r^2 / (2 alpha l^2))^-alpha */
} rsf_family;

/* Matrix selector: Sigma or one of its theta-derivatives (Sec. 1, below
 * Eq. (gradient)).  RSF_D_L2 (the second length scale) exists for
 * anisotropic kernels only; RSF_D_L is then the derivative in l1. */
typedef enum { RSF_SIGMA = 0, RSF_D_L = 1, RSF_D_S2 = 2, RSF_D_NUG = 3, RSF_D_L2 = 4 } rsf_which;

/* Operations of rsf_solve (Sec. 2.3.2): F^-1, F, F^1/2, (F^1/2)^T, F^-1/2,
 * (F^-1/2)^T.  Only RSF_OP_APPLY is defined for derivative factorizations. */
typedef enum {
  RSF_OP_INV = 0, RSF_OP_APPLY = 1, RSF_OP_SQRT = 2, RSF_OP_SQRT_T = 3,
  RSF_OP_INV_SQRT = 4, RSF_OP_INV_SQRT_T = 5
} rsf_op;

/* Kernel description.  theta (host) is (l, s2, nug): length scale, variance,
 * nugget.  With anisotropic != 0 it is (l1, s2, nug, l2) and the family is
 * evaluated at unit length scale on the scaled distance of Sec. 5.1,
 * ||x - y||_theta^2 = (x1 - y1)^2 / l1^2 + (x2 - y2)^2 / l2^2 (Eqs. (specrq)
 * and (specmatern) are RSF_RQ with alpha = 1/2 and RSF_MATERN32, s2 = 1).
 * Scores then have p = 4 components (l1, s2, nug, l2), otherwise p = 3
 * (l, s2, nug).  The quadtree and proxy annulus stay in the points' own
 * coordinates. */
typedef struct {
  int family;       /* rsf_family */
  double alpha;     /* RQ shape parameter (ignored otherwise) */
  int anisotropic;  /* 0: isotropic theta (3 entries); 1: (l1, s2, nug, l2) */
} rsf_kernel;

/* Tuning knobs.  n_occ and n_prox default to the paper's 64 and 256 (Sec. 5);
 * the near-field radius and proxy annulus (in units of the box side) are
 * this library's reading of Sec. 2.3.1, which gives no radii. */
typedef struct {
  int n_occ;        /* max points per leaf box (64) */
  int n_prox;       /* proxy points per box (256) */
  int n_rings;      /* rings of the proxy annulus (8); n_prox % n_rings == 0 */
  double r_near;    /* near field: active DOFs within r_near * side (1.0) */
  double r_in;      /* proxy annulus inner radius / side (1.0) */
  double r_out;     /* proxy annulus outer radius / side (2.0) */
  int oversample;   /* peeling oversampling c (10), Sec. 3.1 */
  int q0;           /* peeling: minimum initial sample count at level 1 (64) */
  uint64_t seed;    /* Philox4x32-10 key of the peeling test matrices (0) */
  int precision;    /* RSF_PREC_FP64 (0): every step in fp64.  RSF_PREC_MIXED
                       (1, default): the IDs, Cholesky/QR factors and
                       log-determinant stay fp64; the multi-RHS solves and
                       the peeling products keep their operands as
                       double-float (fp32-pair, ~48-bit) values and multiply
                       them on the tensor cores, split exactly into seven
                       bf16 slices per operand with exact fp32 accumulation
                       (fp64-class products).  RSF_PREC_MIXED_DF64 (2): the
                       same storage, products in double-float arithmetic on
                       the CUDA cores */
  int trace_form;   /* symmetric operator peeled for Tr(F^-1 F_k) (Sec. 3,
                       which allows any symmetrized form with the same
                       trace).  RSF_TRACE_SYM (0, default): the paper's
                       G = (F^-1 F_k + F_k F^-1) / 2 of Eq. (Gbb), and F^-1
                       itself for Tr(F^-1).  RSF_TRACE_SQRT (1):
                       G = F^-1/2 F_k F^-T/2 and, for Tr(F^-1),
                       F^-1/2 F^-T/2, with F = F^1/2 (F^1/2)^T of Sec. 2.3.2:
                       half the solve passes per test column.
                       RSF_TRACE_HUTCH (2): no peeling -- Hutchinson's
                       estimator (Sec. 3, Eq. (hutch)), the mean of
                       u^T F^-1 u and (F^-1 u)^T F_k u over `probes`
                       Rademacher vectors (Philox stream 1, key seed): a
                       cheap trace with statistical error
                       ~ sqrt(2 / probes) ||G||_F; tol_peel is ignored */
  int refine;       /* sweeps of iterative refinement of alpha = Sigma^-1 z
                       in gp_loglik (Algorithm 1, first line): alpha +=
                       F^-1 (z - Sigma alpha), the residual taken against
                       the exact kernel matrix by an on-the-fly O(n^2)
                       matvec (df64 on the fp32 pipes for the Matern
                       1/2, 3/2, 5/2 kernels and the rational quadratic
                       with integer alpha <= 8, fp64 otherwise), so that
                       z^T alpha does not carry the factorization's
                       eps_fact error.  -1 (default): 1 in the mixed forms
                       where the matvec runs in df64, else 0 */
  int probes;       /* Hutchinson probes for RSF_TRACE_HUTCH (64) */
} rsf_opts;

enum { RSF_TRACE_SYM = 0, RSF_TRACE_SQRT = 1, RSF_TRACE_HUTCH = 2 };

enum { RSF_PREC_FP64 = 0, RSF_PREC_MIXED = 1, RSF_PREC_MIXED_DF64 = 2 };

typedef struct rsf_tree_s* rsf_tree;
typedef struct rsf_handle_s* rsf_handle;

/* Summary of a factorization, for reporting. */
typedef struct {
  int64_t n;
  int levels;            /* L + 1 (levels 0..L) */
  int64_t boxes;         /* skeletonized boxes plus the root */
  int root_size;         /* DOFs left in the root block */
  int max_rank;          /* largest skeleton |S| */
  int max_active;        /* largest |I| */
  int64_t factor_entries;/* entries of T, E and the diagonal blocks */
  double flops;          /* algorithmic fp64 flops of the factorization */
  double kernel_evals;   /* kernel evaluations during the factorization */
  int nsets;             /* independent point sets (1 unless built batched) */
  int solve_df64;        /* the form of the solves: 0 fp64; df64 (fp32-pair)
                            factors with tensor-core (1) or CUDA-core (2)
                            products, as rsf_opts.precision */
  double probe_rel_diff; /* derivative factorization in mixed precision: the
                            relative difference of one df64 and one fp64
                            apply; df64 is kept when it is <= 10 tol.  -1 when
                            no probe ran */
} rsf_info_t;

/* Fills *o with the defaults listed above. */
void rsf_opts_default(rsf_opts* o);

/* Message of the last failing call on this thread ("" if none). */
const char* rsf_last_error(void);

/* Failure detection self-test (no counterpart in the paper).  Every device
 * wait in this library is bounded: the grid barrier of the persistent
 * pivoted-QR kernel gives up after a few seconds, records RSF_ETIMEOUT in the
 * handle's status word and leaves the kernel, so a wait that cannot finish
 * surfaces as an error instead of a hang.  This call runs that barrier with
 * one participant more than it launches (a wait nothing can end) and returns
 * RSF_OK if the wait gave up and reported RSF_ETIMEOUT as designed, RSF_ECUDA
 * otherwise.  It takes a few seconds and leaves the context usable. */
rsf_status rsf_selftest_wait_limit(void* stream);

/* GEMM engine self-check (no counterpart in the paper).  Computes
 * C <- alpha op(A) op(B) + beta C for one column-major problem (device fp64
 * arrays A, B, C; op(X) = X^T when ta / tb is nonzero; op(A) is m x k, op(B)
 * k x n) with one of the batched-GEMM engines that the solves and the
 * peeling use: 0 fp64 on the CUDA cores, 1 df64 operands multiplied on the
 * tensor cores (bf16 slices cut once per operand into work buffers, exact
 * fp32 accumulation over superblocks of 384 terms; batches with fewer than
 * 64 rows fall back to engine 2), 2 df64 arithmetic on the CUDA cores, 3 the
 * tensor-core engine that slices inside the GEMM kernel (K-blocks of 64
 * terms, no work buffers; the allocation-free solve uses it).
 * Operands are copied and, for engines 1 to 3, rounded to df64 pairs first,
 * so the result carries that rounding (~2^-48 relative per operand).
 * Synchronises the stream. */
rsf_status rsf_selftest_gemm(int engine, int m, int n, int k, int ta, int tb, double alpha,
                             const double* A, int lda, const double* B, int ldb, double beta,
                             double* C, int ldc, void* stream);

/* Device-memory hook.  The paper has no counterpart: this lets a host
 * framework back every device allocation the library makes (factor storage,
 * solve and peeling work buffers) with its own allocator, e.g. PyTorch's
 * caching allocator.  alloc(bytes, stream, ctx) returns a device pointer to
 * at least `bytes` bytes that may be used in stream order on `stream`, or
 * NULL on failure (the library call then fails with RSF_ENOMEM); free(ptr,
 * bytes, stream, ctx) returns it, in stream order, on the stream it was
 * allocated for.  Passing NULL for both restores the default
 * (cudaMallocAsync / cudaFreeAsync); one NULL and one non-NULL is
 * RSF_EINVAL.  Memory is always returned through the hook that allocated it,
 * even if the hook changes in between.  The setting is process-wide: change
 * it only while no other thread is inside the library. */
typedef void* (*rsf_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*rsf_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
rsf_status rsf_set_allocator(rsf_alloc_fn alloc_fn, rsf_free_fn free_fn, void* ctx);

/* Quadtree of Sec. 2.1 / Remark (tree) over `points` (device, n x 2).
 * Split while a box holds more than opts->n_occ points; children in Morton
 * order.  The tree keeps its own copy of the points (tree order) and may be
 * reused by rsf_build_on_tree for any kernel and theta.  opts may be NULL. */
rsf_status rsf_tree_build(const double* points, int64_t n, const rsf_opts* opts,
                          void* stream, rsf_tree* out);
void rsf_tree_destroy(rsf_tree t);

/* The tree's point order and box table (Sec. 2.1): *n_out points and
 * *nbox_out boxes (host); when perm and boxes are not NULL also perm (host,
 * n ints: tree position -> input index) and boxes (host, nbox x 6 ints,
 * row-major: level, first tree position, point count, parent box (-1 for a
 * root), child slot (0 SW, 1 SE, 2 NW, 3 NE), point set).  Boxes are numbered
 * breadth first, the roots of all sets first.  Synchronises. */
rsf_status rsf_tree_export(rsf_tree t, int64_t* n_out, int* nbox_out, int* perm, int* boxes);

/* RSF of Sigma (which = RSF_SIGMA, Cholesky of the diagonal blocks) or of a
 * derivative matrix dSigma/dtheta_k (which = RSF_D_L / RSF_D_S2; diagonal
 * blocks kept for application, Remark (indefinite)).  tol is the relative ID
 * tolerance (Def. ID).  The handle owns all factor memory. */
rsf_status rsf_build(const double* points, int64_t n, const rsf_kernel* kernel,
                     const double* theta, int which, double tol,
                     const rsf_opts* opts, void* stream, rsf_handle* out);
rsf_status rsf_build_on_tree(rsf_tree tree, const rsf_kernel* kernel,
                             const double* theta, int which, double tol,
                             const rsf_opts* opts, rsf_handle* out);

/* Batched datasets.  The paper treats one point set; a batch of nsets
 * independent sets has the block-diagonal covariance diag(Sigma_1, ...),
 * factored here as one forest: every set gets its own quadtree (own root
 * square, Sec. 2.1) and the boxes of all sets at one level are skeletonized
 * by the same level-batched launches (boxes of different sets never
 * interact).  points (device, offsets[nsets] x 2 row-major) holds set i in
 * rows offsets[i] .. offsets[i+1]-1; offsets (host, nsets + 1 entries,
 * offsets[0] = 0, strictly increasing) is read during the call only.  The
 * handle then acts on the concatenated index space: rsf_solve applies the
 * block-diagonal operator, rsf_logdet returns the sum over the sets,
 * rsf_logdet_sets the per-set values.  Same theta for every set.
 * RSF_EINVAL for nsets outside 1 .. 16384 or an empty set. */
rsf_status rsf_build_batched(int nsets, const int64_t* offsets, const double* points,
                             const rsf_kernel* kernel, const double* theta, int which,
                             double tol, const rsf_opts* opts, void* stream,
                             rsf_handle* out);

/* log|F| = 2 log|C| (Sec. 2.3.2) to *out (host).  Synchronises the stream.
 * For a batched handle the sum over its sets.  RSF_EINVAL for derivative
 * factorizations. */
rsf_status rsf_logdet(rsf_handle h, double* out);

/* log|F_i| of every point set i of the handle (rsf_get_info's nsets values,
 * host array out).  Synchronises the stream. */
rsf_status rsf_logdet_sets(rsf_handle h, double* out);

/* In place B <- op(F) B for B (device, column-major n x nrhs, ld ldb >= n,
 * original point order).  Stream-ordered (does not synchronise). */
rsf_status rsf_solve(rsf_handle h, double* B, int64_t ldb, int nrhs, int op);

/* rsf_solve without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory at
 * solve time -- code running inside another framework's memory budget (its
 * caching allocator has already reserved the device memory, so cudaMalloc
 * would fail or fragment that pool) and latency-critical loops that must not
 * pay for an allocation's implicit synchronisation.
 *
 * Same arguments, result and errors as rsf_solve, but every work buffer is
 * carved from one file-scope device array of RSF_NOALLOC_SCRATCH_DOUBLES
 * doubles (32 MiB), which every GPU that loads the library holds until the
 * process exits.  A call needs nrhs * (2 n + the active DOFs of all levels +
 * those of the largest level) doubles; larger requests return RSF_EINVAL
 * without touching B.  The device the handle was built on must be the
 * current device (else RSF_EINVAL): the scratch address is per device.  The
 * first call on a device looks up the array's device address; make that
 * first call before any stream capture.  All calls share the one array and nothing in it needs to
 * start at zero, but calls whose work overlaps on the GPU (different streams,
 * or concurrent host threads) race on it: serialise them. */
#define RSF_NOALLOC_SCRATCH_DOUBLES (1 << 22)
rsf_status rsf_solve_noalloc(rsf_handle h, double* B, int64_t ldb, int nrhs, int op);

/* Trace by weak peeling (Sec. 3) to *trace (host): Tr(F^-1) when Fk is NULL,
 * else Tr((F^-1 Fk + Fk F^-1)/2) (Algorithm 1).  tol_peel is the relative
 * cut-off of the sibling-block ranks.  Synchronises. */
rsf_status rsf_peel_trace(rsf_handle F, rsf_handle Fk, double tol_peel,
                          const rsf_opts* opts, double* trace);

/* Log-likelihood from a factorization of Sigma (Algorithm 1, first part):
 * alpha = F^-1 z, quad = z^T alpha, loglik = -quad/2 - log|F|/2 - n/2 log 2pi.
 * z (device, n), alpha_out (device, n, or NULL), loglik/quad host (quad may be
 * NULL).  Synchronises. */
rsf_status gp_loglik(rsf_handle F, const double* z, double* alpha_out,
                     double* loglik, double* quad);

/* Score (Algorithm 1, loop over theta) given F ~ Sigma and alpha = F^-1 z:
 * builds F_l ~ dSigma/dl on F's tree, peels Tr(F^-1) and
 * Tr((F^-1 F_l + F_l F^-1)/2), and uses Sigma = s2 Sigma_s2 + nug I for the
 * variance component.  score (host, p) = (g_l, g_s2, g_nug); terms (host, 2p,
 * or NULL) = (quad_l, quad_s2, quad_nug, trace_l, trace_s2, trace_nug).  For
 * an anisotropic kernel (p = 4) F_l2 ~ dSigma/dl2 is built and peeled as
 * well: score = (g_l1, g_s2, g_nug, g_l2), terms = (quads of l1, s2, nug, l2;
 * traces of l1, s2, nug, l2). */
rsf_status gp_score(rsf_handle F, const double* alpha, double tol_fact,
                    double tol_peel, const rsf_opts* opts, double* score,
                    double* terms);

/* Algorithm 1 end to end: tree, F, loglik and (when score != NULL) the
 * score.  points, z device; loglik, score (p), terms (2p, or NULL) host,
 * p as for gp_score. */
rsf_status gp_loglik_and_score(const double* points, const double* z, int64_t n,
                               const rsf_kernel* kernel, const double* theta,
                               double tol_fact, double tol_peel,
                               const rsf_opts* opts, void* stream,
                               double* loglik, double* score, double* terms);

/* Algorithm 1 for nsets independent datasets in one forest (see
 * rsf_build_batched for points and offsets; z device, offsets[nsets]
 * entries in the same order as the points).  Per set i: loglik[i] and, when
 * score != NULL, score[p i .. p i + p - 1] and terms[2p i .. 2p i + 2p - 1] (host), each
 * exactly what gp_loglik_and_score returns for that set alone up to the
 * peeling's test matrices (shared by all sets). */
rsf_status gp_loglik_and_score_batched(int nsets, const int64_t* offsets,
                                       const double* points, const double* z,
                                       const rsf_kernel* kernel, const double* theta,
                                       double tol_fact, double tol_peel,
                                       const rsf_opts* opts, void* stream,
                                       double* loglik, double* score, double* terms);

/* Profile log-likelihood (Sec. 5.5, Eq. (prof)) for z ~ N(mu 1, s Sigma(theta))
 * with the mean level mu and the variance level s profiled out, as printed
 * with A = Sigma + 1 1^T:
 *   lt   = -1/2 log|Sigma| - n/2 log(z^T A^-1 z) + n/2 (log n - 1 - log 2 pi)
 *   gt_k = -1/2 Tr(Sigma^-1 Sigma_k) + n/2 gamma^T Sigma_k gamma / z^T gamma,
 *          gamma = A^-1 z,
 * (the printed constant "log n - 1 - 2 pi" read as log n - 1 - log 2 pi, the
 * value at the maximizing s = z^T A^-1 z / n).  gamma comes from alpha =
 * F^-1 z and beta = F^-1 1 (one two-column solve, refined as in gp_loglik)
 * by Sherman-Morrison; the traces are peeled exactly as in gp_score.  The
 * paper's model has unit variance in Sigma (theta = (l, 1, nug)); any s2 is
 * accepted and gt_s2 is the derivative in it.  points, z device; loglik (1),
 * score (p, as for gp_score; or NULL for lt alone) and terms (2p + 4, or
 * NULL) host: terms = (gamma^T Sigma_k gamma for the p parameters;
 * Tr(Sigma^-1 Sigma_k) for the same (zero when score is NULL); z^T gamma;
 * log|F|; 1^T Sigma^-1 z; 1^T Sigma^-1 1).  Synchronises. */
rsf_status gp_profile_loglik_and_score(const double* points, const double* z, int64_t n,
                                       const rsf_kernel* kernel, const double* theta,
                                       double tol_fact, double tol_peel,
                                       const rsf_opts* opts, void* stream,
                                       double* loglik, double* score, double* terms);

/* gp_profile_loglik_and_score for nsets independent datasets in one forest
 * (points, offsets and z as in gp_loglik_and_score_batched): per set i,
 * loglik[i], score[p i ..] and terms[(2p + 4) i ..]; each set has its own mean and
 * variance level. */
rsf_status gp_profile_loglik_and_score_batched(int nsets, const int64_t* offsets,
                                               const double* points, const double* z,
                                               const rsf_kernel* kernel, const double* theta,
                                               double tol_fact, double tol_peel,
                                               const rsf_opts* opts, void* stream,
                                               double* loglik, double* score, double* terms);

/* How gp_conditional applies the cross covariance Sigma_12. */
typedef enum {
  RSF_COND_RSF = 0,    /* the remark's route: F of the joint matrix of
                          [new points; points], Sigma_12 v = (F [0; v])(0:m) */
  RSF_COND_DIRECT = 1  /* Sigma_12 v summed on the fly from the kernel (fp64,
                          O(m n) work, exact Sigma_12; mean only) */
} rsf_cond_method;

/* Conditional distribution of z' at m new points given z at n points
 * (Remark conditional, Sec. 4): z' | z ~ N(Sigma_12 Sigma_22^-1 z,
 * Sigma_11 - Sigma_12 Sigma_22^-1 Sigma_12^T) under the same kernel, the
 * nugget on equal indices only (Sigma_12 holds none).  Sigma_22^-1 z comes
 * from F_22 (refined as in gp_loglik).  Samples follow the remark:
 * y = F^1/2 w with F the joint factorization, sample = mean + y(0:m) -
 * Sigma_12 F_22^-1 y(m:m+n), so their covariance is the conditional one up to
 * the factorizations' tolerance.  points (n x 2), z (n), new_points (m x 2),
 * mean (m) device; w (device, (m + n) x q column-major, leading dimension
 * m + n, joint order: new points first) and samples (device, m x q,
 * leading dimension m) only when q > 0, which needs RSF_COND_RSF.  The
 * caller draws w (e.g. N(0, I)).  tol is the factorizations' ID tolerance.
 * RSF_EINVAL for n or m < 1, q < 0, an unknown method, or samples asked of
 * RSF_COND_DIRECT.  Synchronises. */
rsf_status gp_conditional(const double* points, int64_t n, const double* z,
                          const double* new_points, int64_t m,
                          const rsf_kernel* kernel, const double* theta, double tol,
                          const rsf_opts* opts, void* stream, int method,
                          double* mean, const double* w, int q, double* samples);

/* Factorization summary (host struct). */
rsf_status rsf_get_info(rsf_handle h, rsf_info_t* info);

/* Number of this library's kernel launches since the counter was last reset
 * (host-side count of launches issued). */
int64_t rsf_launch_count(int reset);

/* Kernel timing for reporting: while enabled, the library records CUDA events
 * on the launching stream around its batched GEMM launches (category 0 in
 * fp64, 8 in df64 arithmetic on the CUDA cores, 9 on the tensor cores), its
 * pivoted-QR launches (1; category 2 is no
 * longer used: the pivot steps run inside the same persistent launch) and
 * around the phases 3-7 (peeling applications, subtraction of coarser levels,
 * sketch and rank detection, compression of the blocks, factorizations), with
 * each GEMM launch's algorithmic fp64-equivalent flops.  rsf_profile_read
 * returns the totals of a category since the last reset (launches, summed
 * event time in ms, flops, bytes; any output may be NULL) and synchronises
 * the recorded events. */
void rsf_profile_enable(int on);
rsf_status rsf_profile_read(int category, int reset, int64_t* launches, double* ms,
                            double* flops, double* bytes);

/* Frees a handle and all its device memory.  Safe on NULL. */
void rsf_destroy(rsf_handle h);

#ifdef __cplusplus
}
#endif

#endif /* RSF_H */
