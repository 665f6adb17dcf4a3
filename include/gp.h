/*
 * gp.h -- C ABI of libgp: Gaussian-process likelihood and kriging on one
 * NVIDIA GB300 (sm_103a).
 *
 * The method is that of Franey, Ranjan & Chipman, "A Short Note on Gaussian
 * Process Modeling for Large Datasets using Graphics Processing Units":
 *   Section 2, eq. (2): power-exponential correlation
 *       R_ij = prod_k exp(-theta_k |x_ik - x_jk|^p),  p in (0, 2];
 *   Section 2, eq. (3): mu_hat = (1'R^-1 1)^-1 1'R^-1 Y,
 *       sigma2_hat = (Y - 1 mu_hat)' R^-1 (Y - 1 mu_hat) / n;
 *   Section 2, eq. (4): -2 log L = log|R| + n log[(Y-1mu)'R^-1(Y-1mu)];
 *   Section 3: one evaluation of R, one Cholesky factorisation and a few
 *       triangular solves per likelihood value; prediction at N points from
 *       one fit.
 * A diagonal nugget delta >= 0 is added: R_delta = R + delta I (delta = 0
 * allowed).  Cross-correlations r(x*) used for prediction carry no nugget.
 *
 * Conventions for every call:
 *   - Array arguments are DEVICE pointers unless the name ends in _host.
 *     The caller owns them; the library never frees caller memory.
 *   - Matrices are row-major: x is n x d with x[i*d + k]; theta is T x d.
 *   - Work is enqueued on the context's stream.  Calls that return results
 *     to the host (gp_fit, gp_predict's status, *_host variants) synchronise
 *     that stream before returning; the others are asynchronous and report
 *     only argument and launch errors in their return value.
 *   - Return value: GP_OK or a negative gp_status.  The message of the last
 *     failure is available from gp_last_error().
 *   - Arguments are validated: 1 <= n <= 2^20, 1 <= d <= 64,
 *     1 <= T <= 2^30, 0 < p <= 2 (for the power-exponential family; Matern
 *     families ignore p), delta >= 0 and finite.  theta values are checked
 *     on the device: a
 *     theta_k that is negative or not finite makes that candidate's status
 *     GP_EINVAL and its outputs NaN; the rest of the batch completes.
 *   - Per-candidate failures never fail the call: a Cholesky pivot that is
 *     not positive gives status GP_ENOTPD and -2logL = +inf; Q at rounding
 *     level (Y in the span of 1, e.g. n = 1) gives GP_EDEGENERATE and
 *     -2logL = -inf.
 *   - Threads: a context, and the models and plans made from it, are used by
 *     one host thread at a time.  Separate contexts are independent: one per
 *     thread and stream runs their work concurrently on the GPU (the serving
 *     loop does so).
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gp_ctx gp_ctx;
typedef struct gp_model gp_model;
typedef struct gp_plan gp_plan;

/* Arithmetic of the factorisation.
 * GP_FP64:  assembly, Cholesky and solves in IEEE double.
 * GP_MIXED: the panel solves and trailing updates of the blocked Cholesky
 *           on the tensor cores: operands split into bf16 slices, exact fp32
 *           accumulation of the product groups (Ozaki-style), recombined in
 *           double-float (a pair of floats, ~48 significant bits).  Everything
 *           else runs in double-float on the FP32 pipes, not in IEEE double:
 *           the assembly of R (a table-driven exp, ~46 bits), the factor and
 *           inverse of each diagonal block, the forward and backward
 *           substitutions, and the iterative refinement, whose residual
 *           b - R x is formed against a double-float copy of R.  Only the
 *           logarithms of the pivots (log|R|) and the last scalar steps
 *           (mu_hat, Q, -2logL from the double-float sums) are IEEE double.
 * GP_FP32:  the GP_MIXED factorisation with 3 slices in the trailing
 *           updates: 24 significant bits, the precision of an FP32 factor,
 *           at 6 tensor-core products per tile update instead of 15.  Meant
 *           for well-conditioned R: the error of -2logL grows like
 *           cond_1(R) 2^-30 (see gp_nll_batch_ex).
 * GP_AUTO:  per candidate, the cheapest of GP_FP32, GP_MIXED and GP_FP64
 *           whose error bound, from a condition estimate, meets the
 *           context's auto_tol (gp_nll_batch_ex); synchronises.  In
 *           gp_cholesky, which has no candidates to route, GP_MIXED. */
typedef enum {
    GP_FP64 = 0,
    GP_MIXED = 1,
    GP_FP32 = 2,
    GP_AUTO = 3
} gp_precision;

/* Correlation families (gp_options.correlation).
 * GP_CORR_POWEXP:   eq. (2), prod_k exp(-theta_k |x_ik - x_jk|^p), p in (0, 2].
 * GP_CORR_MATERN*:  the Matern family Section 2 names as a numerically more
 *                   stable alternative (it gives no formula), taken in the
 *                   same product form with h = theta_k |x_ik - x_jk| and the
 *                   closed forms for smoothness nu = 1/2, 3/2, 5/2:
 *                   exp(-h), (1 + sqrt3 h) exp(-sqrt3 h),
 *                   (1 + sqrt5 h + 5 h^2/3) exp(-sqrt5 h).  p is ignored.
 * The nugget and every other convention are the same for all families. */
typedef enum {
    GP_CORR_POWEXP = 0,
    GP_CORR_MATERN12 = 1,
    GP_CORR_MATERN32 = 2,
    GP_CORR_MATERN52 = 3
} gp_correlation;

typedef enum {
    GP_OK = 0,
    GP_EINVAL = -1,       /* bad argument                                  */
    GP_ENOMEM = -2,       /* device memory or HBM budget exhausted         */
    GP_ENOTPD = -3,       /* R(theta) not positive definite in arithmetic  */
    GP_ECUDA = -4,        /* CUDA runtime or launch error                  */
    GP_ETIMEOUT = -5,     /* a bounded device wait gave up                 */
    GP_EDEGENERATE = -6,  /* Q = 0 at rounding level: -2logL = -inf        */
    GP_ENOTSUP = -7       /* configuration not built into this library     */
} gp_status;

/* Tunables; gp_default_options() fills the defaults. */
typedef struct {
    int slices;           /* GP_MIXED: bf16 slices per double operand (2..6), default 5 */
    int panel_slices;     /* GP_MIXED: slices of the panel-solve GEMM; fixed at 7 (all
                             product groups exact), other values are rejected */
    int refine_iters;     /* GP_MIXED: most iterative-refinement steps of the solves
                             (0..10), default 1.  Each candidate stops earlier once the
                             error its -2logL has left from Q falls below the error of
                             its log|R|, which no refinement changes: an estimate from
                             its own pivots, 2^-8s (1 + delta) sum_i 1 / L_ii^2 for s
                             slices (2^-40 at the default 5).  Steps
                             that no candidate takes still cost their launches */
    int nugget_in_var;    /* kriging variance uses 1 + delta (1) or 1 (0), default 1 */
    int max_batch;        /* instances factored concurrently (0 = from the budget) */
    int update_groups;    /* GP_MIXED: fp32 accumulators of the trailing update: 3 or 4
                             (128-wide tiles, the last group rounded) or 7 (64-wide
                             tiles, every group exact) */
    int inject_timeout;   /* test hook, default 0, bits: 1 = the first CTA of the first
                             trailing-update launch of each GP_MIXED batch waits 5 ms on
                             a barrier nothing signals, gives up, and the instances it
                             would have updated come back GP_ETIMEOUT; 2 = the first CTA
                             of each tensor-core variance pass of gp_predict does the
                             same and its points' s2 come back NaN (the bounded-wait
                             failure paths, exercised without faulting the GPU) */
    int fuse_panels;      /* GP_MIXED, default 1: panels are factored in pairs with a
                             one-panel look-ahead and both applied to the trailing tiles
                             in one 256-wide pass (half the passes over the trailing
                             matrix); 0: one pass per panel.  Needs update_groups = 4 */
    double auto_tol;      /* GP_AUTO: relative error of -2logL each candidate must meet,
                             default 1e-6 */
    int update_tile;      /* split path: columns of a trailing-update output tile, 128
                             (default) or 64 (twice the work items, for small problems;
                             same products in the same order, so the same results).
                             64 needs update_groups = 4 */
    int assemble_cols;    /* split path: tile columns per CTA of the double-float
                             assembly, 16 (default) or 32; same results */
    int correlation;      /* gp_correlation of every call that builds R or r, default
                             GP_CORR_POWEXP; a fit keeps the family it was made with,
                             and its predictions use that one */
    int predict_tc;       /* gp_predict, default 1: v = L^-1 r for the variances as a
                             block forward substitution of split bf16 GEMMs on the tensor
                             cores (5 slices in the updates, 7 in the diagonal steps,
                             double-float accumulation; variance error ~1e-10 sigma2_hat
                             where cond(R) <= 5e8); 0: the substitution in double-float
                             on the FP32 pipes.  Means are r'w in double-float either way */
} gp_options;

void gp_default_options(gp_options* opt);

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  hbm_budget_bytes
 * bounds the device workspace the context and its models may allocate
 * (0 = 3/4 of the device's free memory).  Returns GP_OK and *ctx, or an
 * error with *ctx = NULL. */
int gp_create(gp_ctx** ctx, int device, size_t hbm_budget_bytes, void* cuda_stream);

/* Free the context's workspace and synchronise its stream.  Workspace and
 * models come from the stream-ordered allocator (cudaMallocAsync), so a
 * context growing its workspace does not stall contexts on other streams. */
void gp_destroy(gp_ctx* ctx);

/* Message of the last failure on this context ("" if none).  Valid until
 * the next call on the context. */
const char* gp_last_error(const gp_ctx* ctx);

/* Switch the stream later calls enqueue on. */
int gp_set_stream(gp_ctx* ctx, void* cuda_stream);

/* Replace the context's tunables (copied). */
int gp_set_options(gp_ctx* ctx, const gp_options* opt);

/* Copy the context's current tunables into *opt (gp_autotune may change them). */
int gp_get_options(const gp_ctx* ctx, gp_options* opt);

/* Bytes of device workspace currently held by the context. */
size_t gp_workspace_bytes(const gp_ctx* ctx);

/* Phase timers.  While timing is on, every group of kernel launches is
 * bracketed by CUDA events on the context's stream; gp_phase_times
 * synchronises the stream, returns the accumulated milliseconds and kernel
 * launches per phase (GP_PHASE_*) since the previous call, and resets them.
 * The launch counts are kept whether or not timing is on. */
enum {
    GP_PHASE_ASSEMBLE = 0,   /* theta checks + correlation assembly        */
    GP_PHASE_POTRF = 1,      /* diagonal-tile factorisation (and inverse)  */
    GP_PHASE_TRSM = 2,       /* panel solve                                */
    GP_PHASE_UPDATE = 3,     /* trailing update                            */
    GP_PHASE_SOLVE = 4,      /* triangular solves, refinement, reductions  */
    GP_PHASE_SPLIT = 5,      /* bf16 slicing of panels (GP_MIXED)          */
    GP_PHASE_PREDICT = 6,    /* kriging kernels                            */
    GP_NUM_PHASES = 8
};
int gp_set_timing(gp_ctx* ctx, int on);
int gp_phase_times(gp_ctx* ctx, double* ms, long long* launches, int nphases);

/* Kernels this context has launched since it was created. */
long long gp_launch_count(const gp_ctx* ctx);

/* R(theta) + delta I by eq. (2) (Section 2) for ONE theta (length d).
 * layout 0: dense n x n row-major, both triangles (R[i*n + j]).
 * layout 1: the factorisation's storage: lower-triangular 128 x 128 tiles,
 *           tile (I, J) (I >= J) at offset (J*nt - J*(J-1)/2 + I - J)*16384
 *           doubles with nt = ceil(n/128), column-major inside a tile
 *           (element (r, c) at r + 128 c); rows and columns >= n hold the
 *           identity; diagonal tiles hold both triangles.
 *           R must hold nt(nt+1)/2 * 16384 doubles.
 * layout 2: the split-precision path's storage: the tiles of layout 1 with
 *           each entry as a pair of floats (hi, lo), hi + lo ~ R_ij to about
 *           46 bits (exp evaluated in double-float arithmetic); same size in
 *           bytes as layout 1.  Entries below 2^-125 are zero.
 * Asynchronous. */
int gp_corr_assemble(gp_ctx* ctx, int n, int d, const double* x, const double* theta,
                     double p, double delta, double* R, int layout);

/* The Cholesky factor of R(theta) + delta I (Section 3: one factorisation
 * per likelihood value) for ONE theta, in the tile layout of
 * gp_corr_assemble (layout 1): the lower triangle of every tile holds L
 * (the upper triangle of diagonal tiles is unspecified).  prec selects the
 * factorisation (GP_MIXED: the split-precision factor, returned in double).
 * L must hold nt(nt+1)/2 * 16384 doubles.  *status_host receives GP_OK,
 * GP_ENOTPD or GP_EINVAL.  Synchronises. */
int gp_cholesky(gp_ctx* ctx, int n, int d, const double* x, const double* theta, double p,
                double delta, int prec, double* L, int* status_host);

/* Profile -2 log-likelihood, eq. (4), at T candidate theta vectors (T x d),
 * with the profile estimates of eq. (3).  Outputs (length T each):
 *   nll[t]        -2logL = log|R| + n log Q  (eq. 4 read literally)
 *   mu_hat[t]     eq. (3)
 *   sigma2_hat[t] Q / n, eq. (3)
 *   logdet[t]     log|R| = 2 sum log L_ii   (may be NULL)
 *   status[t]     GP_OK, GP_ENOTPD, GP_EDEGENERATE or GP_EINVAL
 * prec selects the factorisation's arithmetic (gp_precision).
 * The candidates are factored in batches sized by the context's budget.
 * Asynchronous. */
int gp_nll_batch(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                 const double* theta, double p, double delta, int prec,
                 double* nll, double* mu_hat, double* sigma2_hat, double* logdet,
                 int* status);

/* Gradient of -2 log L (eq. 4) with respect to theta, with -2logL itself,
 * at T candidates (T x d):
 *   grad[t*d + k] = d(-2logL)/dtheta_k = tr(R^-1 dR_k) - (n/Q) w' dR_k w,
 * w = R^-1 (Y - 1 mu_hat) (mu_hat minimises Q, so it does not move the
 * gradient), dR_k = dR/dtheta_k (zero on the diagonal: the nugget does not
 * depend on theta); for every gp_correlation.  Section 2 names a multi-start
 * gradient-based search as a possibly faster alternative to its GA; this is
 * the gradient such a search needs.  -2logL, mu_hat and w come from the
 * IEEE-double factor (nll equals gp_nll_batch's GP_FP64 result); R^-1 is
 * formed from that factor in double-float, about 48 bits (L^-1 by tile
 * diagonals, then L^-T L^-1: twice the factorisation's n^3/6 multiply-adds),
 * so the gradient's relative error is about cond(R) 2^-47 at worst.  nll,
 * status as gp_nll_batch; grad rows are NaN where the status is not GP_OK.
 * d <= 16 (GP_ENOTSUP above).
 * Asynchronous. */
int gp_nll_grad_batch(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                      const double* theta, double p, double delta, double* nll, double* grad,
                      int* status);

/* gp_nll_batch with two more outputs (length T, each may be NULL):
 *   cond1[t]     1-norm condition estimate of R(theta_t) + delta I: ||R||_1
 *                times Hager's estimate of ||R^-1||_1 (W. W. Hager, SIAM J.
 *                Sci. Stat. Comput. 5, 1984; the iteration LAPACK's
 *                condition estimators refine).  It is taken with the candidate's own split-precision factor
 *                after the likelihood: up to five rounds of two solves, all
 *                candidates in step.  A lower bound of the true value up to
 *                the factor's error, in practice within a small factor.  NaN
 *                where the status is GP_EINVAL or GP_ENOTPD.  Not available
 *                with GP_FP64: cond1 must then be NULL (GP_ENOTSUP).
 *   prec_used[t] the arithmetic the candidate's outputs come from: GP_FP32,
 *                GP_MIXED or GP_FP64 (prec itself unless prec is GP_AUTO).
 * GP_AUTO evaluates every candidate with GP_FP32 and its estimate.  One whose
 * status is not GP_OK, or whose cond1 * 2^-30 exceeds the context's auto_tol,
 * is evaluated again with GP_MIXED, whose bound is cond1 * 2^-(8 s + 6) for s
 * slices; one that fails that test as well is evaluated with GP_FP64.  The
 * bounds are the largest error of -2logL per unit of cond_1 measured on the
 * n = 4000 benchmark batch (cond_1 from 2e7 to 4e11), with a margin of 10 or
 * more.  cond1 then holds each candidate's last split-precision estimate.
 * GP_AUTO synchronises the stream (the routing reads the estimates on the
 * host) and takes its staging buffers from the stream-ordered allocator.
 * Other precisions are asynchronous like gp_nll_batch. */
int gp_nll_batch_ex(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                    const double* theta, double p, double delta, int prec,
                    double* nll, double* mu_hat, double* sigma2_hat, double* logdet,
                    int* status, double* cond1, int* prec_used);

/* Launch-shape autotuner.  Times gp_nll_batch(prec) on the caller's batch
 * for every combination of update_tile (128, 64), fuse_panels (1, 0) and
 * assemble_cols (16, 32) -- one untimed call, then `reps` calls timed with
 * CUDA events on the context's stream, median -- and keeps the fastest as
 * the context's options.  update_tile and assemble_cols never change results; fuse_panels changes the rounding of the trailing updates (both
 * settings meet the split path's accuracy).  trials (may be NULL) receives
 * up to max_trials entries and *ntrials the number of combinations timed.
 * prec: GP_MIXED or GP_FP32 (GP_ENOTSUP otherwise: the FP64 path has no
 * shape choices).  Outputs go to a staging area; synchronises. */
typedef struct {
    int update_tile;
    int fuse_panels;
    int assemble_cols;
    double ms;            /* median device time of one gp_nll_batch call */
} gp_tune_trial;
int gp_autotune(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                const double* theta, double p, double delta, int prec, int reps,
                gp_tune_trial* trials, int max_trials, int* ntrials);

/* A batch recorded as one CUDA graph.  gp_plan_nll_batch evaluates the call
 * once (eagerly, so that its outputs are also valid on return), then records
 * the same call's kernel sequence on a private stream and instantiates it;
 * gp_plan_launch replays it on the context's current stream as a single
 * graph launch.  The paper evaluates candidates one after another (Section 3);
 * the graph removes the per-kernel launch cost of a batch, which dominates
 * for small n.
 *   - The plan binds the argument ADDRESSES: every replay reads the current
 *     contents of x, y and theta and overwrites the outputs.  The caller
 *     keeps those buffers alive, and n, d, T, p, delta and prec fixed, for
 *     the plan's lifetime.
 *   - The plan owns its workspace (counted against the context's budget like
 *     a model), so other calls on the context do not disturb it; replays of
 *     one plan must not overlap each other on the GPU.
 *   - prec: GP_FP64, GP_MIXED or GP_FP32 (GP_AUTO routes on the host and is
 *     rejected with GP_ENOTSUP).  cond1 may be NULL.
 *   - The context's options at creation are baked in.
 * gp_plan_nll_batch synchronises; gp_plan_launch is asynchronous and adds
 * the plan's kernels to the context's launch count.  A plan may outlive its
 * context (gp_plan_destroy then frees it synchronously). */
int gp_plan_nll_batch(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                      const double* theta, double p, double delta, int prec, double* nll,
                      double* mu_hat, double* sigma2_hat, double* logdet, int* status,
                      double* cond1, gp_plan** plan);
int gp_plan_launch(gp_plan* plan);
long long gp_plan_kernels(const gp_plan* plan);   /* kernels in one replay */
size_t gp_plan_bytes(const gp_plan* plan);        /* device bytes the plan holds */
void gp_plan_destroy(gp_plan* plan);

/* gp_nll_batch with every array in host memory: the call copies the inputs
 * to the device, evaluates, copies the outputs back and synchronises.
 * Host buffers may be pageable or pinned. */
int gp_nll_batch_host(gp_ctx* ctx, int n, int d, const double* x_host,
                      const double* y_host, int T, const double* theta_host, double p,
                      double delta, int prec, double* nll_host, double* mu_hat_host,
                      double* sigma2_hat_host, double* logdet_host, int* status_host);

/* gp_nll_batch in IEEE double (GP_FP64) for callers that cannot let the
 * library allocate device memory -- services that reserve their whole device
 * budget at start-up, hosts whose allocator must account for every byte, or
 * callers that cannot afford the device-wide synchronisation of cudaMalloc
 * and cudaFree.  The paper has no counterpart: it is an interface variant,
 * not part of the method.
 *   - Working memory is one fixed array of GP_NOALLOC_SCRATCH_BYTES inside
 *     the library (reserved on every GPU that loads the library, until the
 *     process exits); the call allocates nothing.  Candidates are processed
 *     in as many rounds as the array needs; n above GP_NOALLOC_MAX_N does not
 *     fit one candidate and is rejected with GP_ENOMEM and a message.
 *   - The first call on a device looks up the array's device address (a
 *     runtime query, done once per device, with the context's device made
 *     current); make that first call before any stream capture.
 *   - Every call on a device shares the array: calls whose work overlaps on
 *     the GPU (other streams, other contexts, other threads) race and corrupt
 *     each other's results.  Calls in order on one stream are safe; nothing
 *     needs clearing between calls (every buffer is written before it is
 *     read).
 * Arguments, outputs and asynchrony are those of gp_nll_batch. */
#define GP_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
#define GP_NOALLOC_MAX_N 2816
int gp_nll_batch_noalloc(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                         const double* theta, double p, double delta, double* nll,
                         double* mu_hat, double* sigma2_hat, double* logdet, int* status);

/* Fit at one theta (length d): assemble, factor, solve, and keep on the
 * device what kriging needs (Section 3: one factorisation, then solves per
 * test point).  prec:
 *   GP_FP64 (and GP_AUTO): the factor in IEEE double; kriging means and
 *       variances to double precision (the paper, too, refines its final
 *       fit with double-precision runs, Sections 4-5).
 *   GP_MIXED, GP_FP32: the split-precision factor of gp_nll_batch, with its
 *       iterative refinement: kriging means carry about cond(R) 2^-46 of
 *       relative error (w is refined), variances about cond(R) 2^-40 (the
 *       solve v = L^-1 r uses the split factor); several times faster than
 *       GP_FP64 from n ~ 4000 on.  The context's workspace grows as for
 *       gp_nll_batch with T = 1.
 * Kept on the device: the factor L, w = R^-1 (Y - 1 mu_hat), a = L^-1 1 and a
 * copy of x, as double-float pairs (hi + lo floats, ~48 bits) for the
 * kriging kernel, and the scalars.  Synchronises.  On GP_OK (or
 * GP_EDEGENERATE: the mean is still usable), *model owns that device memory
 * until gp_model_free.  A fit whose R is not positive definite returns
 * GP_ENOTPD and no model. */
int gp_fit(gp_ctx* ctx, int n, int d, const double* x, const double* y,
           const double* theta, double p, double delta, int prec, gp_model** model);

/* gp_nll_batch at T candidates, then a fit (as gp_fit) at the best of them:
 * the one with the smallest -2logL among those with status GP_OK (ties: the
 * first).  The model is built from that candidate's own factor, which the
 * batch has just computed, with no second factorisation (unless the batch ran
 * in several chunks and the best one's factor was overwritten: then it is
 * factored again, with the same result).  This is the last step of a
 * multi-start search (Section 4: the paper's GA ends with the best
 * candidate's fit and its predictions).
 *   prec: GP_FP64, GP_MIXED or GP_FP32 (GP_ENOTSUP for GP_AUTO); the model
 *         carries that precision (gp_fit).
 *   nll .. status: as gp_nll_batch (device arrays of length T, logdet may be
 *         NULL).
 *   *best_host: index of the best candidate, or -1 if none gave GP_OK (the
 *         call then returns GP_ENOTPD and no model).
 * Synchronises.  Returns GP_OK or GP_EDEGENERATE with *model set, or an
 * error. */
int gp_fit_batch(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                 const double* theta, double p, double delta, int prec, double* nll,
                 double* mu_hat, double* sigma2_hat, double* logdet, int* status,
                 int* best_host, gp_model** model);

/* Scalars of a fit: out[0..5] = -2logL, mu_hat, sigma2_hat, log|R|, Q, a'a. */
int gp_model_scalars(const gp_model* model, double* out_host);

/* Kriging prediction (Section 3: one R, one factorisation, two solves per
 * test point) at N points xstar (N x d, device):
 *   yhat[m] = mu_hat + r' R^-1 (Y - 1 mu_hat)
 *   s2[m]   = sigma2_hat [c0 - r'R^-1 r + (1 - 1'R^-1 r)^2 / (1'R^-1 1)]
 * with r_i = corr(z(x*_m), z(x_i)) by eq. (2), c0 = 1 + delta (or 1 when
 * the context's nugget_in_var is 0).  s2 may be NULL (mean only).
 * With predict_tc (the default) the call first cuts the model's factor into
 * bf16 slices in its workspace (gp_call_bytes counts them) and then forms
 * v = L^-1 r 128 points at a time on the tensor cores; yhat has the same
 * bits with or without s2.  A variance pass that gives up on a bounded wait
 * leaves NaN in the s2 of the points it had not finished.
 * 0 <= N <= 2^30 per call (GP_EINVAL beyond: split larger sets).
 * Asynchronous; the model must outlive the enqueued work. */
int gp_predict(gp_ctx* ctx, const gp_model* model, int N, const double* xstar,
               double* yhat, double* s2);

/* Release a model's device memory (stream-ordered on the context's stream,
 * which is then synchronised).  A model may outlive its context: gp_destroy
 * detaches it, and gp_model_free then releases it synchronously. */
void gp_model_free(gp_model* model);

/* Device bytes a model holds (0 for NULL). */
size_t gp_model_bytes(const gp_model* model);

/* Calls whose device memory gp_call_bytes reports. */
typedef enum {
    GP_CALL_NLL_BATCH = 0,  /* gp_nll_batch / gp_nll_batch_ex at precision prec, count = T */
    GP_CALL_NLL_GRAD = 1,   /* gp_nll_grad_batch, count = T */
    GP_CALL_FIT = 2,        /* gp_fit: the model's bytes (gp_model_bytes); count unused */
    GP_CALL_PREDICT = 3     /* gp_predict with variances (s2 != NULL), count = N test
                               points, n and d those of the model */
} gp_call;

/* Device bytes a call would allocate for these sizes: for GP_CALL_FIT the model,
 * otherwise the workspace the call grows the context's arena to (what
 * gp_workspace_bytes reports after the call on a context whose arena was
 * smaller).  The candidates of a batch are processed in chunks that fit the
 * budget, as the calls themselves do, so the figure is for one chunk.
 * GP_AUTO gives an upper bound: the largest workspace of its three tiers plus
 * its routing buffers.  Per candidate these are the buffers of Section 3's
 * work (one R, its factor, the solves), so they grow like n^2 / 2.
 * Host arithmetic only: no device access and no allocation, so it works
 * without a GPU.
 *   ctx    the context whose options, budget and device (SM count) the call
 *          would use, or NULL: default options, no budget limit, 152 SMs.
 *   call   a gp_call.  prec: a gp_precision, read for GP_CALL_NLL_BATCH only.
 *   bytes  out (host).
 * Returns GP_OK; GP_EINVAL for sizes the call rejects (n, d, count) or an
 * unknown call or precision; GP_ENOTSUP where the call is not built for the
 * sizes (gradient with d > 16); GP_ENOMEM where the call would fail for the
 * context's budget. */
int gp_call_bytes(gp_ctx* ctx, int call, int n, int d, int count, int prec, size_t* bytes);

#ifdef __cplusplus
}
#endif

#endif /* GP_H */
