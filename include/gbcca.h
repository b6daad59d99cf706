/*
 * gbcca.h - C ABI of the GB300 (sm_103a) sketch-preconditioned Riemannian
 * solver for regularized CCA and Fisher LDA on tall data (n >> d).
 *
 * Method: Shustin & Avron, "Faster Randomized Methods for Orthogonality
 * Constrained Problems".  Problem statements: Def. 4.1 (CCA) and Def. 5.1
 * (FDA).  Algorithm: Alg. 1 (CCA) and Alg. 2 (FDA) - sketch the data,
 * factor the sketch preconditioner M = Z^T S^T S Z + lambda I as R^T R
 * (Sec. 3), warm-start from the exact solution of the sketched problem, then
 * run Riemannian CG on the generalized Stiefel manifold with the metric
 * g(xi, eta) = tr(xi^T M eta) (Table 1).
 *
 * Conventions for every entry point:
 *   - Matrices are row-major.  A data matrix of n rows and d columns with
 *     leading dimension ld (elements, ld >= d) has element (i, j) at
 *     base[i * ld + j].  Iterates U (dx x k), V (dy x k), W (d x k) are dense
 *     row-major float64 with leading dimension k.
 *   - Pointers named "device" must point to memory of the current CUDA device;
 *     "host" pointers are plain CPU memory.  The library never frees memory
 *     it did not allocate.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work of a call is ordered on that stream; a call
 *     returns after its work is enqueued unless it says it synchronizes.
 *   - Return value: GBCCA_OK (0) or a negative gbcca_status.  No C++
 *     exception crosses this interface.  gbcca_last_error() gives a one-line
 *     description of the most recent failure on the calling thread.
 *   - A plan is not thread-safe: one thread at a time may use it.
 */
#ifndef GBCCA_H
#define GBCCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbcca_plan_s* gbcca_plan_t;

/* Storage type of the data matrices X, Y (the arithmetic type of the data
 * pass is FP32 accumulate for BF16/FP32 data and FP64 for FP64 data). */
enum gbcca_dtype { GBCCA_BF16 = 0, GBCCA_FP32 = 1, GBCCA_FP64 = 2 };

/* Preconditioner M of the Riemannian metric.
 *   COUNTSKETCH  M = (S Z)^T (S Z) + lambda I, S a CountSketch (Sec. 3).
 *   SRHT         S a subsampled randomized Hadamard transform (App. A).
 *   IDENTITY     M = I (no preconditioning; the "M = I" ablation of Sec. 6).
 *   EXACT        M = Z^T Z + lambda I (the "M = Sigma" ablation of Sec. 6;
 *                S = I, costs O(n d^2)); FP64 CCA plans only (cca_plan
 *                returns GBCCA_ERR_UNSUPPORTED otherwise). */
enum gbcca_sketch {
  GBCCA_SKETCH_COUNTSKETCH = 0,
  GBCCA_SKETCH_SRHT = 1,
  GBCCA_SKETCH_IDENTITY = 2,
  GBCCA_SKETCH_EXACT = 3
};

enum gbcca_status {
  GBCCA_OK = 0,
  GBCCA_ERR_INVALID_ARG = -1,   /* bad shape, pointer or option           */
  GBCCA_ERR_UNSUPPORTED = -2,   /* valid but not implemented (size limit) */
  GBCCA_ERR_OOM = -3,           /* device allocation failed               */
  GBCCA_ERR_NOT_SPD = -4,       /* a Cholesky pivot was not positive      */
  GBCCA_ERR_MAXITER = -5,       /* max_iter reached; results are written  */
  GBCCA_ERR_TIMEOUT = -6,       /* a bounded device wait ran out          */
  GBCCA_ERR_CUDA = -7,          /* CUDA runtime error                     */
  GBCCA_ERR_STATE = -8          /* call out of order (e.g. solve before precondition) */
};

/* Options of a plan.  Fill with gbcca_default_options() and override. */
typedef struct {
  int32_t sketch;        /* enum gbcca_sketch                                   */
  int64_t s;             /* sketch rows; 0 = 4 (dx + dy) for CCA, 3 d for LDA   */
  uint64_t seed;         /* seed of the library's own sketch draws              */
  int32_t max_iter;      /* Riemannian CG iteration cap (default 1000)          */
  double gtol;           /* stop when ||grad||_M <= gtol ||grad_0||_M (1e-8)    */
  int32_t refine;        /* final Rayleigh-Ritz step of BF16/FP32 plans: 1
                            (default) over span(U) with Grams from an FP64
                            pass (exact products of the stored data), 2 over
                            span([U, eta]) with the Grams of the plan's own
                            pass.  FP64 plans always use span([U, eta]) with
                            their exact FP64 pass.                           */
  int32_t warm_start;    /* 1: start from the exact solution of the sketched
                            problem (Alg. 1 step 4 / Alg. 2 step 5); 0: start
                            from the U/V (W) buffers passed to the solve call  */
  int32_t check_every;   /* iterations between convergence read-backs (8)      */
  int32_t time_passes;   /* 1: time the data kernel of every fused pass (the
                            kernel that streams X and Y) with CUDA events on
                            the solve's stream (reported in gbcca_info)         */
  int32_t graphs;        /* 1: each batch of check_every iterations is replayed
                            from a CUDA graph that the plan captures on its own
                            stream at the first solve (re-captured when the
                            data pointers change; with time_passes the timing
                            events are recorded by the graph); 0: the kernels
                            are launched one by one.  Both run the same
                            kernels in the same order.                          */
  double rtol;           /* stop when the Rayleigh-Ritz values of the subspace
                            span([U, eta]) x span([V, eta_V]) (the values the
                            final refinement reports) change by less than rtol
                            relative to the largest of them, at two consecutive
                            checks (check_every iterations apart); 0 (default)
                            = off.  Either rule (gtol or rtol) ends the
                            iteration.                                      */
  int32_t tensor_cores;  /* 1 (default): the data pass runs on the tensor-core
                            kernels where the plan is eligible (CCA: BF16 or
                            FP32 data, any shape, BF16 rows 16-byte aligned;
                            FDA: FP32 data, d <= 1024); 0:
                            the CUDA-core kernels only (for comparisons)     */
  int32_t warm_iters;    /* block power iterations of the CCA warm start (the
                            exact CCA of the sketched pair, Alg. 1 step 4);
                            0 = the default 12, which reaches the exact
                            sketched solution to ~1e-6 in subspace angle     */
  int64_t wait_cycles;   /* bound, in GPU clock cycles, on one pipeline wait of
                            the FDA tensor-core pass for FP32 data (0 = the
                            default 2e9, about one second; the CCA passes
                            always use the default).  A wait that runs
                            out stops the pass early: every CTA drains its own
                            copies and MMAs, and the call returns
                            GBCCA_ERR_TIMEOUT.  Small values exist to exercise
                            that path.                                      */
  int32_t retraction;    /* retraction onto St_B (Table 1): 0 (default) the QR
                            retraction, computed as (U + xi) L^{-T} with
                            L L^T = (U + xi)^T B (U + xi); 1 the polar
                            retraction (U + xi) ((U + xi)^T B (U + xi))^{-1/2}
                            (for tangent xi: (U + xi)(I + xi^T B xi)^{-1/2}),
                            the inverse square root from a k x k symmetric
                            eigendecomposition per line-search trial.  The
                            starting point is normalized by the same map.   */
} gbcca_options;

/* Per-solve report (host struct filled by the solve calls). */
typedef struct {
  int32_t iters;         /* Riemannian CG iterations taken                      */
  int32_t passes;        /* fused data passes over the n rows                   */
  int32_t status;        /* gbcca_status of the solve                           */
  int32_t stalled;       /* 1 if the line search found no decrease (f at its
                            rounding floor), which also ends the iteration      */
  double grad_norm;      /* ||grad||_M at the last iterate                      */
  double grad_norm0;     /* ||grad||_M at the first iterate                     */
  double objective;      /* f at the iterate before the final Rayleigh-Ritz step */
  double pass_ms;        /* with opt.time_passes: mean device time of the data
                            kernel of one fused pass (ms, CUDA events), else 0  */
  int32_t pass_count;    /* passes included in pass_ms                          */
} gbcca_info;

/* Fills `opt` with defaults (CountSketch, s = 0, seed 0, max_iter 1000,
 * gtol 1e-8, refine 1, warm_start 1, check_every 8, time_passes 0, graphs 1,
 * rtol 0, tensor_cores 1, warm_iters 0 (12), wait_cycles 0, retraction 0).
 * Returns GBCCA_OK or
 * GBCCA_ERR_INVALID_ARG if opt is NULL. */
int gbcca_default_options(gbcca_options* opt);

/* Regularized CCA plan (Def. 4.1; Alg. 1 inputs: X n x dx, Y n x dy,
 * s >= max(dx, dy)).  Validates shapes (1 <= k <= min(dx, dy) <= 1024,
 * k <= 20, n >= max(dx, dy)), copies `opt` (host; NULL = defaults), allocates
 * all device workspace (sketches, R factors, iterates, pass partials) on the
 * current device, and writes the handle to *plan (host).  Returns
 * GBCCA_ERR_OOM if the workspace does not fit. */
int cca_plan(gbcca_plan_t* plan, int64_t n, int32_t dx, int32_t dy, int32_t k,
             int32_t dtype, const gbcca_options* opt);

/* Alg. 1 steps 2-5 (Sec. 3 preconditioner, Sec. 4.4): sketch X and Y with the
 * same S, factor M_xx = R_x^T R_x and M_yy = R_y^T R_y in FP64 (R from the
 * Cholesky factorization of the sketch Gram, which is the R factor of the QR
 * of [S Z; sqrt(lambda) I]), and compute the warm start (exact CCA of the
 * sketched pair, step 4).  X (n x dx, leading dimension ldx) and Y (n x dy,
 * ldy) are device pointers of the plan's dtype; the caller owns them and must
 * keep them valid and unchanged until the last cca_solve on this plan.
 * lambda_x, lambda_y >= 0, and > 0 unless the sketch has full column rank.
 * Optional explicit sketch randomness (device, may be NULL to let the
 * library draw from opt.seed): CountSketch: h (int32, n entries in [0, s)),
 * g (int8, n entries +-1); SRHT: h = sampled row indices (int32, s entries,
 * distinct, in [0, n_pad)), g = signs (int8, n_pad entries), n_pad the
 * power of two >= n.  The two views' Cholesky factorizations run
 * concurrently: view 1 on a stream owned by the plan, ordered after the
 * work already on `stream` and joined back to it by events.  Synchronizes
 * `stream` to check the factorizations;
 * returns GBCCA_ERR_NOT_SPD if a factor breaks down. */
int cca_precondition(gbcca_plan_t plan, const void* X, int64_t ldx, const void* Y, int64_t ldy,
                     double lambda_x, double lambda_y, const int32_t* sketch_h,
                     const int8_t* sketch_g, void* stream);

/* Alg. 1 step 8: Riemannian CG for max tr(U^T Sxy V N) on
 * St_Sxx(k, dx) x St_Syy(k, dy) with the metric of M (Sec. 4.2-4.4).
 * mu (host, k entries, strictly decreasing, > 0; NULL = 1 + (k - 1 - i) / 100
 * for i = 0 .. k - 1) is the diagonal of N; the solution does not depend on
 * N (Thm 4.1), its conditioning does (Thm 4.4): near-equal weights converge
 * the subspace fastest and the final Rayleigh-Ritz step separates the pairs.  tol overrides opt.gtol when > 0.  U (dx x k), V (dy x k)
 * and sigma (k) are device buffers (float64, caller-owned); with
 * opt.warm_start = 0, U and V also provide the starting point.  On return
 * sigma holds the canonical correlations sigma_1 >= ... >= sigma_k and U, V
 * the canonical weights (U^T Sxx U = I, V^T Syy V = I, U^T Sxy V = diag(sigma)),
 * from a final Rayleigh-Ritz step on the computed subspaces.  info (host,
 * may be NULL) receives the report.  This call synchronizes `stream`
 * every opt.check_every iterations to read the convergence flag.
 * Returns GBCCA_OK, GBCCA_ERR_MAXITER (results still written) or an error. */
int cca_solve(gbcca_plan_t plan, const double* mu, double tol, double* U, double* V,
              double* sigma, gbcca_info* info, void* stream);

/* Fisher LDA plan (Def. 5.1; Alg. 2 inputs X n x d, labels, s >= d).
 * 2 <= n_classes <= 64, 1 <= k <= n_classes - 1, k <= 20, d <= 1024. */
int lda_plan(gbcca_plan_t* plan, int64_t n, int32_t d, int32_t n_classes, int32_t k,
             int32_t dtype, const gbcca_options* opt);

/* Alg. 2 end to end: class statistics (S_B = Yhat^T Yhat and the class means
 * that define Xhat, Sec. 5.1), sketch of Xhat, preconditioner, warm start
 * (exact FDA of the sketch), Riemannian CG for max tr(W^T S_B W N) on
 * St_{S_w + lambda I}(k, d), and a final Rayleigh-Ritz step.  X (device,
 * n x d, ld), labels (device int32, n entries in [0, n_classes); every class
 * must be non-empty), W (device float64, d x k; also the start when
 * opt.warm_start = 0), rho (device float64, k: the generalized eigenvalues of
 * (S_B, S_w + lambda I)), mu as for cca_solve, info (host, may be NULL).
 * X and labels must stay valid until the call returns.  Synchronizes like
 * cca_solve. */
int lda_solve(gbcca_plan_t plan, const void* X, int64_t ldx, const int32_t* labels,
              double lambda, const double* mu, double tol, const int32_t* sketch_h,
              const int8_t* sketch_g, double* W, double* rho, gbcca_info* info, void* stream);

/* One fused data pass (the per-iteration hot path, Sec. 4.4 / Cor. 4.6):
 * with Phi_x (dx x 2k) and Phi_y (dy x 2k) device float64 row-major (columns
 * [U, eta_U] and [V, eta_V]), computes in one sweep over the rows of the
 * plan's X and Y (set by cca_precondition):
 *   W = [X Phi_x, Y Phi_y] (n x 4k, kept on chip), Gx = X^T W (dx x 4k),
 *   Gy = Y^T W (dy x 4k), Gram = W^T W (4k x 4k),
 * written as float64 row-major device arrays (caller-owned).  Arithmetic is
 * the plan's: FP64 for FP64 data, FP32 accumulation otherwise.  For an LDA
 * plan (after lda_solve) the pass is the FDA one: Phi (d x 2k) in Phi_x,
 * Phi_y ignored, W = Xhat Phi, Gx = Xhat^T W (d x 2k), Gram (2k x 2k), Gy
 * unused.  Enqueued on `stream`; no synchronization. */
int gbcca_fused_pass(gbcca_plan_t plan, const double* Phi_x, const double* Phi_y,
                     double* Gx, double* Gy, double* Gram, void* stream);

/* Copies an internal result of the last precondition / solve to `dst`
 * (device float64 buffer of at least gbcca_query_size(plan, what) elements).
 * Used to check each step of the method on its own. */
enum gbcca_query {
  GBCCA_Q_SKETCH_X = 0,   /* S X  (s x dx), or S Xhat for LDA              */
  GBCCA_Q_SKETCH_Y = 1,   /* S Y  (s x dy)                                 */
  GBCCA_Q_R_X = 2,        /* R_x  (dx x dx, upper triangular)              */
  GBCCA_Q_R_Y = 3,        /* R_y  (dy x dy)                                */
  GBCCA_Q_WARM_U = 4,     /* warm start U~ (dx x k) before qf_B            */
  GBCCA_Q_WARM_V = 5,     /* warm start V~ (dy x k)                        */
  GBCCA_Q_HISTORY = 6,    /* per iteration (f, ||grad||_M, t): 3 (max_iter+1) */
  GBCCA_Q_CLASS_MEANS = 7, /* LDA class means (n_classes x d)              */
  GBCCA_Q_RITZ = 8        /* with opt.rtol > 0: the Ritz values of every check
                             of the last solve, row r (k values) after
                             iteration (r + 1) check_every;
                             (max_iter / check_every + 2) x k, zero rows
                             after the last check                          */
};
int64_t gbcca_query_size(gbcca_plan_t plan, int32_t what);
int gbcca_query(gbcca_plan_t plan, int32_t what, double* dst, void* stream);

/* Draws the library's own sketch randomness for `seed` (Sec. 3 CountSketch:
 * h[n] in [0, s), g[n] = +-1; App. A SRHT: rows[s] distinct in [0, n_pad),
 * signs[n_pad]) into device buffers.  Every value is a function of
 * (seed, index) through SplitMix64 (Steele, Lea & Flood 2014):
 * r = mix(seed + (i + 1) 0x9E3779B97F4A7C15); CountSketch h = ((r >> 32) s)
 * >> 32, g = (r & 1) ? -1 : +1; SRHT signs from bit 0 of the stream at
 * seed ^ 0xD1B54A32D192ED03, rows = pi(0..s-1) for a 4-round Feistel
 * permutation pi of [0, n_pad) keyed by seed ^ 0x8CB92BA72F3D8DD7 (odd log2
 * sizes use cycle walking).  kind = GBCCA_SKETCH_COUNTSKETCH (h: n entries,
 * g: n entries) or GBCCA_SKETCH_SRHT (h: s rows, g: n signs, n a power of
 * two). */
int gbcca_sketch_draws(int32_t kind, int64_t n, int64_t s, uint64_t seed, int32_t* h,
                       int8_t* g, void* stream);

/* Allocation-free Gram of a sketch: C = A^T A + lambda I, the matrix whose
 * Cholesky factor is the preconditioner R of Sec. 3 (A = S Z, e.g. read back
 * with GBCCA_Q_SKETCH_X).  The paper has no counterpart for the
 * allocation-free form; it exists for callers that may not allocate device
 * memory during a call: processes that reserve HBM in their own pool up front,
 * and callers that cannot accept the device-wide synchronization cudaMalloc /
 * cudaFree may cause.
 *   A       device, row-major m x d FP64, row stride lda >= d (elements)
 *   C       device, d x d FP64 row-major output (caller-owned)
 *   lambda  >= 0, added to the diagonal
 * Arithmetic: FP64 split-K partial sums over row chunks, added in a fixed
 * order (deterministic).  Memory: the partials live in a static 8 MiB device
 * array of the library (no allocation, nothing needs zeroing), so
 * d <= gbcca_sketch_gram_noalloc_max_d() (1024); larger d returns
 * GBCCA_ERR_INVALID_ARG without device work.  The first call on a device
 * looks up the array's address; make it before recording a stream capture.
 * The array is shared by all callers on a device: calls that may run at the
 * same time (different streams, unordered threads) race and must be
 * ordered by the caller.  Work is ordered on `stream`; returns GBCCA_OK,
 * GBCCA_ERR_INVALID_ARG or GBCCA_ERR_CUDA. */
int gbcca_sketch_gram_noalloc(const double* A, int64_t lda, int64_t m, int32_t d, double lambda, double* C,
                              void* stream);
int32_t gbcca_sketch_gram_noalloc_max_d(void);

/* ---------------------------------------------------------------- batches
 * Several prepared plans solved together.  The paper states one problem at a
 * time (Alg. 1 / Alg. 2 run per instance); the batch only schedules those
 * instances on one GPU.  Each plan must have been bound to its data
 * (cca_precondition / lda_solve's preconditioning through a previous call)
 * with opt.warm_start on, and stays owned by the caller; its data must stay
 * valid while the batch exists.  Every iteration, the data passes of the
 * plans the tensor-core pass serves (CCA, BF16 or FP32 data; k > 12 in two
 * column groups of Phi) run as ONE persistent launch (two when some plans
 * have a view wider than 512 columns: those run in 4-CTA clusters) over a schedule of (instance,
 * 64-row tile range) segments cut into near-equal work per 2-CTA cluster;
 * the other plans run their own passes.  Each plan's small kernels run on a
 * graph branch of their own, and each plan stops on its own rule (its
 * options); a finished plan leaves the schedule.  The result of every plan
 * is the one its own cca_solve / lda_solve would give up to the rounding of
 * its pass. */
typedef struct gbcca_batch_s* gbcca_batch_t;

typedef struct {
  int32_t clusters;      /* 2-CTA clusters of the batched launch; 0 (default):
                            the fastest of a few candidates, timed once per
                            batch on the plans' start points              */
  int32_t graphs;        /* 1 (default): batches of iterations replay a
                            captured CUDA graph; 0: launched one by one    */
  int32_t batch_iters;   /* iterations per replay (default 8)              */
} gbcca_batch_options;

typedef struct {
  int32_t iterations;          /* lockstep iterations run, the qf_B step included */
  int32_t clusters;            /* clusters of the batched launch                  */
  int32_t batched_plans;       /* plans whose passes ran in the batched launch    */
  int32_t reserved;
  double batched_pass_ms;      /* device time of one batched pass over all of
                                  them at the chosen schedule (CUDA events)       */
  double batched_pass_bytes;   /* its algorithmic bytes: sum of n (dx + dy) x the
                                  element size of each plan's data                */
} gbcca_batch_report;

/* Fills `opt` with the defaults (clusters 0, graphs 1, batch_iters 8). */
int gbcca_default_batch_options(gbcca_batch_options* opt);

/* Creates a batch over plans[0 .. count - 1] (host array of handles,
 * 1 <= count <= 1024, no repeats).  Returns GBCCA_OK, GBCCA_ERR_INVALID_ARG,
 * GBCCA_ERR_STATE (a plan not bound to data, or without warm start),
 * GBCCA_ERR_OOM or GBCCA_ERR_CUDA. */
int gbcca_batch_create(gbcca_batch_t* batch, const gbcca_plan_t* plans, int32_t count,
                       const gbcca_batch_options* opt);

/* Solves every plan of the batch.  U, V, sigma: host arrays of `count`
 * device pointers, entry i as for plan i's cca_solve (U dx x k, V dy x k,
 * sigma k) or lda_solve (W in U, rho in sigma, V unused); infos: host array
 * of `count` reports or NULL; report: host, or NULL.  Returns GBCCA_OK, the
 * first plan's GBCCA_ERR_MAXITER (all results still written), or the first
 * error.  Synchronizes `stream`. */
int gbcca_batch_solve(gbcca_batch_t batch, double* const* U, double* const* V, double* const* sigma,
                      gbcca_info* infos, gbcca_batch_report* report, void* stream);

/* One batched data pass alone (every plan of the batch must be served by
 * the tensor-core pass): for plan i, with Phi_x[i] (dx x 2k) and Phi_y[i]
 * (dy x 2k), writes G[i] = [X^T W, Y^T W] ((dx + dy) x 4k) and Gram[i] =
 * W^T W (4k x 4k), W = [X Phi_x, Y Phi_y], as gbcca_fused_pass does for one
 * plan.  Resets each plan's iteration state.  Synchronizes `stream`. */
int gbcca_batch_fused_pass(gbcca_batch_t batch, const double* const* Phi_x, const double* const* Phi_y,
                           double* const* G, double* const* Gram, void* stream);

void gbcca_batch_destroy(gbcca_batch_t batch);

/* ---------------------------------------------------------------- serving
 * A request loop over solves that arrive over time; like the batch, it only
 * schedules the paper's per-problem algorithms (Alg. 1 / Alg. 2) on one GPU.
 * Requests wait in a FIFO queue until the device memory they need (their
 * data copies, plan workspace and outputs, counted when their plan is made)
 * fits the budget beside the running ones; a request larger than the whole
 * budget fails with GBCCA_ERR_OOM.  At admission the server copies the
 * request's data into its own device buffers (rows padded to 16 bytes),
 * makes and preconditions the plan, and sets up the iteration.  Every
 * gbcca_server_step advances all running requests by tick_iters lockstep
 * iterations (the batch executor: one persistent tensor-core launch per
 * iteration for the plans it serves), then refines the finished ones, keeps
 * their outputs and returns their memory to the budget, so queued requests
 * join the next step.  One thread drives a server. */
typedef struct gbcca_server_s* gbcca_server_t;

typedef struct {
  int64_t hbm_budget;    /* device bytes the running requests may hold
                            (default 120 GiB)                               */
  int32_t max_active;    /* running requests at most (default 64, <= 1024)   */
  int32_t tick_iters;    /* lockstep iterations per step (default 8)         */
  int32_t graphs;        /* 1 (default): a step whose running set is the one
                            of the previous step replays a captured graph    */
} gbcca_server_options;

typedef struct {
  int32_t kind;          /* 0 = CCA, 1 = FDA                                 */
  int32_t dtype;         /* gbcca_dtype of the data                          */
  int64_t n;
  int32_t dx;            /* CCA: columns of X; FDA: d                        */
  int32_t dy;            /* CCA: columns of Y                                */
  int32_t k;
  int32_t n_classes;     /* FDA                                              */
  double lambda_x;       /* FDA: lambda                                      */
  double lambda_y;
  const void* X;         /* row-major n x dx, row stride ldx elements, in
                            memory the GPU can read (device, or pinned or
                            registered host memory); read at admission, so it
                            must stay valid until the request is running     */
  int64_t ldx;
  const void* Y;         /* CCA: n x dy, row stride ldy                      */
  int64_t ldy;
  const int32_t* labels; /* FDA: n labels in [0, n_classes), same rule       */
  gbcca_options opt;     /* solver options (warm_start is forced on)         */
} gbcca_request;

typedef struct {
  double submit_s;       /* host steady-clock seconds since the server was
                            created: submission, admission, finish          */
  double admit_s;
  double finish_s;
  int64_t device_bytes;  /* device memory the request held while running:
                            its plan's allocations, its data copies and
                            outputs, as requested from the allocator        */
} gbcca_request_times;

/* Fills `opt` with the defaults above. */
int gbcca_default_server_options(gbcca_server_options* opt);

int gbcca_server_create(gbcca_server_t* server, const gbcca_server_options* opt);

/* Queues a request (host struct, copied); *id receives its handle.  Only the
 * request's form is checked here; a request the library cannot serve fails
 * at admission (its result call reports why).  No device work. */
int gbcca_server_submit(gbcca_server_t server, const gbcca_request* req, int64_t* id);

/* One tick: admission, tick_iters iterations of every running request,
 * retirement of the finished ones.  Writes the queued and running counts
 * (host, may be NULL).  Work is ordered on `stream` and the call
 * synchronizes it. */
int gbcca_server_step(gbcca_server_t server, int32_t* queued, int32_t* running, void* stream);

/* 0 queued, 1 running, 2 finished, 3 failed; GBCCA_ERR_INVALID_ARG for an
 * unknown id. */
int gbcca_server_state(gbcca_server_t server, int64_t id);

/* Result of a finished or failed request, then forgets it.  U (dx x k), V
 * (dy x k, CCA), vals (k: correlations or FDA values): float64 buffers in
 * device or host memory, or NULL to skip; info and times: host, or NULL.
 * Returns the request's status (GBCCA_OK, GBCCA_ERR_MAXITER with results,
 * or the error that ended it), GBCCA_ERR_STATE while it is queued or
 * running.  Synchronous. */
int gbcca_server_result(gbcca_server_t server, int64_t id, double* U, double* V, double* vals, gbcca_info* info,
                        gbcca_request_times* times);

void gbcca_server_destroy(gbcca_server_t server);

/* Number of CUDA kernels this library has launched in this process (all
 * plans and threads); a host-side counter for profiling. */
int64_t gbcca_launch_count(void);

void gbcca_plan_destroy(gbcca_plan_t plan);
const char* gbcca_status_string(int status);
const char* gbcca_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GBCCA_H */
