// Internal plan of the gbcca library: shapes, options and device workspace.
#pragma once
#include <vector>

#include "common.cuh"

namespace gbcca {

constexpr int kMaxK = 20;       // columns of an iterate (p in the paper)
constexpr int kMaxD = 1024;     // columns of one data view
constexpr int kMaxBatch = 1024;  // plans of one batch
constexpr int kMaxClasses = 64; // LDA classes
constexpr int kMaxTimedBatch = 256;  // iterations per batch when passes are timed

enum ProblemKind { kCCA = 0, kLDA = 1 };

// Scalars and k x k matrices of the Riemannian CG state, resident on the
// device so one iteration runs without host round trips.
struct DevState {
  int iter, done, status, stalled, passes, ls_trials, first, force_zero_step;
  double t, f, df, t_prev, df_prev, gn, gn0, beta, t0, gtol, ftrial_best;
  double mu[kMaxK];
  double lam[2];
  double Linv[2][kMaxK * kMaxK];    // L^{-T} of the accepted retraction, per view
  double S[2][3][kMaxK * kMaxK];    // Sylvester solutions (grad, eta, old grad)
  double sigma[kMaxK];              // Rayleigh-Ritz values at the end
  double rot[2][2 * kMaxK * kMaxK]; // Rayleigh-Ritz rotation per view (rr_m x k)
  int rr_m;                         // dimension of the Rayleigh-Ritz subspace used (k or 2k)
  int rr_ok;                        // 1 if the last Rayleigh-Ritz step factored its Grams
  int ritz_checks;                  // Ritz-value checks recorded in this solve
  int ritz_small;                   // consecutive checks whose change was below rtol
  int check_iter;                   // iterations done at this iteration's pass (0: no check)
  int ritz_stop;                    // the Ritz-value rule has been met (done after the join)
  double YW[kMaxClasses * kMaxK];   // FDA: Yhat times the current W (l x k)
  double ftrial[64];                // line-search trial values (diagnostics)
  double Qsyl[2][kMaxK * kMaxK];    // eigenvectors of the last Sylvester coefficient
  int max_iter;
  int ntrials;
  int qsyl_valid;
  double dacc[2][6];                // direction: per-view inner products
  int dcount;                       // direction: views finished this iteration
  int ls_count;                     // line search: trials finished this iteration
};

// One generalized Stiefel factor: the data view it is built on and the
// iterate that lives on it.
struct View {
  int d = 0;
  const void* Z = nullptr;  // caller-owned data, row-major n x d, leading dim ld
  int64_t ld = 0;
  double lam = 0;
  int ocol = 0;             // first column of this view's block in the pass W
  double* SZ = nullptr;     // sketch S Z (s x d)
  float* SZh = nullptr;     // S Z as a float pair (FP32/BF16 plans)
  float* SZl = nullptr;
  double* R = nullptr;      // d x d upper triangular, R^T R = M
  double* Rinv = nullptr;   // d x d, R^{-1}
  float* Rinv32 = nullptr;  // FP32 copy for the low-precision path
  float* Minv_hi = nullptr; // M^{-1} = R^{-1} R^{-T} as a float pair (low-precision plans)
  float* Minv_lo = nullptr;
  float* RRh = nullptr;     // d x 2k: RR[:, 0:2k] as a float pair (input of the M^{-1} product)
  float* RRl = nullptr;
  double* Phi = nullptr;    // d x 2k: [U | eta]
  float* Phi32 = nullptr;   // FP32 copy of Phi for the low-precision pass
  double* Meta = nullptr;   // d x k: M eta
  double* gold = nullptr;   // d x k: previous Riemannian gradient
  double* Mgold = nullptr;  // d x k: M * previous gradient
  double* LL = nullptr;     // d x 4k: [M^{-1} B U | M^{-1} egrad | eta | grad]
  double* RR = nullptr;     // d x 4k: [B U | egrad | M eta | M grad]
  double* tmp = nullptr;    // d x 2k scratch for M^{-1}
  double* warm = nullptr;   // d x k warm start
  double* wsU = nullptr;    // d x 2k warm-start iteration block
  double* wsT = nullptr;    // d x 2k warm-start scratch
};

struct Plan {
  int kind = kCCA;
  int64_t n = 0;
  int k = 0;
  int dtype = GBCCA_FP64;
  gbcca_options opt{};
  int nviews = 0;
  View v[2];
  int D = 0;    // total data columns (dx + dy, or d)
  int NC = 0;   // pass columns: 4k (CCA) or 2k (LDA)
  int64_t s = 0, n_pad = 0;
  int l = 0;    // LDA classes
  bool preconditioned = false;
  int64_t dev_bytes = 0;   // device memory the plan allocated (workspace, copies of the data)
  int dev = 0;
  int sm_count = 0;

  // sketch randomness and CountSketch sort buffers
  int32_t* h = nullptr;     // CountSketch buckets (n) or SRHT rows (s)
  int8_t* g = nullptr;      // CountSketch signs (n) or SRHT signs (n_pad)
  int32_t* cs_tab = nullptr;  // per-chunk bucket counters (cs_nch x s)
  int32_t* cs_off = nullptr;  // bucket offsets (s + 1)
  int32_t* perm = nullptr;    // rows sorted by bucket (n)
  int cs_nch = 0;
  void* srht_T = nullptr;     // SRHT stage-1 scratch (n_pad x dmax)

  // pass buffers
  double* G = nullptr;        // D x NC
  double* Gt = nullptr;       // NC x D: G column-major (tensor-core pass plans), for the Gram
  double* Gram = nullptr;     // NC x NC
  void* Wbuf = nullptr;       // n x NC (pass intermediate)
  void* partG = nullptr;      // chunksB x D x NC
  void* partGram = nullptr;   // ctasA x NC x NC
  void* partCls = nullptr;    // ctasA x l x NC (LDA per-class sums)
  int ctasA = 0, chunksB = 0;

  // LDA
  const int32_t* labels = nullptr;
  double* counts = nullptr;   // l
  double* means = nullptr;    // l x d
  double* Yhat = nullptr;     // l x d
  double* Cls = nullptr;      // l x NC: class means times Phi
  double* YPhi = nullptr;     // l x 2k: Yhat Phi
  double* clsPart = nullptr;  // class-statistics partials

  // RCG state
  DevState* st = nullptr;
  DevState* st_host = nullptr;  // pinned mirror for read-back
  int* flag_host = nullptr;     // pinned mirror of the device error flag
  double* phigram = nullptr;    // per view 2k x 2k Gram of Phi
  double* phipart = nullptr;    // partials of phigram
  double* phired = nullptr;     // per view 2k x 2k Gram of Phi (summed partials)
  double* cross = nullptr;      // per view 4k x 4k cross Gram (final)
  double* crosspart = nullptr;  // partials
  int thinCtas = 0;
  double* history = nullptr;    // 3 (max_iter + 1)
  double* ritz_hist = nullptr;  // Ritz values at every check: (max_iter / check_every + 2) x k
  int ritz_len = 0;             // rows of ritz_hist
  double* mt_part = nullptr;    // slice partials of mat_thin
  float* dfx = nullptr;         // 2 x dmax x 2k floats: split blocks for double-float products
  double* ls_f = nullptr;       // line-search trial values (kNTrials)
  double* ls_L = nullptr;       // line-search trial factors (kNTrials x 2 x kMaxK^2)
  double* ws = nullptr;         // FP64 scratch for dense routines
  int64_t ws_len = 0;
  int* flag = nullptr;          // device error flag (NOT_SPD etc.)
  cudaEvent_t ev[2 * kMaxTimedBatch];  // pass timing (opt.time_passes)
  int nev = 0;

  // tensor-core pass (BF16 CCA): TMA descriptors of X and Y (CUtensorMap,
  // 128 bytes each, rebuilt when the data pointers change), the swizzled Phi
  // image and the per-CTA FP32 partials of G
  alignas(64) unsigned char tc_map[2][128];
  const void* tc_map_for[2] = {nullptr, nullptr};
  uint8_t* tc_img = nullptr;
  float* tc_part = nullptr;
  int tc_clusters = 0;
  // one batch of RCG iterations as a CUDA graph: captured on the plan's own
  // stream (the caller's may be the legacy default stream, which cannot be
  // captured), replayed on the solve's stream; the key records what the
  // captured launches depend on besides plan-owned memory
  cudaStream_t cap_stream = nullptr;
  // side stream and fork/join events for independent per-view work
  cudaStream_t side_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaEvent_t ritz_fork = nullptr, ritz_join = nullptr;  // the Ritz-check branch of an iteration
  // an iteration's Phi Gram on a branch beside the pass reduction: the
  // solver asks for it (fork_after_pass), the tensor-core pass records
  // pass_fork after its data kernels (pass_forked)
  cudaEvent_t pass_fork = nullptr, pass_join = nullptr;
  bool fork_after_pass = false, pass_forked = false;
  cudaGraphExec_t batch_exec = nullptr;
  const void* batch_key_ptr[3] = {nullptr, nullptr, nullptr};
  int batch_key_n = 0;
  bool batch_key_timed = false;
  long long batch_launches = 0;  // kernels in one replay (for the launch counter)
  // tensor-core pass for FP32 data: row-interleaved BF16 hi/lo copies of
  // the bound views (FDA: of the class-centred rows; rows 2i / 2i + 1 hold
  // hi / lo of data row i), leading dimension ts_ld; ts_ready once made
  __nv_bfloat16* ts_copy[2] = {nullptr, nullptr};
  int64_t ts_ld[2] = {0, 0};
  bool ts_ready = false;
  cudaEvent_t kev0 = nullptr;  // when set: recorded around the data kernel of the next pass
  cudaEvent_t kev1 = nullptr;  // resident 2-CTA clusters of the tensor-core pass (0: not yet queried)
};

// sketch.cu
int sketch_draws(int kind, int64_t n, int64_t s, uint64_t seed, int32_t* h, int8_t* g,
                 cudaStream_t st);
int countsketch_apply(Plan& p, int view, bool center, cudaStream_t st);
int countsketch_prepare(Plan& p, cudaStream_t st);
int srht_apply(Plan& p, int view, cudaStream_t st);

// dense.cu
// C = A^T B + diag_add I over m rows, FP64 (split-K partials in ws).
int gram_tn(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t m, int d1,
            int d2, double* C, double diag_add, double* ws, int64_t ws_len, cudaStream_t st);
// The same in double-float arithmetic (~2^-44 relative per product) from
// float-pair inputs (m x d1 and m x d2, row-major) at FP32 instruction rates;
// tri: A and B lower triangular (zero rows of a tile skipped).
int gram_df_split(const float* Ah, const float* Al, int64_t lda, const float* Bh, const float* Bl, int64_t ldb,
                  int64_t m, int d1, int d2, double* C, double diag_add, double* ws, int64_t ws_len, cudaStream_t st,
                  bool tri = false);
int cholesky_upper(double* A, int d, int* flag, cudaStream_t st);
// C = A^T A + lambda I (A: m x d FP64, row stride lda) with the split-K
// partials in a static device scratch instead of plan memory; d <= noalloc_max_d().
int gram_noalloc(const double* A, int64_t lda, int64_t m, int d, double lambda, double* C, cudaStream_t st);
int noalloc_max_d();
// Double-float matrices (hi + lo float pairs) times FP64 thin blocks:
// Y_b[:, 0:c] = A_b X_b[:, 0:c] for up to two problems in one launch
// (A_b m x K row-major; c even, <= 40; X rows 16-byte aligned).
struct DfmvProblem {
  const float* hi;   // A, m x K
  const float* lo;
  const float* Xh;   // X, K x c (row stride ldx floats)
  const float* Xl;
  double* Y;         // m x c (row stride ldy doubles)
  int m, K;
  int ldx, ldy;
};
struct DfmvArgs {
  DfmvProblem p[2];
  int c;             // columns of X and Y (at most 64)
  const int* done;
  int kc;            // K chunk staged in shared memory (set by dfmv)
};
int dfmv(const DfmvArgs& a, int nprob, cudaStream_t st);
// hi/lo split of the first c columns of X (rows x ldx) into rows x c floats
int split_rows(const double* X, int rows, int c, int ldx, float* hi, float* lo, cudaStream_t st);
// hi/lo split of A (r x c, row-major) or of its transpose (c x r)
int split_df(const double* A, int r, int c, bool trans, float* hi, float* lo, cudaStream_t st);
// M^{-1} = R^{-1} R^{-T} as a double-float pair (d x d)
int minv_df_build(const double* Rinv, int d, float* hi, float* lo, double* ws, int64_t ws_len, cudaStream_t st);
// Rinv = R^{-1} (upper triangular, d x d); ws holds at least d * d doubles.
int tri_inverse_upper(const double* R, double* Rinv, int d, double* ws, int64_t ws_len, cudaStream_t st);
int to_f32(const double* a, float* b, int64_t len, cudaStream_t st);
// C (m x c, ldc) = op(A) B (rows of B = columns of op(A), ldb); A is
// ra x ca row-major; tri = 1 skips the zero half of an upper-triangular A.
// `part` is scratch of ceil(K / 64) * m * min(c, 40) doubles.
template <typename T>
int mat_thin(const T* A, int ra, int ca, bool transA, bool tri, const double* B, int64_t ldb, double* C,
             int64_t ldc, int c, double* part, cudaStream_t st);

// pass.cu
int fused_pass(Plan& p, bool low, bool gram_only, cudaStream_t st, int phi_cols = 0,
               const int* done = nullptr);
int fused_pass_cores(Plan& p, bool low, bool gram_only, cudaStream_t st, int phi_cols,
               const int* done);
int exact_gram(Plan& p, int view, double* out, cudaStream_t st);
int lda_class_stats(Plan& p, cudaStream_t st);

// pass_tc.cu
bool tc_pass_eligible(const Plan& p);
int tc_pass(Plan& p, cudaStream_t st, const int* done);
int tc_phi_image(Plan& p, int h1, cudaStream_t st, const int* done);
int tc_groups(const Plan& p);
bool tc_quad(const Plan& p);
// batched tensor-core pass over several eligible plans (one persistent launch)
struct TcBatch;
TcBatch* tc_batch_create(Plan* const* plans, int n, cudaStream_t st, int* rc);
void tc_batch_destroy(TcBatch* b);
int tc_batch_schedule(TcBatch* b, const bool* active, int clusters, cudaStream_t st);
int tc_batch_pre(const TcBatch* b, Plan& p, cudaStream_t st);
int tc_batch_launch(TcBatch* b, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1);
int tc_batch_post(const TcBatch* b, int i, Plan& p, cudaStream_t st, const int* done);
int tc_batch_h1(const TcBatch* b);
int* tc_batch_err(TcBatch* b);
int tc_batch_max_clusters(const TcBatch* b);
int tc_batch_clusters(const TcBatch* b);
int64_t tc_batch_bytes(const TcBatch* b, const bool* active);

// hilo_copy.cu: the BF16 hi/lo copy of FP32 data for the tensor-core pass
int hilo_alloc(Plan& p);
int hilo_prepare(Plan& p, cudaStream_t st);

// api.cu
int lda_bind(Plan& p, const void* X, int64_t ldx, const int32_t* labels, double lambda, const int32_t* sketch_h,
             const int8_t* sketch_g, cudaStream_t st);

// batch.cu: lockstep executor over several plans
struct Batch;
Batch* batch_make(Plan* const* plans, int count, const gbcca_batch_options* opt, int* rc);
void batch_free(Batch* b);
int batch_size(const Batch& b);
int batch_tune(Batch& b, cudaStream_t st);
int batch_iterate(Batch& b, const std::vector<char>& active, int nb, bool graph, cudaStream_t st);
int batch_poll(Batch& b, std::vector<char>& active, gbcca_info* infos, cudaStream_t st, int* err_plan);

// rcg.cu
int rcg_run(Plan& p, const double* mu, double tol, double* out0, double* out1, double* vals,
            gbcca_info* info, cudaStream_t st);
// the pieces of rcg_run, for executors that interleave several plans
int rcg_begin(Plan& p, const double* mu, double tol, const double* start0, const double* start1, cudaStream_t st);
int iteration_post(Plan& p, bool low, cudaStream_t st);
int rcg_finish(Plan& p, double* out0, double* out1, double* vals, gbcca_info* info, double pass_ms, int pass_count,
               cudaStream_t st);
int read_state_async(Plan& p, cudaStream_t st);
int check_flag(Plan& p, gbcca_info* info, cudaStream_t st);
int warm_start(Plan& p, cudaStream_t st);

}  // namespace gbcca
