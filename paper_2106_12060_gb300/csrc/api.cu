// C ABI of the gbcca library: plans, preconditioning (Alg. 1 steps 2-5,
// Alg. 2 steps 2-6), solves (Alg. 1 step 8, Alg. 2 step 9), the stand-alone
// fused pass, and read-back of intermediate results.
#include <cstring>
#include <new>

#include "plan.h"

namespace gbcca {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }
std::atomic<long long> g_launches{0};

namespace {

template <typename T>
int dalloc(T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  cudaError_t e = counted_malloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)count);
  if (e != cudaSuccess) {
    set_last_error(std::string("cudaMalloc of ") + std::to_string(sizeof(T) * count) + " bytes: " +
                   cudaGetErrorString(e));
    cudaGetLastError();
    return GBCCA_ERR_OOM;
  }
  return GBCCA_OK;
}

void dfree(void* p) {
  if (p != nullptr) cudaFree(p);
}

int64_t next_pow2(int64_t n) {
  int64_t m = 1;
  while (m < n) m <<= 1;
  return m;
}

void free_plan(Plan* p) {
  if (p == nullptr) return;
  for (int v = 0; v < 2; ++v) {
    View& w = p->v[v];
    for (void* q : {(void*)w.SZ, (void*)w.R, (void*)w.Rinv, (void*)w.Rinv32, (void*)w.Minv_hi, (void*)w.Minv_lo, (void*)w.SZh, (void*)w.SZl, (void*)w.RRh, (void*)w.RRl, (void*)w.Phi, (void*)w.Phi32,
                    (void*)w.Meta, (void*)w.gold, (void*)w.Mgold, (void*)w.LL, (void*)w.RR, (void*)w.tmp,
                    (void*)w.warm, (void*)w.wsU, (void*)w.wsT})
      dfree(q);
  }
  for (void* q : {(void*)p->h, (void*)p->g, (void*)p->cs_tab, (void*)p->cs_off, (void*)p->perm, p->srht_T,
                  (void*)p->G, (void*)p->Gt, (void*)p->Gram, p->Wbuf, p->partG, p->partGram, p->partCls, (void*)p->counts,
                  (void*)p->means, (void*)p->Yhat, (void*)p->Cls, (void*)p->YPhi, (void*)p->clsPart, (void*)p->st,
                  (void*)p->phigram, (void*)p->phipart, (void*)p->phired, (void*)p->cross, (void*)p->crosspart, (void*)p->history, (void*)p->ritz_hist,
                  (void*)p->ws, (void*)p->flag, (void*)p->tc_img, (void*)p->tc_part, (void*)p->mt_part, (void*)p->dfx, (void*)p->ls_f, (void*)p->ls_L})
    dfree(q);
  for (int v = 0; v < 2; ++v) dfree(p->ts_copy[v]);
  if (p->st_host != nullptr) cudaFreeHost(p->st_host);
  if (p->flag_host != nullptr) cudaFreeHost(p->flag_host);
  for (int i = 0; i < p->nev; ++i) cudaEventDestroy(p->ev[i]);
  if (p->batch_exec != nullptr) cudaGraphExecDestroy(p->batch_exec);
  if (p->cap_stream != nullptr) cudaStreamDestroy(p->cap_stream);
  if (p->side_stream != nullptr) cudaStreamDestroy(p->side_stream);
  if (p->fork_ev != nullptr) cudaEventDestroy(p->fork_ev);
  if (p->join_ev != nullptr) cudaEventDestroy(p->join_ev);
  if (p->ritz_fork != nullptr) cudaEventDestroy(p->ritz_fork);
  if (p->ritz_join != nullptr) cudaEventDestroy(p->ritz_join);
  if (p->pass_fork != nullptr) cudaEventDestroy(p->pass_fork);
  if (p->pass_join != nullptr) cudaEventDestroy(p->pass_join);
  delete p;
}

int alloc_plan(Plan* p) {
  const int k = p->k, k2 = 2 * k, k4 = 4 * k;
  int dmax = 0;
  for (int v = 0; v < p->nviews; ++v) dmax = std::max(dmax, p->v[v].d);
  for (int v = 0; v < p->nviews; ++v) {
    View& w = p->v[v];
    const int d = w.d;
    GB_TRY(dalloc(&w.SZ, p->s * d));
    GB_TRY(dalloc(&w.R, (int64_t)d * d));
    GB_TRY(dalloc(&w.Rinv, (int64_t)d * d));
    GB_TRY(dalloc(&w.Rinv32, (int64_t)d * d));
    if (p->dtype != GBCCA_FP64) {
      GB_TRY(dalloc(&w.Minv_hi, (int64_t)d * d));
      GB_TRY(dalloc(&w.Minv_lo, (int64_t)d * d));
      GB_TRY(dalloc(&w.RRh, (int64_t)d * k2));
      GB_TRY(dalloc(&w.RRl, (int64_t)d * k2));
      GB_TRY(dalloc(&w.SZh, p->s * d));
      GB_TRY(dalloc(&w.SZl, p->s * d));
    }
    GB_TRY(dalloc(&w.Phi, (int64_t)d * k2));
    GB_TRY(dalloc(&w.Phi32, (int64_t)d * k2));
    GB_TRY(dalloc(&w.Meta, (int64_t)d * k));
    GB_TRY(dalloc(&w.gold, (int64_t)d * k));
    GB_TRY(dalloc(&w.Mgold, (int64_t)d * k));
    GB_TRY(dalloc(&w.LL, (int64_t)d * k4));
    GB_TRY(dalloc(&w.RR, (int64_t)d * k4));
    GB_TRY(dalloc(&w.tmp, (int64_t)d * k2));
    GB_TRY(dalloc(&w.warm, (int64_t)d * k));
    GB_TRY(dalloc(&w.wsU, (int64_t)d * k2));
    GB_TRY(dalloc(&w.wsT, (int64_t)d * k2));
  }
  const bool srht = p->opt.sketch == GBCCA_SKETCH_SRHT;
  if (srht) {
    GB_TRY(dalloc(&p->h, p->s));
    GB_TRY(dalloc(&p->g, p->n_pad));
    GB_TRY(dalloc(&p->cs_tab, 1024));
    GB_TRY(dalloc(&p->cs_off, 1025));
    GB_TRY(dalloc(&p->perm, p->s));
    size_t tsz = p->dtype == GBCCA_FP64 ? sizeof(double) : sizeof(float);
    void* t = nullptr;
    cudaError_t e = counted_malloc(&t, tsz * (size_t)p->n_pad * dmax);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_last_error("SRHT scratch allocation failed");
      return GBCCA_ERR_OOM;
    }
    p->srht_T = t;
  } else {
    p->cs_nch = (int)std::max<int64_t>(1, std::min<int64_t>(p->sm_count, (p->n + 255) / 256));
    GB_TRY(dalloc(&p->h, p->n));
    GB_TRY(dalloc(&p->g, p->n));
    GB_TRY(dalloc(&p->cs_tab, (int64_t)p->cs_nch * p->s));
    GB_TRY(dalloc(&p->cs_off, p->s + 1));
    GB_TRY(dalloc(&p->perm, std::max<int64_t>(p->n, p->s)));
  }
  GB_TRY(dalloc(&p->G, (int64_t)p->D * p->NC));
  GB_TRY(dalloc(&p->Gram, (int64_t)p->NC * p->NC));
  p->ctasA = (int)std::max<int64_t>(1, std::min<int64_t>(2 * p->sm_count, (p->n + 63) / 64));
  int nb = 0;
  for (int v = 0; v < p->nviews; ++v) nb += ceil_div(p->v[v].d, 64);
  p->chunksB = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(2 * p->sm_count, nb), (p->n + 31) / 32));
  size_t esz = sizeof(double);
  {
    void* t = nullptr;
    if (counted_malloc(&t, esz * (size_t)p->n * p->NC) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("pass intermediate allocation failed");
      return GBCCA_ERR_OOM;
    }
    p->Wbuf = t;
  }
  {
    double* t;
    GB_TRY(dalloc(&t, (int64_t)p->chunksB * p->D * p->NC));
    p->partG = t;
    GB_TRY(dalloc(&t, (int64_t)p->ctasA * p->NC * p->NC));
    p->partGram = t;
    GB_TRY(dalloc(&t, (int64_t)p->ctasA * std::max(1, p->l) * p->NC));
    p->partCls = t;
  }
  if (p->kind == kLDA) {
    GB_TRY(dalloc(&p->counts, p->l));
    GB_TRY(dalloc(&p->means, (int64_t)p->l * p->D));
    GB_TRY(dalloc(&p->Yhat, (int64_t)p->l * p->D));
    GB_TRY(dalloc(&p->Cls, 2 * (int64_t)p->l * k2));
    GB_TRY(dalloc(&p->YPhi, (int64_t)p->l * k2));
    GB_TRY(dalloc(&p->clsPart, 128 * (int64_t)p->l * p->D + 128 * (int64_t)p->l));
  }
  GB_TRY(dalloc(&p->st, 1));
  GB_CUDA(cudaMallocHost(reinterpret_cast<void**>(&p->st_host), sizeof(DevState)));
  GB_CUDA(cudaMallocHost(reinterpret_cast<void**>(&p->flag_host), sizeof(int)));
  const int nblk = ceil_div(dmax, 16);  // thin-Gram row blocks
  GB_TRY(dalloc(&p->phigram, 4096));
  GB_TRY(dalloc(&p->phipart, (int64_t)p->nviews * nblk * 4 * k * k));
  GB_TRY(dalloc(&p->phired, (int64_t)p->nviews * 4 * k * k));
  GB_TRY(dalloc(&p->cross, (int64_t)p->nviews * 16 * k * k));
  GB_TRY(dalloc(&p->crosspart, (int64_t)p->nviews * nblk * std::max(16 * k * k, p->l * p->l)));
  GB_TRY(dalloc(&p->history, 3 * (int64_t)(p->opt.max_iter + 1)));
  p->ritz_len = p->opt.max_iter / std::max(1, p->opt.check_every) + 2;
  GB_TRY(dalloc(&p->ritz_hist, (int64_t)p->ritz_len * k));
  p->ws_len = 8 * (int64_t)dmax * dmax + 3 * (int64_t)dmax * std::max(std::max(p->l, k2), 1) + 4096;
  GB_TRY(dalloc(&p->ws, p->ws_len));
  GB_TRY(dalloc(&p->mt_part, (int64_t)ceil_div(dmax, 64) * dmax * 40));
  GB_TRY(dalloc(&p->dfx, 2 * (int64_t)dmax * k2));
  GB_TRY(dalloc(&p->ls_f, 64));
  GB_TRY(dalloc(&p->ls_L, 64 * 2 * (int64_t)kMaxK * kMaxK));
  GB_TRY(dalloc(&p->flag, 1));
  GB_CUDA(cudaMemset(p->flag, 0, sizeof(int)));
  const bool tc_cca = p->kind == kCCA && (p->dtype == GBCCA_BF16 || p->dtype == GBCCA_FP32);
  const bool tc_fda = p->kind == kLDA && p->dtype == GBCCA_FP32 && dmax <= 1024;
  if ((tc_cca || tc_fda) && p->opt.tensor_cores) {
    // Phi images per column group (two groups for 2k > 24): CCA both views'
    // (twice the K-boxes for views wider than 512), FDA the one view's in 16
    // K-boxes; and the per-cluster partial slabs of every group
    const int64_t img = (2 * k <= 24 ? 1 : 2) * (tc_cca ? 2 * (dmax > 512 ? 2 : 1) : 2) * 49152;
    GB_TRY(dalloc(&p->tc_img, img));
    GB_CUDA(cudaMemset(p->tc_img, 0, img));
    GB_TRY(dalloc(&p->Gt, (int64_t)p->D * p->NC));
    GB_TRY(dalloc(&p->tc_part, (int64_t)p->sm_count * p->D * (k4 + 8)));
  }
  GB_TRY(hilo_alloc(*p));
  GB_CUDA(cudaStreamCreateWithFlags(&p->side_stream, cudaStreamNonBlocking));
  GB_CUDA(cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming));
  GB_CUDA(cudaEventCreateWithFlags(&p->join_ev, cudaEventDisableTiming));
  GB_CUDA(cudaEventCreateWithFlags(&p->ritz_fork, cudaEventDisableTiming));
  GB_CUDA(cudaEventCreateWithFlags(&p->ritz_join, cudaEventDisableTiming));
  GB_CUDA(cudaEventCreateWithFlags(&p->pass_fork, cudaEventDisableTiming));
  GB_CUDA(cudaEventCreateWithFlags(&p->pass_join, cudaEventDisableTiming));
  if (p->opt.time_passes) {
    for (int i = 0; i < 2 * kMaxTimedBatch; ++i) {
      GB_CUDA(cudaEventCreate(&p->ev[i]));
      p->nev = i + 1;
    }
  }
  return GBCCA_OK;
}

int check_options(const gbcca_options& o) {
  if (o.sketch < 0 || o.sketch > 3) return GBCCA_ERR_INVALID_ARG;
  if (o.max_iter < 1 || o.s < 0 || !(o.gtol >= 0) || o.check_every < 1 || o.wait_cycles < 0 || !(o.rtol >= 0) ||
      o.warm_iters < 0 || o.retraction < 0 || o.retraction > 1)
    return GBCCA_ERR_INVALID_ARG;
  return GBCCA_OK;
}

int make_plan(gbcca_plan_t* out, int kind, int64_t n, int d0, int d1, int nviews, int k, int l, int dtype,
              const gbcca_options* opt) {
  if (out == nullptr) {
    set_last_error("plan pointer is NULL");
    return GBCCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (dtype < GBCCA_BF16 || dtype > GBCCA_FP64) {
    set_last_error("unknown dtype");
    return GBCCA_ERR_INVALID_ARG;
  }
  Plan* p = new (std::nothrow) Plan();
  if (p == nullptr) return GBCCA_ERR_OOM;
  gbcca_default_options(&p->opt);
  if (opt != nullptr) p->opt = *opt;
  if (check_options(p->opt) != GBCCA_OK) {
    delete p;
    set_last_error("invalid options");
    return GBCCA_ERR_INVALID_ARG;
  }
  if (p->opt.sketch == GBCCA_SKETCH_EXACT && (dtype != GBCCA_FP64 || kind != kCCA)) {
    delete p;
    set_last_error("the exact metric (M = Sigma) is implemented for FP64 CCA plans");
    return GBCCA_ERR_UNSUPPORTED;
  }
  p->kind = kind;
  p->n = n;
  p->k = k;
  p->l = l;
  p->dtype = dtype;
  p->nviews = nviews;
  p->v[0].d = d0;
  p->v[1].d = nviews > 1 ? d1 : 0;
  p->D = d0 + (nviews > 1 ? d1 : 0);
  p->NC = nviews * 2 * k;
  int dmax = std::max(d0, nviews > 1 ? d1 : 0);
  if (p->opt.s == 0) p->s = kind == kCCA ? 4 * (int64_t)(d0 + d1) : 3 * (int64_t)d0;
  else p->s = p->opt.s;
  p->n_pad = next_pow2(n);
  if (p->opt.sketch == GBCCA_SKETCH_SRHT) {
    if (p->s > p->n_pad) p->s = p->n_pad;
  } else if (p->s > n) {
    p->s = n;
  }
  if (p->s < dmax) {
    delete p;
    set_last_error("sketch size s must be >= the number of columns of each view");
    return GBCCA_ERR_INVALID_ARG;
  }
  if (p->opt.sketch == GBCCA_SKETCH_SRHT && p->n_pad > (1ll << 19)) {
    delete p;
    set_last_error("SRHT supports n <= 2^19 rows; use CountSketch for taller data");
    return GBCCA_ERR_UNSUPPORTED;
  }
  GB_CUDA(cudaGetDevice(&p->dev));
  GB_CUDA(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->dev));
  g_alloc_bytes = 0;
  int r = alloc_plan(p);
  p->dev_bytes = g_alloc_bytes;
  if (r != GBCCA_OK) {
    free_plan(p);
    return r;
  }
  *out = reinterpret_cast<gbcca_plan_t>(p);
  return GBCCA_OK;
}

__global__ void identity_kernel(double* A, int d) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < d * d) A[e] = (e / d == e % d) ? 1.0 : 0.0;
}

int read_flag(Plan& p, cudaStream_t st) {
  int f = 0;
  GB_CUDA(cudaMemcpyAsync(&f, p.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  GB_CUDA(cudaStreamSynchronize(st));
  GB_CUDA(cudaMemsetAsync(p.flag, 0, sizeof(int), st));
  return flag_status(f);
}

// Sketch every view, factor the sketch preconditioner and compute the warm
// start; then install the metric factor the options ask for.
// Derived forms of R^{-1} used by the iterations: the FP32 copy and, for
// FP32/BF16 plans, the double-float M^{-1}.
int finish_factor(Plan& p, int v, cudaStream_t st) {
  View& w = p.v[v];
  GB_TRY(to_f32(w.Rinv, w.Rinv32, (int64_t)w.d * w.d, st));
  if (w.Minv_hi != nullptr) GB_TRY(minv_df_build(w.Rinv, w.d, w.Minv_hi, w.Minv_lo, p.ws, p.ws_len, st));
  return GBCCA_OK;
}

int precondition_common(Plan& p, const int32_t* sh, const int8_t* sg, cudaStream_t st) {
  const bool center = p.kind == kLDA;
  GB_TRY(hilo_prepare(p, st));
  const bool srht = p.opt.sketch == GBCCA_SKETCH_SRHT;
  if (srht) {
    if (sh != nullptr && sg != nullptr) {
      GB_CUDA(cudaMemcpyAsync(p.h, sh, sizeof(int32_t) * p.s, cudaMemcpyDeviceToDevice, st));
      GB_CUDA(cudaMemcpyAsync(p.g, sg, sizeof(int8_t) * p.n_pad, cudaMemcpyDeviceToDevice, st));
    } else {
      GB_TRY(sketch_draws(GBCCA_SKETCH_SRHT, p.n_pad, p.s, p.opt.seed, p.h, p.g, st));
    }
    for (int v = 0; v < p.nviews; ++v) GB_TRY(srht_apply(p, v, st));
  } else {
    if (sh != nullptr && sg != nullptr) {
      GB_CUDA(cudaMemcpyAsync(p.h, sh, sizeof(int32_t) * p.n, cudaMemcpyDeviceToDevice, st));
      GB_CUDA(cudaMemcpyAsync(p.g, sg, sizeof(int8_t) * p.n, cudaMemcpyDeviceToDevice, st));
    } else {
      GB_TRY(sketch_draws(GBCCA_SKETCH_COUNTSKETCH, p.n, p.s, p.opt.seed, p.h, p.g, st));
    }
    GB_TRY(countsketch_prepare(p, st));
    for (int v = 0; v < p.nviews; ++v) GB_TRY(countsketch_apply(p, v, center, st));
  }
  for (int v = 0; v < p.nviews; ++v) {
    View& w = p.v[v];
    if (w.SZh != nullptr) {
      // FP32/BF16 data: the Gram only shapes the preconditioner; double-float
      // arithmetic (~2^-44 relative per product) at FP32 instruction rates
      GB_TRY(split_rows(w.SZ, (int)p.s, w.d, w.d, w.SZh, w.SZl, st));
      GB_TRY(gram_df_split(w.SZh, w.SZl, w.d, w.SZh, w.SZl, w.d, p.s, w.d, w.d, w.R, w.lam, p.ws, p.ws_len, st));
    } else {
      GB_TRY(gram_tn(w.SZ, w.d, w.SZ, w.d, p.s, w.d, w.d, w.R, w.lam, p.ws, p.ws_len, st));
    }
  }
  // The views' blocked Cholesky factorizations and triangular inverses touch
  // only their own R, R^{-1}, workspace half (and the error flag) and are
  // latency bound: view 1 runs on the plan's side stream, between a fork and
  // a join event, while view 0 runs on `st`.
  if (p.nviews > 1) {
    const int64_t half = p.ws_len / 2;
    GB_CUDA(cudaEventRecord(p.fork_ev, st));
    GB_CUDA(cudaStreamWaitEvent(p.side_stream, p.fork_ev, 0));
    GB_TRY(cholesky_upper(p.v[1].R, p.v[1].d, p.flag, p.side_stream));
    GB_TRY(tri_inverse_upper(p.v[1].R, p.v[1].Rinv, p.v[1].d, p.ws + half, p.ws_len - half, p.side_stream));
    GB_TRY(cholesky_upper(p.v[0].R, p.v[0].d, p.flag, st));
    GB_TRY(tri_inverse_upper(p.v[0].R, p.v[0].Rinv, p.v[0].d, p.ws, half, st));
    GB_CUDA(cudaEventRecord(p.join_ev, p.side_stream));
    GB_CUDA(cudaStreamWaitEvent(st, p.join_ev, 0));
  } else {
    GB_TRY(cholesky_upper(p.v[0].R, p.v[0].d, p.flag, st));
    GB_TRY(tri_inverse_upper(p.v[0].R, p.v[0].Rinv, p.v[0].d, p.ws, p.ws_len, st));
  }
  GB_TRY(read_flag(p, st));
  for (int v = 0; v < p.nviews; ++v) GB_TRY(finish_factor(p, v, st));
  if (p.opt.warm_start) {
    GB_TRY(warm_start(p, st));
    GB_TRY(read_flag(p, st));
  }
  if (p.opt.sketch == GBCCA_SKETCH_IDENTITY) {
    for (int v = 0; v < p.nviews; ++v) {
      int d = p.v[v].d;
      identity_kernel<<<ceil_div(d * d, 256), 256, 0, st>>>(p.v[v].R, d);
      GB_CHECK_LAUNCH();
      identity_kernel<<<ceil_div(d * d, 256), 256, 0, st>>>(p.v[v].Rinv, d);
      GB_CHECK_LAUNCH();
      GB_TRY(finish_factor(p, v, st));
    }
  } else if (p.opt.sketch == GBCCA_SKETCH_EXACT) {
    if (p.dtype != GBCCA_FP64 || p.kind != kCCA) {
      set_last_error("the exact metric (M = Sigma) is implemented for FP64 CCA plans");
      return GBCCA_ERR_UNSUPPORTED;
    }
    for (int v = 0; v < p.nviews; ++v) {
      View& w = p.v[v];
      GB_TRY(gram_tn((const double*)w.Z, w.ld, (const double*)w.Z, w.ld, p.n, w.d, w.d, w.R, w.lam, p.ws,
                     p.ws_len, st));
      GB_TRY(cholesky_upper(w.R, w.d, p.flag, st));
      GB_TRY(tri_inverse_upper(w.R, w.Rinv, w.d, p.ws, p.ws_len, st));
      GB_TRY(finish_factor(p, v, st));
    }
    GB_TRY(read_flag(p, st));
  }
  p.preconditioned = true;
  return GBCCA_OK;
}

Plan* as_plan(gbcca_plan_t h) { return reinterpret_cast<Plan*>(h); }

}  // namespace

// FDA: bind X and the labels, class statistics, sketch and preconditioner
// (everything of lda_solve before its iterations).
int lda_bind(Plan& p, const void* X, int64_t ldx, const int32_t* labels, double lambda, const int32_t* sketch_h,
             const int8_t* sketch_g, cudaStream_t st) {
  p.v[0].Z = X;
  p.v[0].ld = ldx;
  p.v[0].lam = lambda;
  p.labels = labels;
  p.preconditioned = false;
  GB_TRY(lda_class_stats(p, st));
  {
    const int r = read_flag(p, st);
    if (r == GBCCA_ERR_NOT_SPD) {
      set_last_error("lda_solve: every class needs at least one sample");
      return GBCCA_ERR_INVALID_ARG;
    }
    if (r != GBCCA_OK) return r;
  }
  return precondition_common(p, sketch_h, sketch_g, st);
}

}  // namespace gbcca

using namespace gbcca;

extern "C" {

int gbcca_default_options(gbcca_options* opt) {
  if (opt == nullptr) return GBCCA_ERR_INVALID_ARG;
  std::memset(opt, 0, sizeof(*opt));
  opt->sketch = GBCCA_SKETCH_COUNTSKETCH;
  opt->s = 0;
  opt->seed = 0;
  opt->max_iter = 1000;
  opt->gtol = 1e-8;
  opt->refine = 1;
  opt->warm_start = 1;
  opt->check_every = 8;
  opt->graphs = 1;
  opt->tensor_cores = 1;
  return GBCCA_OK;
}

int cca_plan(gbcca_plan_t* plan, int64_t n, int32_t dx, int32_t dy, int32_t k, int32_t dtype,
             const gbcca_options* opt) {
  if (n < 1 || dx < 1 || dy < 1 || k < 1 || k > kMaxK || k > dx || k > dy || dx > kMaxD || dy > kMaxD ||
      n < std::max(dx, dy)) {
    set_last_error("cca_plan: need 1 <= k <= min(dx, dy, 20), dx, dy <= 1024, n >= max(dx, dy)");
    return GBCCA_ERR_INVALID_ARG;
  }
  return make_plan(plan, kCCA, n, dx, dy, 2, k, 0, dtype, opt);
}

int lda_plan(gbcca_plan_t* plan, int64_t n, int32_t d, int32_t n_classes, int32_t k, int32_t dtype,
             const gbcca_options* opt) {
  if (n < 1 || d < 1 || d > kMaxD || n_classes < 2 || n_classes > kMaxClasses || k < 1 || k > kMaxK ||
      k > n_classes - 1 || k > d || n < d) {
    set_last_error("lda_plan: need 2 <= classes <= 64, 1 <= k <= min(classes - 1, d, 20), d <= 1024, n >= d");
    return GBCCA_ERR_INVALID_ARG;
  }
  return make_plan(plan, kLDA, n, d, 0, 1, k, n_classes, dtype, opt);
}

int cca_precondition(gbcca_plan_t plan, const void* X, int64_t ldx, const void* Y, int64_t ldy, double lambda_x,
                     double lambda_y, const int32_t* sketch_h, const int8_t* sketch_g, void* stream) {
  Plan* p = as_plan(plan);
  if (p == nullptr || p->kind != kCCA || X == nullptr || Y == nullptr || ldx < p->v[0].d || ldy < p->v[1].d ||
      !(lambda_x >= 0) || !(lambda_y >= 0)) {
    set_last_error("cca_precondition: bad plan, pointer, leading dimension or lambda");
    return GBCCA_ERR_INVALID_ARG;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  p->v[0].Z = X;
  p->v[0].ld = ldx;
  p->v[0].lam = lambda_x;
  p->v[1].Z = Y;
  p->v[1].ld = ldy;
  p->v[1].lam = lambda_y;
  p->preconditioned = false;
  return precondition_common(*p, sketch_h, sketch_g, st);
}

int cca_solve(gbcca_plan_t plan, const double* mu, double tol, double* U, double* V, double* sigma,
              gbcca_info* info, void* stream) {
  Plan* p = as_plan(plan);
  if (p == nullptr || p->kind != kCCA || U == nullptr || V == nullptr || sigma == nullptr) {
    set_last_error("cca_solve: bad plan or output pointer");
    return GBCCA_ERR_INVALID_ARG;
  }
  if (!p->preconditioned) {
    set_last_error("cca_solve before cca_precondition");
    return GBCCA_ERR_STATE;
  }
  if (mu != nullptr)
    for (int i = 0; i < p->k; ++i)
      if (!(mu[i] > 0) || (i > 0 && !(mu[i] < mu[i - 1]))) {
        set_last_error("mu must be positive and strictly decreasing");
        return GBCCA_ERR_INVALID_ARG;
      }
  return rcg_run(*p, mu, tol, U, V, sigma, info, reinterpret_cast<cudaStream_t>(stream));
}

int lda_solve(gbcca_plan_t plan, const void* X, int64_t ldx, const int32_t* labels, double lambda, const double* mu,
              double tol, const int32_t* sketch_h, const int8_t* sketch_g, double* W, double* rho, gbcca_info* info,
              void* stream) {
  Plan* p = as_plan(plan);
  if (p == nullptr || p->kind != kLDA || X == nullptr || labels == nullptr || W == nullptr || rho == nullptr ||
      ldx < p->v[0].d || !(lambda >= 0)) {
    set_last_error("lda_solve: bad plan, pointer, leading dimension or lambda");
    return GBCCA_ERR_INVALID_ARG;
  }
  if (mu != nullptr)
    for (int i = 0; i < p->k; ++i)
      if (!(mu[i] > 0) || (i > 0 && !(mu[i] < mu[i - 1]))) {
        set_last_error("mu must be positive and strictly decreasing");
        return GBCCA_ERR_INVALID_ARG;
      }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  GB_TRY(lda_bind(*p, X, ldx, labels, lambda, sketch_h, sketch_g, st));
  return rcg_run(*p, mu, tol, W, nullptr, rho, info, st);
}

__global__ void scatter_rows_kernel(const double* G, int NC, int row0, int d, double* out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < d * NC) out[e] = G[(int64_t)row0 * NC + e];
}

int gbcca_fused_pass(gbcca_plan_t plan, const double* Phi_x, const double* Phi_y, double* Gx, double* Gy,
                     double* Gram, void* stream) {
  Plan* p = as_plan(plan);
  if (p == nullptr || Phi_x == nullptr || Gx == nullptr || Gram == nullptr ||
      (p->kind == kCCA && (Phi_y == nullptr || Gy == nullptr))) {
    set_last_error("gbcca_fused_pass: bad plan or pointer");
    return GBCCA_ERR_INVALID_ARG;
  }
  if (p->v[0].Z == nullptr || (p->kind == kLDA && p->labels == nullptr)) {
    set_last_error("gbcca_fused_pass: the plan has no data yet");
    return GBCCA_ERR_STATE;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int k2 = 2 * p->k;
  GB_CUDA(cudaMemcpyAsync(p->v[0].Phi, Phi_x, sizeof(double) * p->v[0].d * k2, cudaMemcpyDeviceToDevice, st));
  if (p->kind == kCCA)
    GB_CUDA(cudaMemcpyAsync(p->v[1].Phi, Phi_y, sizeof(double) * p->v[1].d * k2, cudaMemcpyDeviceToDevice, st));
  GB_TRY(fused_pass(*p, p->dtype != GBCCA_FP64, false, st, 0, nullptr));
  scatter_rows_kernel<<<ceil_div(p->v[0].d * p->NC, 256), 256, 0, st>>>(p->G, p->NC, 0, p->v[0].d, Gx);
  GB_CHECK_LAUNCH();
  if (p->kind == kCCA) {
    scatter_rows_kernel<<<ceil_div(p->v[1].d * p->NC, 256), 256, 0, st>>>(p->G, p->NC, p->v[0].d, p->v[1].d, Gy);
    GB_CHECK_LAUNCH();
  }
  GB_CUDA(cudaMemcpyAsync(Gram, p->Gram, sizeof(double) * p->NC * p->NC, cudaMemcpyDeviceToDevice, st));
  return GBCCA_OK;
}

int64_t gbcca_query_size(gbcca_plan_t plan, int32_t what) {
  Plan* p = as_plan(plan);
  if (p == nullptr) return -1;
  switch (what) {
    case GBCCA_Q_SKETCH_X: return p->s * p->v[0].d;
    case GBCCA_Q_SKETCH_Y: return p->kind == kCCA ? p->s * p->v[1].d : -1;
    case GBCCA_Q_R_X: return (int64_t)p->v[0].d * p->v[0].d;
    case GBCCA_Q_R_Y: return p->kind == kCCA ? (int64_t)p->v[1].d * p->v[1].d : -1;
    case GBCCA_Q_WARM_U: return (int64_t)p->v[0].d * p->k;
    case GBCCA_Q_WARM_V: return p->kind == kCCA ? (int64_t)p->v[1].d * p->k : -1;
    case GBCCA_Q_HISTORY: return 3 * (int64_t)(p->opt.max_iter + 1);
    case GBCCA_Q_CLASS_MEANS: return p->kind == kLDA ? (int64_t)p->l * p->v[0].d : -1;
    case GBCCA_Q_RITZ: return (int64_t)p->ritz_len * p->k;
  }
  return -1;
}

int gbcca_query(gbcca_plan_t plan, int32_t what, double* dst, void* stream) {
  Plan* p = as_plan(plan);
  int64_t n = gbcca_query_size(plan, what);
  if (p == nullptr || dst == nullptr || n < 0) {
    set_last_error("gbcca_query: bad plan, pointer or query");
    return GBCCA_ERR_INVALID_ARG;
  }
  const double* src = nullptr;
  switch (what) {
    case GBCCA_Q_SKETCH_X: src = p->v[0].SZ; break;
    case GBCCA_Q_SKETCH_Y: src = p->v[1].SZ; break;
    case GBCCA_Q_R_X: src = p->v[0].R; break;
    case GBCCA_Q_R_Y: src = p->v[1].R; break;
    case GBCCA_Q_WARM_U: src = p->v[0].warm; break;
    case GBCCA_Q_WARM_V: src = p->v[1].warm; break;
    case GBCCA_Q_HISTORY: src = p->history; break;
    case GBCCA_Q_CLASS_MEANS: src = p->means; break;
    case GBCCA_Q_RITZ: src = p->ritz_hist; break;
  }
  GB_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                          reinterpret_cast<cudaStream_t>(stream)));
  return GBCCA_OK;
}

int gbcca_sketch_draws(int32_t kind, int64_t n, int64_t s, uint64_t seed, int32_t* h, int8_t* g, void* stream) {
  if (h == nullptr || g == nullptr || n < 1 || s < 1) {
    set_last_error("gbcca_sketch_draws: bad pointer or size");
    return GBCCA_ERR_INVALID_ARG;
  }
  return sketch_draws(kind, n, s, seed, h, g, reinterpret_cast<cudaStream_t>(stream));
}

int gbcca_sketch_gram_noalloc(const double* A, int64_t lda, int64_t m, int32_t d, double lambda, double* C,
                              void* stream) {
  if (A == nullptr || C == nullptr || m < 1 || d < 1 || lda < d || !(lambda >= 0.0)) {
    set_last_error("gbcca_sketch_gram_noalloc: bad pointer, size or lambda");
    return GBCCA_ERR_INVALID_ARG;
  }
  return gram_noalloc(A, lda, m, d, lambda, C, reinterpret_cast<cudaStream_t>(stream));
}

int32_t gbcca_sketch_gram_noalloc_max_d(void) { return noalloc_max_d(); }

int64_t gbcca_launch_count(void) { return (int64_t)g_launches.load(); }

void gbcca_plan_destroy(gbcca_plan_t plan) { free_plan(as_plan(plan)); }

const char* gbcca_status_string(int status) {
  switch (status) {
    case GBCCA_OK: return "ok";
    case GBCCA_ERR_INVALID_ARG: return "invalid argument";
    case GBCCA_ERR_UNSUPPORTED: return "unsupported";
    case GBCCA_ERR_OOM: return "out of device memory";
    case GBCCA_ERR_NOT_SPD: return "matrix not positive definite";
    case GBCCA_ERR_MAXITER: return "iteration limit reached";
    case GBCCA_ERR_TIMEOUT: return "device wait timed out";
    case GBCCA_ERR_CUDA: return "CUDA error";
    case GBCCA_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* gbcca_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
