// Batched solves: several prepared plans (CCA or FDA, each bound to its data)
// iterate in lockstep, and every iteration's data passes of the plans the
// tensor-core pass serves run as ONE persistent launch over a schedule of
// (instance, 64-row tile range) segments (Alg. 1 / Alg. 2 per instance; the
// per-iteration cost of each is Cor. 4.6 / Cor. 5.6).  Around that launch,
// each plan's own kernels (Phi image before; reduction, Gram and the small
// geometry of Table 1 after) run on a branch of their own, so the plans'
// latency-bound chains overlap one another.  Batches of iterations replay a
// captured CUDA graph; plans that finish leave the schedule (the kernels of
// a finished plan return at once), and the graph is captured again once the
// active set has shrunk by a quarter.
//
// The number of 2-CTA clusters of the batched launch is tuned once per batch
// object: each candidate is timed with events on the plans' start points
// (the pass only reads the data and the Phi images and writes partials, so
// the trials change no state), and the fastest is kept.
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "plan.h"

namespace gbcca {

// Two batched launches serve the tensor-core plans: table 0 in 2-CTA
// clusters, table 1 in 4-CTA clusters (plans with a view wider than 512).
struct Batch {
  std::vector<Plan*> plans;
  std::vector<int> tc_table;       // 0 or 1: the table that serves the plan's pass; -1: its own pass
  std::vector<int> tc_index;       // index in that table
  std::vector<Plan*> tc_plans[2];
  TcBatch* tc[2] = {nullptr, nullptr};
  gbcca_batch_options opt{};
  int clusters[2] = {0, 0};        // chosen clusters of each batched launch
  bool tuned = false;
  double tune_ms = 0;              // batched pass time of the chosen schedules (all plans active)
  int64_t tune_bytes = 0;
  cudaStream_t cap = nullptr;      // capture stream
  std::vector<cudaStream_t> side;  // one branch stream per plan
  cudaEvent_t fork_a = nullptr, fork_b = nullptr;
  std::vector<cudaEvent_t> join_a, join_b;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaGraphExec_t exec = nullptr;
  int exec_n = 0;                  // iterations per replay
  int exec_active = 0;             // active plans when captured
  std::vector<char> exec_mask;     // active set of the capture
  long long exec_launches = 0;
};

namespace {

Batch* as_batch(gbcca_batch_t h) { return reinterpret_cast<Batch*>(h); }

void destroy(Batch* b) {
  if (b == nullptr) return;
  if (b->exec != nullptr) cudaGraphExecDestroy(b->exec);
  tc_batch_destroy(b->tc[0]);
  tc_batch_destroy(b->tc[1]);
  for (cudaStream_t s : b->side)
    if (s != nullptr) cudaStreamDestroy(s);
  if (b->cap != nullptr) cudaStreamDestroy(b->cap);
  for (cudaEvent_t e : b->join_a)
    if (e != nullptr) cudaEventDestroy(e);
  for (cudaEvent_t e : b->join_b)
    if (e != nullptr) cudaEventDestroy(e);
  for (cudaEvent_t e : {b->fork_a, b->fork_b, b->ev0, b->ev1})
    if (e != nullptr) cudaEventDestroy(e);
  delete b;
}

// One lockstep iteration of the active plans, enqueued on `st` (a capturing
// stream or a live one): branch i waits for the fork, the tensor-core plans
// make their Phi images and join before the batched launch, then fork again
// for their reductions and small kernels; the other plans run their whole
// iteration on their branch.  `st` ends after every branch.
int enqueue_iteration(Batch& b, const std::vector<char>& active, cudaStream_t st) {
  const int n = (int)b.plans.size();
  GB_CUDA(cudaEventRecord(b.fork_a, st));
  bool any_tc = false;
  for (int i = 0; i < n; ++i) {
    if (!active[i]) continue;
    Plan& p = *b.plans[i];
    const bool low = p.dtype != GBCCA_FP64;
    GB_CUDA(cudaStreamWaitEvent(b.side[i], b.fork_a, 0));
    if (b.tc_table[i] >= 0) {
      GB_TRY(tc_batch_pre(b.tc[b.tc_table[i]], p, b.side[i]));
      any_tc = true;
    } else {
      GB_TRY(fused_pass(p, low, false, b.side[i], 0, &p.st->done));
      GB_TRY(iteration_post(p, low, b.side[i]));
    }
    GB_CUDA(cudaEventRecord(b.join_a[i], b.side[i]));
  }
  if (any_tc) {
    for (int i = 0; i < n; ++i)
      if (active[i] && b.tc_table[i] >= 0) GB_CUDA(cudaStreamWaitEvent(st, b.join_a[i], 0));
    for (int t = 0; t < 2; ++t)
      if (b.tc[t] != nullptr) GB_TRY(tc_batch_launch(b.tc[t], st, nullptr, nullptr));
    GB_CUDA(cudaEventRecord(b.fork_b, st));
    for (int i = 0; i < n; ++i) {
      if (!active[i] || b.tc_table[i] < 0) continue;
      Plan& p = *b.plans[i];
      GB_CUDA(cudaStreamWaitEvent(b.side[i], b.fork_b, 0));
      GB_TRY(tc_batch_post(b.tc[b.tc_table[i]], b.tc_index[i], p, b.side[i], &p.st->done));
      GB_TRY(iteration_post(p, p.dtype != GBCCA_FP64, b.side[i]));
      GB_CUDA(cudaEventRecord(b.join_b[i], b.side[i]));
    }
  }
  for (int i = 0; i < n; ++i) {
    if (!active[i]) continue;
    GB_CUDA(cudaStreamWaitEvent(st, b.tc_table[i] >= 0 ? b.join_b[i] : b.join_a[i], 0));
  }
  return GBCCA_OK;
}

int replay(Batch& b, const std::vector<char>& active, int nb, cudaStream_t st) {
  int na = 0;
  for (char a : active) na += a ? 1 : 0;
  // the captured graph serves every plan active now, and not too many that
  // have finished since
  bool covered = b.exec != nullptr && b.exec_n == nb && 4 * na > 3 * b.exec_active;
  for (size_t i = 0; covered && i < active.size(); ++i) covered = !active[i] || b.exec_mask[i];
  const bool same = covered;
  if (!same) {
    if (b.exec != nullptr) {
      GB_CUDA(cudaGraphExecDestroy(b.exec));
      b.exec = nullptr;
    }
    const long long l0 = g_launches.load();
    GB_CUDA(cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeRelaxed));
    int rc = GBCCA_OK;
    for (int it = 0; it < nb && rc == GBCCA_OK; ++it) rc = enqueue_iteration(b, active, b.cap);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b.cap, &g);
    if (rc != GBCCA_OK || ec != cudaSuccess) {
      if (g != nullptr) cudaGraphDestroy(g);
      g_launches.fetch_sub(g_launches.load() - l0);
      cudaGetLastError();
      if (rc != GBCCA_OK) return rc;
      set_last_error(std::string("capture of the batched iterations: ") + cudaGetErrorString(ec));
      return GBCCA_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&b.exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      b.exec = nullptr;
      cudaGetLastError();
      set_last_error(std::string("instantiation of the batched iterations: ") + cudaGetErrorString(ei));
      return GBCCA_ERR_CUDA;
    }
    b.exec_launches = g_launches.load() - l0;
    g_launches.fetch_sub(b.exec_launches);
    b.exec_n = nb;
    b.exec_active = na;
    b.exec_mask = active;
  }
  // the captured graph serves the plans active at capture time; plans that
  // finished since return at once inside it
  GB_CUDA(cudaGraphLaunch(b.exec, st));
  g_launches.fetch_add(b.exec_launches);
  return GBCCA_OK;
}

// Time batched launch t over all its plans for `clusters` clusters: one warm
// launch, then the median of three.
int time_schedule(Batch& b, int t, int clusters, cudaStream_t st, double* ms) {
  const size_t m = b.tc_plans[t].size();
  std::unique_ptr<bool[]> a(new bool[std::max<size_t>(m, 1)]);
  for (size_t i = 0; i < m; ++i) a[i] = true;
  GB_TRY(tc_batch_schedule(b.tc[t], a.get(), clusters, st));
  GB_TRY(tc_batch_launch(b.tc[t], st, nullptr, nullptr));
  float tm[3];
  for (int r = 0; r < 3; ++r) {
    GB_TRY(tc_batch_launch(b.tc[t], st, b.ev0, b.ev1));
    GB_CUDA(cudaEventSynchronize(b.ev1));
    GB_CUDA(cudaEventElapsedTime(&tm[r], b.ev0, b.ev1));
  }
  std::sort(tm, tm + 3);
  *ms = tm[1];
  return GBCCA_OK;
}

// Each batched launch's cluster count: the option's, else the fastest of a
// few candidates timed on the plans' start points.
int autotune(Batch& b, cudaStream_t st) {
  b.tune_ms = 0;
  b.tune_bytes = 0;
  for (int t = 0; t < 2; ++t) {
    if (b.tc[t] == nullptr) continue;
    const int maxc = tc_batch_max_clusters(b.tc[t]);
    std::vector<int> cand;
    if (b.opt.clusters > 0) {
      cand.push_back(std::min(b.opt.clusters, maxc));
    } else {
      for (int c : {maxc, maxc - 2, maxc - 4, (3 * maxc) / 4, maxc / 2})
        if (c >= 1 && std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
    }
    double best = 1e300;
    int best_c = cand[0];
    for (int c : cand) {
      double ms = 0;
      GB_TRY(time_schedule(b, t, c, st, &ms));
      if (ms < best) {
        best = ms;
        best_c = c;
      }
    }
    // the device error flag of the batched kernel must be clear after the trials
    int err = 0;
    GB_CUDA(cudaMemcpyAsync(&err, tc_batch_err(b.tc[t]), sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (err != 0) {
      GB_CUDA(cudaMemsetAsync(tc_batch_err(b.tc[t]), 0, sizeof(int), st));
      return flag_status(err);
    }
    b.clusters[t] = best_c;
    b.tune_ms += best;
    std::unique_ptr<bool[]> a(new bool[std::max<size_t>(b.tc_plans[t].size(), 1)]);
    for (size_t i = 0; i < b.tc_plans[t].size(); ++i) a[i] = true;
    b.tune_bytes += tc_batch_bytes(b.tc[t], a.get());
  }
  b.tuned = true;
  return GBCCA_OK;
}

}  // namespace

Batch* batch_make(Plan* const* plans, int count, const gbcca_batch_options* opt, int* rc) {
  *rc = GBCCA_OK;
  auto* b = new (std::nothrow) Batch();
  if (b == nullptr) {
    *rc = GBCCA_ERR_OOM;
    return nullptr;
  }
  gbcca_default_batch_options(&b->opt);
  if (opt != nullptr) b->opt = *opt;
  for (int i = 0; i < count; ++i) {
    Plan* p = plans[i];
    b->plans.push_back(p);
    const bool tc = p->kind == kCCA && p->dtype != GBCCA_FP64 && p->opt.tensor_cores && p->tc_img != nullptr &&
                    tc_pass_eligible(*p);
    const int t = tc ? (tc_quad(*p) ? 1 : 0) : -1;
    b->tc_table.push_back(t);
    b->tc_index.push_back(t >= 0 ? (int)b->tc_plans[t].size() : -1);
    if (t >= 0) b->tc_plans[t].push_back(p);
  }
  auto fail = [&](cudaError_t e) {
    set_last_error(std::string("batch: ") + cudaGetErrorString(e));
    cudaGetLastError();
    destroy(b);
    *rc = GBCCA_ERR_CUDA;
    return nullptr;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(e);
  b->side.assign(count, nullptr);
  b->join_a.assign(count, nullptr);
  b->join_b.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    if ((e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreateWithFlags(&b->join_a[i], cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreateWithFlags(&b->join_b[i], cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  }
  if ((e = cudaEventCreateWithFlags(&b->fork_a, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  if ((e = cudaEventCreateWithFlags(&b->fork_b, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  if ((e = cudaEventCreate(&b->ev0)) != cudaSuccess) return fail(e);
  if ((e = cudaEventCreate(&b->ev1)) != cudaSuccess) return fail(e);
  for (int t = 0; t < 2; ++t) {
    if (b->tc_plans[t].empty()) continue;
    b->tc[t] = tc_batch_create(b->tc_plans[t].data(), (int)b->tc_plans[t].size(), b->cap, rc);
    if (b->tc[t] == nullptr) {
      destroy(b);
      return nullptr;
    }
    b->clusters[t] = b->opt.clusters > 0 ? std::min(b->opt.clusters, tc_batch_max_clusters(b->tc[t]))
                                         : tc_batch_max_clusters(b->tc[t]);
  }
  return b;
}

void batch_free(Batch* b) { destroy(b); }

int batch_size(const Batch& b) { return (int)b.plans.size(); }

// nb lockstep iterations of the active plans (a captured graph when asked
// and nb is the batch's replay length, else launched one by one), after
// writing the schedule of the active tensor-core plans.
int batch_iterate(Batch& b, const std::vector<char>& active, int nb, bool graph, cudaStream_t st) {
  for (int t = 0; t < 2; ++t) {
    if (b.tc[t] == nullptr) continue;
    std::unique_ptr<bool[]> a(new bool[std::max<size_t>(b.tc_plans[t].size(), 1)]);
    for (size_t i = 0; i < b.plans.size(); ++i)
      if (b.tc_table[i] == t) a[b.tc_index[i]] = active[i] != 0;
    GB_TRY(tc_batch_schedule(b.tc[t], a.get(), b.clusters[t], st));
  }
  if (graph) return replay(b, active, nb, st);
  for (int it = 0; it < nb; ++it) GB_TRY(enqueue_iteration(b, active, st));
  return GBCCA_OK;
}

// After iterations: reads every active plan's state (synchronizing `st`),
// returns the first device-reported failure, and clears active[i] for the
// plans that finished.  err_plan (may be NULL) gets the index of a plan
// whose own flag reported an error, else -1.
int batch_poll(Batch& b, std::vector<char>& active, gbcca_info* infos, cudaStream_t st, int* err_plan) {
  const int n = (int)b.plans.size();
  if (err_plan != nullptr) *err_plan = -1;
  for (int i = 0; i < n; ++i)
    if (active[i]) GB_TRY(read_state_async(*b.plans[i], st));
  int tc_err[2] = {0, 0};
  for (int t = 0; t < 2; ++t)
    if (b.tc[t] != nullptr)
      GB_CUDA(cudaMemcpyAsync(&tc_err[t], tc_batch_err(b.tc[t]), sizeof(int), cudaMemcpyDeviceToHost, st));
  GB_CUDA(cudaStreamSynchronize(st));
  for (int t = 0; t < 2; ++t) {
    if (tc_err[t] == 0) continue;
    GB_CUDA(cudaMemsetAsync(tc_batch_err(b.tc[t]), 0, sizeof(int), st));
    GB_CUDA(cudaStreamSynchronize(st));
    set_last_error("batched tensor-core pass: a bounded pipeline wait ran out");
    return flag_status(tc_err[t]);
  }
  for (int i = 0; i < n; ++i) {
    if (!active[i]) continue;
    Plan& p = *b.plans[i];
    const int rc = check_flag(p, infos != nullptr ? &infos[i] : nullptr, st);
    if (rc != GBCCA_OK) {
      if (err_plan != nullptr) *err_plan = i;
      return rc;
    }
    if (p.st_host->done) active[i] = 0;
  }
  return GBCCA_OK;
}

int batch_tune(Batch& b, cudaStream_t st) {
  if ((b.tc[0] == nullptr && b.tc[1] == nullptr) || b.tuned) return GBCCA_OK;
  for (int t = 0; t < 2; ++t)
    for (Plan* p : b.tc_plans[t]) GB_TRY(tc_batch_pre(b.tc[t], *p, st));
  return autotune(b, st);
}

}  // namespace gbcca

using namespace gbcca;

extern "C" {

int gbcca_default_batch_options(gbcca_batch_options* opt) {
  if (opt == nullptr) return GBCCA_ERR_INVALID_ARG;
  std::memset(opt, 0, sizeof(*opt));
  opt->clusters = 0;
  opt->graphs = 1;
  opt->batch_iters = 8;
  return GBCCA_OK;
}

int gbcca_batch_create(gbcca_batch_t* out, const gbcca_plan_t* plans, int32_t count,
                       const gbcca_batch_options* opt) {
  if (out == nullptr || plans == nullptr || count < 1 || count > kMaxBatch) {
    set_last_error("gbcca_batch_create: need 1 <= count <= 1024 plans");
    return GBCCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (opt != nullptr && (opt->clusters < 0 || opt->batch_iters < 1)) {
    set_last_error("gbcca_batch_create: invalid options");
    return GBCCA_ERR_INVALID_ARG;
  }
  std::vector<Plan*> ps;
  for (int i = 0; i < count; ++i) {
    Plan* p = reinterpret_cast<Plan*>(plans[i]);
    if (p == nullptr || !p->preconditioned || !p->opt.warm_start) {
      set_last_error("gbcca_batch_create: every plan must be preconditioned (bound to its data) with warm_start on");
      return GBCCA_ERR_STATE;
    }
    if (std::find(ps.begin(), ps.end(), p) != ps.end()) {
      set_last_error("gbcca_batch_create: a plan appears twice");
      return GBCCA_ERR_INVALID_ARG;
    }
    ps.push_back(p);
  }
  int rc = GBCCA_OK;
  Batch* b = batch_make(ps.data(), count, opt, &rc);
  if (b == nullptr) return rc;
  *out = reinterpret_cast<gbcca_batch_t>(b);
  return GBCCA_OK;
}

int gbcca_batch_solve(gbcca_batch_t h, double* const* U, double* const* V, double* const* vals, gbcca_info* infos,
                      gbcca_batch_report* report, void* stream) {
  Batch* b = as_batch(h);
  if (b == nullptr || U == nullptr || vals == nullptr) {
    set_last_error("gbcca_batch_solve: NULL argument");
    return GBCCA_ERR_INVALID_ARG;
  }
  const int n = (int)b->plans.size();
  for (int i = 0; i < n; ++i) {
    if (U[i] == nullptr || vals[i] == nullptr || (b->plans[i]->kind == kCCA && (V == nullptr || V[i] == nullptr))) {
      set_last_error("gbcca_batch_solve: NULL output pointer");
      return GBCCA_ERR_INVALID_ARG;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n; ++i) GB_TRY(rcg_begin(*b->plans[i], nullptr, 0.0, nullptr, nullptr, st));
  GB_TRY(batch_tune(*b, st));
  std::vector<char> active(n, 1);
  int max_iter = 0;
  for (Plan* p : b->plans) max_iter = std::max(max_iter, p->opt.max_iter);
  const int nb = b->opt.batch_iters;
  int launched = -1;  // the first iteration is the qf_B step
  int lockstep = 0;
  bool first = true;
  while (true) {
    const int m = first ? 1 : std::min(nb, max_iter - launched);
    GB_TRY(batch_iterate(*b, active, m, b->opt.graphs && !first && m == nb, st));
    launched += m;
    lockstep += m;
    first = false;
    GB_TRY(batch_poll(*b, active, infos, st, nullptr));
    int running = 0;
    for (int i = 0; i < n; ++i) {
      if (launched >= b->plans[i]->opt.max_iter) active[i] = 0;
      running += active[i] ? 1 : 0;
    }
    if (running == 0 || launched >= max_iter) break;
  }
  int status = GBCCA_OK;
  for (int i = 0; i < n; ++i) {
    Plan& p = *b->plans[i];
    const int rc = rcg_finish(p, U[i], p.kind == kCCA ? V[i] : nullptr, vals[i], infos != nullptr ? &infos[i] : nullptr,
                              0.0, 0, st);
    if (rc != GBCCA_OK && status == GBCCA_OK) status = rc;
    if (rc != GBCCA_OK && rc != GBCCA_ERR_MAXITER) return rc;
  }
  if (report != nullptr) {
    std::memset(report, 0, sizeof(*report));
    report->iterations = lockstep;
    report->clusters = b->clusters[0] > 0 ? b->clusters[0] : b->clusters[1];
    report->batched_plans = (int32_t)(b->tc_plans[0].size() + b->tc_plans[1].size());
    report->batched_pass_ms = b->tune_ms;
    report->batched_pass_bytes = (double)b->tune_bytes;
  }
  return status;
}

int gbcca_batch_fused_pass(gbcca_batch_t h, const double* const* Phi_x, const double* const* Phi_y, double* const* G,
                           double* const* Gram, void* stream) {
  Batch* b = as_batch(h);
  if (b == nullptr || Phi_x == nullptr || Phi_y == nullptr || G == nullptr || Gram == nullptr) {
    set_last_error("gbcca_batch_fused_pass: NULL argument");
    return GBCCA_ERR_INVALID_ARG;
  }
  const int n = (int)b->plans.size();
  if (b->tc_plans[0].size() + b->tc_plans[1].size() != (size_t)n) {
    set_last_error("gbcca_batch_fused_pass: every plan of the batch must be served by the tensor-core pass");
    return GBCCA_ERR_UNSUPPORTED;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n; ++i) {
    Plan& p = *b->plans[i];
    const int k2 = 2 * p.k;
    GB_CUDA(cudaMemsetAsync(&p.st->done, 0, sizeof(int), st));
    GB_CUDA(cudaMemcpyAsync(p.v[0].Phi, Phi_x[i], sizeof(double) * p.v[0].d * k2, cudaMemcpyDeviceToDevice, st));
    GB_CUDA(cudaMemcpyAsync(p.v[1].Phi, Phi_y[i], sizeof(double) * p.v[1].d * k2, cudaMemcpyDeviceToDevice, st));
    GB_TRY(tc_batch_pre(b->tc[b->tc_table[i]], p, st));
  }
  for (int t = 0; t < 2; ++t) {
    if (b->tc[t] == nullptr) continue;
    const int m = (int)b->tc_plans[t].size();
    std::unique_ptr<bool[]> a(new bool[std::max(m, 1)]);
    for (int i = 0; i < m; ++i) a[i] = true;
    GB_TRY(tc_batch_schedule(b->tc[t], a.get(),
                             b->opt.clusters > 0 ? b->opt.clusters : tc_batch_max_clusters(b->tc[t]), st));
    GB_TRY(tc_batch_launch(b->tc[t], st, nullptr, nullptr));
  }
  for (int i = 0; i < n; ++i) {
    Plan& p = *b->plans[i];
    GB_TRY(tc_batch_post(b->tc[b->tc_table[i]], b->tc_index[i], p, st, nullptr));
    const int k4 = 4 * p.k;
    GB_CUDA(cudaMemcpyAsync(G[i], p.G, sizeof(double) * p.D * k4, cudaMemcpyDeviceToDevice, st));
    GB_CUDA(cudaMemcpyAsync(Gram[i], p.Gram, sizeof(double) * k4 * k4, cudaMemcpyDeviceToDevice, st));
  }
  int err[2] = {0, 0};
  for (int t = 0; t < 2; ++t)
    if (b->tc[t] != nullptr)
      GB_CUDA(cudaMemcpyAsync(&err[t], tc_batch_err(b->tc[t]), sizeof(int), cudaMemcpyDeviceToHost, st));
  GB_CUDA(cudaStreamSynchronize(st));
  for (int t = 0; t < 2; ++t) {
    if (err[t] == 0) continue;
    GB_CUDA(cudaMemsetAsync(tc_batch_err(b->tc[t]), 0, sizeof(int), st));
    return flag_status(err[t]);
  }
  return GBCCA_OK;
}

void gbcca_batch_destroy(gbcca_batch_t h) { destroy(as_batch(h)); }

}  // extern "C"
