// Serving loop: solves that arrive over time share the GPU.  Each request
// (a CCA or FDA problem with its data anywhere the GPU can read) waits in a
// FIFO queue until the device memory it needs fits the server's budget; at
// admission its data are copied into device buffers the server owns (rows
// padded to 16 bytes, so every BF16 plan can take the tensor-core pass), its
// plan is made and preconditioned, and its iteration state set up (Alg. 1 /
// Alg. 2 steps 1-5).  Every tick advances all running requests by a few
// lockstep iterations through the batch executor (one persistent
// tensor-core launch per iteration for the plans it serves, the other plans'
// passes and every plan's small kernels on graph branches of their own);
// requests that finish are refined, their outputs kept, and their memory
// returned to the budget, so waiting requests join the next tick
// (continuous batching).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "plan.h"

namespace gbcca {
namespace {

enum { kQueued = 0, kRunning = 1, kFinished = 2, kFailed = 3 };

struct Req {
  gbcca_request r{};
  int state = kQueued;
  int status = GBCCA_OK;
  Plan* plan = nullptr;
  void* X = nullptr;
  void* Y = nullptr;
  int32_t* labels = nullptr;
  double* out = nullptr;   // U | V | values (device), kept until fetched
  int64_t bytes = 0;       // device bytes held while running
  int64_t held = 0;        // the same, kept for the report
  gbcca_info info{};
  double t_submit = 0, t_admit = 0, t_finish = 0;
};

struct Server {
  gbcca_server_options opt{};
  std::chrono::steady_clock::time_point t0;
  int64_t used = 0;
  int64_t next_id = 1;
  std::deque<int64_t> queue;
  std::vector<int64_t> running;
  std::unordered_map<int64_t, Req> reqs;
  Batch* batch = nullptr;
  std::vector<int64_t> batch_ids;  // running requests the batch was made for
  bool stable = false;             // the batch served the previous tick unchanged
};

double now_s(const Server& s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s.t0).count();
}

int elt_size(int dtype) { return dtype == GBCCA_BF16 ? 2 : (dtype == GBCCA_FP32 ? 4 : 8); }
int64_t padded_ld(int d, int dtype) {
  const int per16 = 16 / elt_size(dtype);
  return (int64_t)(d + per16 - 1) / per16 * per16;
}

void release(Req& q) {
  if (q.plan != nullptr) gbcca_plan_destroy(reinterpret_cast<gbcca_plan_t>(q.plan));
  q.plan = nullptr;
  for (void* p : {q.X, q.Y, (void*)q.labels})
    if (p != nullptr) cudaFree(p);
  q.X = q.Y = nullptr;
  q.labels = nullptr;
}

// Makes the request's plan and device copies; *bytes = the device memory
// they take (the plan's allocations, the copies and the outputs, counted as
// requested).  On failure everything made is released.
int materialize(Req& q, cudaStream_t st, int64_t* bytes) {
  const gbcca_request& r = q.r;
  (void)st;
  gbcca_options o = r.opt;
  o.warm_start = 1;
  gbcca_plan_t h = nullptr;
  int rc = r.kind == kCCA ? cca_plan(&h, r.n, r.dx, r.dy, r.k, r.dtype, &o)
                          : lda_plan(&h, r.n, r.dx, r.n_classes, r.k, r.dtype, &o);
  if (rc != GBCCA_OK) return rc;
  q.plan = reinterpret_cast<Plan*>(h);
  const int es = elt_size(r.dtype);
  const int64_t lx = padded_ld(r.dx, r.dtype);
  const int64_t ly = r.kind == kCCA ? padded_ld(r.dy, r.dtype) : 0;
  cudaError_t e = cudaMalloc(&q.X, (size_t)r.n * lx * es);
  if (e == cudaSuccess && r.kind == kCCA) e = cudaMalloc(&q.Y, (size_t)r.n * ly * es);
  if (e == cudaSuccess && r.kind == kLDA) e = cudaMalloc(reinterpret_cast<void**>(&q.labels), sizeof(int32_t) * r.n);
  const int64_t nout = (int64_t)(r.dx + (r.kind == kCCA ? r.dy : 0)) * r.k + r.k;
  if (e == cudaSuccess && q.out == nullptr) e = cudaMalloc(reinterpret_cast<void**>(&q.out), sizeof(double) * nout);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release(q);
    set_last_error("server: allocation of the request's device copies failed");
    return GBCCA_ERR_OOM;
  }
  *bytes = q.plan->dev_bytes + (int64_t)r.n * (lx + ly) * es + (r.kind == kLDA ? 4 * r.n : 0) + 8 * nout;
  return GBCCA_OK;
}

// Copies the data in, preconditions, and sets up the iteration state.
int start(Req& q, cudaStream_t st) {
  const gbcca_request& r = q.r;
  const int es = elt_size(r.dtype);
  const int64_t lx = padded_ld(r.dx, r.dtype);
  GB_CUDA(cudaMemcpy2DAsync(q.X, lx * es, r.X, r.ldx * es, (size_t)r.dx * es, r.n, cudaMemcpyDefault, st));
  if (r.kind == kCCA) {
    const int64_t ly = padded_ld(r.dy, r.dtype);
    GB_CUDA(cudaMemcpy2DAsync(q.Y, ly * es, r.Y, r.ldy * es, (size_t)r.dy * es, r.n, cudaMemcpyDefault, st));
    GB_TRY(cca_precondition(reinterpret_cast<gbcca_plan_t>(q.plan), q.X, lx, q.Y, ly, r.lambda_x, r.lambda_y,
                            nullptr, nullptr, st));
  } else {
    GB_CUDA(cudaMemcpyAsync(q.labels, r.labels, sizeof(int32_t) * r.n, cudaMemcpyDefault, st));
    GB_TRY(lda_bind(*q.plan, q.X, lx, q.labels, r.lambda_x, nullptr, nullptr, st));
  }
  return rcg_begin(*q.plan, nullptr, 0.0, nullptr, nullptr, st);
}

void fail(Server& s, Req& q, int rc) {
  release(q);
  if (q.bytes > 0) s.used -= q.bytes;
  q.bytes = 0;
  q.state = kFailed;
  q.status = rc;
  q.info = gbcca_info{};
  q.info.status = rc;
  q.t_finish = now_s(s);
}

// FIFO admission while the head fits the budget (a head larger than the
// whole budget fails with GBCCA_ERR_OOM; a head that only waits for running
// requests to finish blocks the queue, so requests are served in order).
int admit(Server& s, cudaStream_t st, bool* changed) {
  while (!s.queue.empty() && (int)s.running.size() < s.opt.max_active) {
    Req& q = s.reqs[s.queue.front()];
    int64_t bytes = 0;
    int rc = materialize(q, st, &bytes);
    if (rc == GBCCA_OK && s.used + bytes > s.opt.hbm_budget) {
      release(q);
      if (!s.running.empty()) break;  // wait for memory to come back
      rc = GBCCA_ERR_OOM;
      set_last_error("server: the request needs more device memory than the whole budget");
    }
    const int64_t id = s.queue.front();
    s.queue.pop_front();
    if (rc != GBCCA_OK) {
      fail(s, q, rc);
      continue;
    }
    q.bytes = q.held = bytes;
    s.used += bytes;
    q.t_admit = now_s(s);
    rc = start(q, st);
    if (rc != GBCCA_OK) {
      cudaStreamSynchronize(st);
      fail(s, q, rc);
      continue;
    }
    q.state = kRunning;
    s.running.push_back(id);
    *changed = true;
  }
  return GBCCA_OK;
}

// Refinement and outputs of a finished request; its memory goes back to the
// budget (the small output buffer stays until fetched).
void retire(Server& s, Req& q, cudaStream_t st) {
  const gbcca_request& r = q.r;
  double* U = q.out;
  double* V = r.kind == kCCA ? q.out + (int64_t)r.dx * r.k : nullptr;
  double* vals = q.out + (int64_t)(r.dx + (r.kind == kCCA ? r.dy : 0)) * r.k;
  const int rc = rcg_finish(*q.plan, U, V, vals, &q.info, 0.0, 0, st);
  release(q);
  s.used -= q.bytes;
  q.bytes = 0;
  q.status = rc;
  q.state = (rc == GBCCA_OK || rc == GBCCA_ERR_MAXITER) ? kFinished : kFailed;
  q.t_finish = now_s(s);
}

Server* as_server(gbcca_server_t h) { return reinterpret_cast<Server*>(h); }

}  // namespace
}  // namespace gbcca

using namespace gbcca;

extern "C" {

int gbcca_default_server_options(gbcca_server_options* opt) {
  if (opt == nullptr) return GBCCA_ERR_INVALID_ARG;
  std::memset(opt, 0, sizeof(*opt));
  opt->hbm_budget = (int64_t)120 << 30;
  opt->max_active = 64;
  opt->tick_iters = 8;
  opt->graphs = 1;
  return GBCCA_OK;
}

int gbcca_server_create(gbcca_server_t* out, const gbcca_server_options* opt) {
  if (out == nullptr) return GBCCA_ERR_INVALID_ARG;
  *out = nullptr;
  auto* s = new (std::nothrow) Server();
  if (s == nullptr) return GBCCA_ERR_OOM;
  gbcca_default_server_options(&s->opt);
  if (opt != nullptr) s->opt = *opt;
  if (s->opt.hbm_budget <= 0 || s->opt.max_active < 1 || s->opt.max_active > kMaxBatch || s->opt.tick_iters < 1) {
    delete s;
    set_last_error("gbcca_server_create: invalid options");
    return GBCCA_ERR_INVALID_ARG;
  }
  s->t0 = std::chrono::steady_clock::now();
  *out = reinterpret_cast<gbcca_server_t>(s);
  return GBCCA_OK;
}

int gbcca_server_submit(gbcca_server_t h, const gbcca_request* req, int64_t* id) {
  Server* s = as_server(h);
  if (s == nullptr || req == nullptr || id == nullptr || (req->kind != kCCA && req->kind != kLDA) ||
      req->X == nullptr || req->n < 1 || req->ldx < req->dx ||
      (req->kind == kCCA && (req->Y == nullptr || req->ldy < req->dy)) ||
      (req->kind == kLDA && req->labels == nullptr) || req->dtype < GBCCA_BF16 || req->dtype > GBCCA_FP64) {
    set_last_error("gbcca_server_submit: bad request");
    return GBCCA_ERR_INVALID_ARG;
  }
  const int64_t i = s->next_id++;
  Req& q = s->reqs[i];
  q.r = *req;
  q.t_submit = now_s(*s);
  s->queue.push_back(i);
  *id = i;
  return GBCCA_OK;
}

int gbcca_server_step(gbcca_server_t h, int32_t* queued, int32_t* running, void* stream) {
  Server* s = as_server(h);
  if (s == nullptr) return GBCCA_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool changed = false;
  GB_TRY(admit(*s, st, &changed));
  if (!s->running.empty()) {
    if (changed || s->batch == nullptr || s->batch_ids != s->running) {
      if (s->batch != nullptr) batch_free(s->batch);
      s->batch = nullptr;
      std::vector<Plan*> ps;
      for (int64_t i : s->running) ps.push_back(s->reqs[i].plan);
      gbcca_batch_options bo{};
      gbcca_default_batch_options(&bo);
      bo.batch_iters = s->opt.tick_iters;
      int rc = GBCCA_OK;
      s->batch = batch_make(ps.data(), (int)ps.size(), &bo, &rc);
      if (s->batch == nullptr) return rc;
      s->batch_ids = s->running;
      s->stable = false;
    }
    std::vector<char> active(s->running.size(), 1);
    GB_TRY(batch_iterate(*s->batch, active, s->opt.tick_iters, s->opt.graphs && s->stable, st));
    s->stable = true;
    int err_plan = -1;
    const int rc = batch_poll(*s->batch, active, nullptr, st, &err_plan);
    if (rc != GBCCA_OK) {
      // a request's own failure ends that request; a failure of the shared
      // launch ends every request of the batch
      for (size_t j = 0; j < s->running.size(); ++j)
        if (err_plan < 0 || (int)j == err_plan) fail(*s, s->reqs[s->running[j]], rc);
      std::vector<int64_t> keep;
      for (int64_t i : s->running)
        if (s->reqs[i].state == kRunning) keep.push_back(i);
      s->running.swap(keep);
    } else {
      std::vector<int64_t> keep;
      for (size_t j = 0; j < s->running.size(); ++j) {
        Req& q = s->reqs[s->running[j]];
        if (!active[j]) {
          retire(*s, q, st);
        } else {
          keep.push_back(s->running[j]);
        }
      }
      s->running.swap(keep);
    }
    if (s->running != s->batch_ids) s->stable = false;
  }
  if (queued != nullptr) *queued = (int32_t)s->queue.size();
  if (running != nullptr) *running = (int32_t)s->running.size();
  return GBCCA_OK;
}

int gbcca_server_state(gbcca_server_t h, int64_t id) {
  Server* s = as_server(h);
  if (s == nullptr) return GBCCA_ERR_INVALID_ARG;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return GBCCA_ERR_INVALID_ARG;
  return it->second.state;
}

int gbcca_server_result(gbcca_server_t h, int64_t id, double* U, double* V, double* vals, gbcca_info* info,
                        gbcca_request_times* times) {
  Server* s = as_server(h);
  if (s == nullptr) return GBCCA_ERR_INVALID_ARG;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    set_last_error("gbcca_server_result: unknown request");
    return GBCCA_ERR_INVALID_ARG;
  }
  Req& q = it->second;
  if (q.state != kFinished && q.state != kFailed) {
    set_last_error("gbcca_server_result: the request has not finished");
    return GBCCA_ERR_STATE;
  }
  const gbcca_request& r = q.r;
  if (q.state == kFinished && q.out != nullptr) {
    const int64_t nu = (int64_t)r.dx * r.k, nv = r.kind == kCCA ? (int64_t)r.dy * r.k : 0;
    if (U != nullptr) GB_CUDA(cudaMemcpy(U, q.out, sizeof(double) * nu, cudaMemcpyDefault));
    if (V != nullptr && nv > 0) GB_CUDA(cudaMemcpy(V, q.out + nu, sizeof(double) * nv, cudaMemcpyDefault));
    if (vals != nullptr) GB_CUDA(cudaMemcpy(vals, q.out + nu + nv, sizeof(double) * r.k, cudaMemcpyDefault));
  }
  if (info != nullptr) *info = q.info;
  if (times != nullptr) {
    times->submit_s = q.t_submit;
    times->admit_s = q.t_admit;
    times->finish_s = q.t_finish;
    times->device_bytes = q.held;
  }
  const int status = q.status;
  if (q.out != nullptr) cudaFree(q.out);
  s->reqs.erase(it);
  return status;
}

void gbcca_server_destroy(gbcca_server_t h) {
  Server* s = as_server(h);
  if (s == nullptr) return;
  if (s->batch != nullptr) batch_free(s->batch);
  for (auto& kv : s->reqs) {
    release(kv.second);
    if (kv.second.out != nullptr) cudaFree(kv.second.out);
  }
  delete s;
}

}  // extern "C"
