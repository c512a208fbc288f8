// Solve server: continuous batching of independent exponential-DG solves.
//
// Requests (a configuration, an initial state, dt and a step count) are
// queued by expdg_server_submit.  Worker threads - each with its own
// non-blocking CUDA stream - take requests in arrival order as soon as the
// device-memory budget admits them (a context's footprint: state, Krylov
// basis and scratch, all resident for the whole solve), so solves that arrive
// while others run start as soon as a worker and memory are free, and their
// kernels overlap on the GPU.  Finished contexts stay cached (idle) and are
// reused by later requests of the same shape, so a request pays no device
// allocation; idle contexts are released when the budget needs room.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/expdg.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Same context layout and behaviour (field by field: padding bytes may differ).
bool same_shape(const expdg_config& a, const expdg_config& b) {
  if (a.dim != b.dim || a.p != b.p || a.eq != b.eq || a.scheme != b.scheme || a.prec != b.prec) return false;
  if (a.m_max != b.m_max || a.m_step != b.m_step || a.max_substeps != b.max_substeps || a.iop != b.iop)
    return false;
  if (a.gamma != b.gamma || a.krylov_tol != b.krylov_tol || a.kappa != b.kappa || a.bc != b.bc) return false;
  if (a.flux != b.flux || a.tile != b.tile) return false;
  for (int d = 0; d < a.dim; ++d)
    if (a.ne[d] != b.ne[d] || a.lo[d] != b.lo[d] || a.hi[d] != b.hi[d]) return false;
  return true;
}

struct Request {
  int64_t id = 0;
  expdg_config cfg{};
  std::vector<double> q;  // initial state on submit, final state when done
  double dt = 0.0;
  int nsteps = 0;
  size_t bytes = 0;
  expdg_status status = EXPDG_OK;
  std::string error;
  expdg_stats stats{};
  double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
  bool done = false;
};

struct Cached {
  expdg_config cfg;
  expdg_ctx* ctx;
  size_t bytes;
};

}  // namespace

struct expdg_server {
  size_t budget = 0;
  size_t used = 0;  // bytes of every live context (busy or idle)
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> pending;
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  std::vector<int64_t> finished;  // done, not yet returned by poll
  std::vector<Cached> idle;
  std::vector<std::thread> workers;
  bool stop = false;
  int64_t next_id = 1;
  int busy = 0;
};

namespace {

// Pick the first pending request (in arrival order, looking at most `window`
// deep) that can run now; returns it with a context (reused or to be created).
// Called with the lock held.
bool take(expdg_server* s, Request** out, expdg_ctx** ctx, size_t* ctx_bytes) {
  const size_t window = 64;
  size_t k = 0;
  for (auto it = s->pending.begin(); it != s->pending.end() && k < window; ++it, ++k) {
    Request* r = *it;
    for (auto c = s->idle.begin(); c != s->idle.end(); ++c) {
      if (same_shape(c->cfg, r->cfg)) {
        *ctx = c->ctx;
        *ctx_bytes = c->bytes;
        s->idle.erase(c);
        s->pending.erase(it);
        *out = r;
        return true;
      }
    }
    // free idle contexts of other shapes while the request does not fit
    while (s->used + r->bytes > s->budget && !s->idle.empty()) {
      Cached victim = s->idle.back();
      s->idle.pop_back();
      s->used -= victim.bytes;
      expdg_destroy(victim.ctx);
    }
    if (s->used + r->bytes <= s->budget) {
      s->used += r->bytes;
      *ctx = nullptr;
      *ctx_bytes = r->bytes;
      s->pending.erase(it);
      *out = r;
      return true;
    }
  }
  return false;
}

void worker(expdg_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  for (;;) {
    Request* r = nullptr;
    expdg_ctx* ctx = nullptr;
    size_t bytes = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || take(s, &r, &ctx, &bytes); });
      if (!r) break;  // stopping
      ++s->busy;
    }
    r->t_start = now_s();
    expdg_status st = EXPDG_OK;
    if (!ctx) st = expdg_create(&r->cfg, &ctx);
    if (st == EXPDG_OK) st = expdg_set_stream(ctx, stream);
    if (st == EXPDG_OK) st = expdg_advance(ctx, r->q.data(), r->dt, r->nsteps, &r->stats);
    if (st != EXPDG_OK && ctx) r->error = expdg_last_error(ctx);
    r->t_done = now_s();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->status = st;
      r->done = true;
      s->finished.push_back(r->id);
      --s->busy;
      if (ctx && st == EXPDG_OK) {
        // the solve has synchronised its stream; detach the worker's stream,
        // which dies with the worker, before the context outlives it in the cache
        expdg_set_stream(ctx, nullptr);
        s->idle.push_back(Cached{r->cfg, ctx, bytes});
      } else {
        if (ctx) expdg_destroy(ctx);
        s->used -= bytes;
      }
    }
    s->cv.notify_all();
  }
  if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

expdg_status expdg_server_create(const expdg_server_config* cfg, expdg_server** out) {
  if (!cfg || !out || cfg->workers < 1 || cfg->workers > 64) return EXPDG_EINVAL;
  *out = nullptr;
  auto* s = new expdg_server();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return EXPDG_ECUDA;
  }
  s->budget = cfg->hbm_budget;
  if (s->budget == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      delete s;
      return EXPDG_ECUDA;
    }
    s->budget = free_b / 10 * 9;
  }
  for (int i = 0; i < cfg->workers; ++i) s->workers.emplace_back(worker, s);
  *out = s;
  return EXPDG_OK;
}

void expdg_server_destroy(expdg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& c : s->idle) expdg_destroy(c.ctx);
  delete s;
}

expdg_status expdg_server_submit(expdg_server* s, const expdg_config* cfg, const double* q0, double dt, int nsteps,
                                 int64_t* id) {
  if (!s || !cfg || !q0 || !id || nsteps < 0) return EXPDG_EINVAL;
  if (!(dt > 0.0) || !std::isfinite(dt)) return EXPDG_EINVAL;
  const size_t bytes = expdg_context_bytes(cfg);
  if (bytes == 0) return EXPDG_EINVAL;
  if (bytes > s->budget) return EXPDG_ENOMEM;
  auto r = std::make_unique<Request>();
  r->cfg = *cfg;
  size_t n = 1;
  const int m = (cfg->eq == EXPDG_BURGERS) ? 1 : cfg->dim + 2;
  for (int d = 0; d < cfg->dim; ++d) n *= (size_t)cfg->ne[d] * (size_t)(cfg->p + 1);
  n *= (size_t)m;
  r->q.assign(q0, q0 + n);
  r->dt = dt;
  r->nsteps = nsteps;
  r->bytes = bytes;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    *id = r->id;
    s->pending.push_back(r.get());
    s->reqs.emplace(r->id, std::move(r));
  }
  s->cv.notify_all();
  return EXPDG_OK;
}

expdg_status expdg_server_poll(expdg_server* s, int64_t* ids, int cap, int* n) {
  if (!s || !n || (cap > 0 && !ids)) return EXPDG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  const int k = std::min<int>(cap, (int)s->finished.size());
  for (int i = 0; i < k; ++i) ids[i] = s->finished[i];
  s->finished.erase(s->finished.begin(), s->finished.begin() + k);
  *n = k;
  return EXPDG_OK;
}

expdg_status expdg_server_fetch(expdg_server* s, int64_t id, double* q_out, expdg_stats* stats, double* times) {
  if (!s) return EXPDG_EINVAL;
  std::unique_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end() || !it->second->done) return EXPDG_EINVAL;
    r = std::move(it->second);
    s->reqs.erase(it);
  }
  if (q_out) std::memcpy(q_out, r->q.data(), r->q.size() * sizeof(double));
  if (stats) *stats = r->stats;
  if (times) {
    times[0] = r->t_start - r->t_submit;  // queueing
    times[1] = r->t_done - r->t_start;    // service
    times[2] = r->t_done - r->t_submit;   // latency
  }
  return r->status;
}

expdg_status expdg_server_info(expdg_server* s, size_t* used_bytes, int* pending, int* running) {
  if (!s) return EXPDG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (used_bytes) *used_bytes = s->used;
  if (pending) *pending = (int)s->pending.size();
  if (running) *running = s->busy;
  return EXPDG_OK;
}

}  // extern "C"
