// C-ABI of libexpdg: contexts, the Krylov phi-sum driver and the exponential
// steps (paper Sec. 2.3 and the EPI2 / EXPRB32 / EXPRB42 footnotes of Sec. 5).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "tables.h"

using namespace expdg;

struct expdg_ctx {
  expdg_config cfg{};
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool ff = false;     // float-float form: float-float Krylov storage and residual
  bool f32op = false;  // FP32 operator applies (EXPDG_MIXED, EXPDG_MIXED_FF)
  int lin_form = 0;    // DgForm of the linear operator apply

  int M = 0, NP = 0;
  size_t nelem = 0, N = 0, ld = 0;
  Tab tab{};
  DGArgs mesh{};  // mesh fields filled, pointers empty
  double lgl_r[MAXP + 1]{}, lgl_w[MAXP + 1]{};
  // FP64 buffers
  double* d_q = nullptr;   // state (copy of a host state, or scratch)
  double* d_q2 = nullptr;  // stage state
  double* d_t2 = nullptr;  // FP64 scratch (state differences)
  double* d_in = nullptr;  // API input scratch
  double* d_out = nullptr; // API output scratch
  // FP32 buffers (float-float and mixed forms)
  float* d_q32b = nullptr;  // FP32 operand of the operator apply (expdg_jv, the EXPRB stage correction)
  float* d_qfx = nullptr;   // the state as interleaved float-float pairs (residual of the FP32-operator forms)
  // mixed form: FP32 copies of the augmentation vectors b_1..b_P, read by the FP32 operator apply
  float* d_bf[EXPDG_MAX_PHI + 1] = {};
  double* d_src = nullptr;  // forcing added to R (expdg_set_source), allocated on first use
  bool has_src = false;
  // linearisation state of the linear operator (compute form: float or double)
  void* d_z = nullptr;
  // vectors in the Krylov storage form
  Vec c[EXPDG_MAX_PHI + 1]{};
  Vec b[EXPDG_MAX_PHI + 1]{};
  Vec w{}, rn{}, t1{}, t3{};
  Basis U{};
  KState* ks = nullptr;
  void* part = nullptr;
  KState* h_ks = nullptr;  // pinned mirror (host-visible block only is refreshed)
  int m_hint[2] = {0, 0};  // m accepted by each stage's first sub-step in the previous step
  int hint_uses[2] = {0, 0};  // steps that used the hint (every 8th also probes one check lower)
  bool probe_next[2] = {false, false};  // the last probe was accepted: probe again
  // CUDA graphs of Arnoldi segments (steps j0 .. j1-1), keyed by (j0, j1, P)
  std::map<long long, cudaGraphExec_t> graphs;
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture
  bool graphs_ok = true;
  std::vector<void*> allocs;
  std::string err;
  // profiling
  bool prof_on = false;
  expdg_kernel_prof prof[EXPDG_K_COUNT]{};
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
};

namespace {

const char* kVersion = "libexpdg 0.1 (sm_103a)";

expdg_status fail(expdg_ctx* ctx, expdg_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

#define CU(ctx, call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(ctx, EXPDG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

template <typename T>
cudaError_t dalloc(expdg_ctx* ctx, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
  if (e != cudaSuccess) return e;
  ctx->allocs.push_back(q);
  // zero-fill on the legacy default stream; expdg_create synchronises that
  // stream before returning, so work the caller later queues on any stream
  // (including non-blocking ones, which never wait for it) sees zeros
  e = cudaMemsetAsync(q, 0, n * sizeof(T) > 0 ? n * sizeof(T) : 16, 0);
  *p = static_cast<T*>(q);
  return e;
}

cudaError_t alloc_vec(expdg_ctx* ctx, Vec* v, size_t n) {
  *v = Vec{};
  if (ctx->ff) {
    cudaError_t e = dalloc(ctx, &v->h, n);
    if (e != cudaSuccess) return e;
    return dalloc(ctx, &v->l, n);
  }
  return dalloc(ctx, &v->d, n);
}

// Where a caller's pointer points: 0 host memory (copied through library
// buffers), 1 memory the context's device reaches directly (its own device
// memory, or managed memory; used in place), -1 device memory of another
// device (rejected: the kernels would dereference it without peer access).
int ptr_kind(const expdg_ctx* ctx, const void* p) {
  if (p == nullptr) return 0;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (at.type == cudaMemoryTypeManaged) return 1;
  if (at.type == cudaMemoryTypeDevice) return at.device == ctx->dev ? 1 : -1;
  return 0;
}
bool is_device_ptr(const expdg_ctx* ctx, const void* p) { return ptr_kind(ctx, p) == 1; }
// EXPDG_EINVAL if any of the caller's pointers is another device's memory.
expdg_status check_ptrs(expdg_ctx* ctx, std::initializer_list<const void*> ps) {
  for (const void* p : ps)
    if (ptr_kind(ctx, p) < 0) {
      ctx->err = "a pointer to another device's memory";
      return EXPDG_EINVAL;
    }
  return EXPDG_OK;
}

Vec null_vec() { return Vec{}; }
Vec dvec(double* p) {
  Vec v{};
  v.d = p;
  return v;
}

// The operator kernel of DgForm `form` on stream s.
cudaError_t launch_dg_form(expdg_ctx* ctx, bool linear, int form, const DGArgs& a, cudaStream_t s) {
  const int p = ctx->cfg.p, eq = ctx->cfg.eq;
  switch (ctx->cfg.dim) {
    case 1: return launch_dg_1d(linear, form, eq, p, a, ctx->tab, s);
    case 2: return launch_dg_2d(linear, form, eq, p, a, ctx->tab, s);
    case 3: return launch_dg_3d(linear, form, eq, p, a, ctx->tab, s);
  }
  return cudaErrorInvalidValue;
}

// The context's linear operator apply (its form) on the context's stream, or
// on an explicit stream (graph capture).
cudaError_t launch_lin(expdg_ctx* ctx, const DGArgs& a) { return launch_dg_form(ctx, true, ctx->lin_form, a, ctx->stream); }
cudaError_t launch_lin_on(expdg_ctx* ctx, const DGArgs& a, cudaStream_t s) {
  return launch_dg_form(ctx, true, ctx->lin_form, a, s);
}

long long graph_key(int j0, int j1, int P) { return ((long long)j0 * 1024 + j1) * 8 + P; }

// The cached graph of Arnoldi steps j0 .. j1-1, or null.
cudaGraphExec_t find_graph(expdg_ctx* ctx, int j0, int j1, int P) {
  if (!ctx->graphs_ok) return nullptr;
  auto it = ctx->graphs.find(graph_key(j0, j1, P));
  return it == ctx->graphs.end() ? nullptr : it->second;
}

// Instantiated graph of Arnoldi steps j0 .. j1-1 for P augmentation vectors,
// captured once on the context's private stream from `launches(j, stream,
// counted = false)` and reused by every later sub-step (their launch
// arguments are the same; the sub-step scalars live in device memory).
// nullptr when capture is not available (the caller launches directly).
template <class F>
cudaGraphExec_t segment_graph(expdg_ctx* ctx, int j0, int j1, int P, F&& launches) {
  if (!ctx->graphs_ok) return nullptr;
  const long long key = graph_key(j0, j1, P);
  auto it = ctx->graphs.find(key);
  if (it != ctx->graphs.end()) return it->second;
  if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ctx->graphs_ok = false;
    return nullptr;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  for (int j = j0; ok && j < j1; ++j) ok = launches(j, ctx->cap_stream, false) == cudaSuccess;
  const bool ended = cudaStreamEndCapture(ctx->cap_stream, &graph) == cudaSuccess;
  ok = ok && ended && graph != nullptr && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    if (exec) cudaGraphExecDestroy(exec);
    cudaGetLastError();
    ctx->graphs_ok = false;  // launch directly from now on
    return nullptr;
  }
  ctx->graphs.emplace(key, exec);
  return exec;
}


cudaEvent_t pool_event(expdg_ctx* ctx) {
  if (ctx->ev_used == ctx->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    ctx->ev_pool.push_back(e);
  }
  return ctx->ev_pool[ctx->ev_used++];
}

// Count (and, when profiling, time) one kernel launch of class cls.
template <class F>
cudaError_t run(expdg_ctx* ctx, int cls, double bytes, F&& launch) {
  ctx->prof[cls].launches++;
  ctx->prof[cls].bytes += bytes;
  if (!ctx->prof_on) return launch();
  cudaEvent_t a = pool_event(ctx), b = pool_event(ctx);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaEventRecord(a, ctx->stream);
  cudaError_t e = launch();
  cudaEventRecord(b, ctx->stream);
  ctx->recs.push_back(expdg_ctx::Rec{cls, a, b});
  return e;
}

#define RUN(ctx, cls, bytes, call) CU(ctx, run(ctx, cls, (double)(bytes), [&]() { return (call); }))

void set_alpha(DGArgs& a, double alpha) {
  a.alpha = alpha;
  a.alpha_h = (float)alpha;
  a.alpha_l = (float)(alpha - (double)a.alpha_h);
}

// R(q) -> out (Krylov storage form), times alpha.  FP64 form: FP64
// throughout.  R of a smooth state is a small difference of large fluxes: an
// FP32 residual (measured in the mixed form: relative error 3e-6 on the 32^3
// p = 3 wave) put broadband noise into the Krylov start vector that cost extra
// Arnoldi steps (m = 37 against 27 at tol 1e-8) and errors above 1e-6 against
// the FP64 form after the 20 - 50 steps of the batched and served solves.
// The FP32-operator forms (mixed and float-float): the state is split once
// into float-float pairs and the residual is computed in float-float
// arithmetic on the FP32 pipes (accurate to about 1e-14 of the flux scale;
// 3.7x faster than the FP64 kernel on the 32^3 p = 3 wave, whose FP64 flux
// and derivative arithmetic is bound by GB300's FP64 pipe); the mixed form
// takes the result as h + l in FP64 (exact).
// converted: ctx->d_qfx already holds q (written by linstate_into).
cudaError_t residual_into(expdg_ctx* ctx, const double* q, Vec out, double alpha, bool converted = false) {
  DGArgs a = ctx->mesh;
  set_alpha(a, alpha);
  a.src = ctx->has_src ? ctx->d_src : nullptr;
  a.status = &ctx->ks->status;
  if (!ctx->f32op) {
    a.q = q;
    a.out = out.d;
    return run(ctx, EXPDG_K_RESIDUAL, 16.0 * ctx->N,
               [&]() { return launch_dg_form(ctx, false, DG_F64, a, ctx->stream); });
  }
  if (!converted) {
    const cudaError_t e =
        run(ctx, EXPDG_K_VECTOR, 16.0 * ctx->N, [&]() { return launch_f64_to_fx(ctx->d_qfx, q, ctx->N, ctx->stream); });
    if (e != cudaSuccess) return e;
  }
  a.q = ctx->d_qfx;
  if (ctx->ff) {
    a.out_h = out.h;
    a.out_l = out.l;
  } else {
    a.out = out.d;
  }
  return run(ctx, EXPDG_K_RESIDUAL, 16.0 * ctx->N, [&]() {
    const int p = ctx->cfg.p, eq = ctx->cfg.eq;
    switch (ctx->cfg.dim) {
      case 1: return launch_dg_fx_1d(eq, p, a, ctx->tab, ctx->stream);
      case 2: return launch_dg_fx_2d(eq, p, a, ctx->tab, ctx->stream);
      case 3: return launch_dg_fx_3d(eq, p, a, ctx->tab, ctx->stream);
    }
    return cudaErrorInvalidValue;
  });
}

// Linearisation state of qt (FP64, device) -> ctx->d_z, in compute form;
// with_fx (FP32-operator forms): qt as float-float pairs into ctx->d_qfx as
// well, for a residual at qt that follows.
cudaError_t linstate_into(expdg_ctx* ctx, const double* qt, bool with_fx = false) {
  float* qfx = (with_fx && ctx->f32op) ? ctx->d_qfx : nullptr;
  const bool f32 = ctx->f32op;
  const double bytes = (8.0 + (f32 ? 4.0 : 8.0) + (qfx ? 8.0 : 0.0)) * ctx->N;
  return run(ctx, EXPDG_K_VECTOR, bytes, [&]() {
    const size_t stride = ctx->mesh.stride;
    switch (ctx->cfg.dim) {
      case 1: return launch_linstate_1d(ctx->cfg.eq, f32, qt, ctx->d_z, stride, ctx->cfg.gamma, ctx->mesh.roe,
                                         qfx, ctx->stream);
      case 2: return launch_linstate_2d(ctx->cfg.eq, f32, qt, ctx->d_z, stride, ctx->cfg.gamma, ctx->mesh.roe,
                                         qfx, ctx->stream);
      case 3: return launch_linstate_3d(ctx->cfg.eq, f32, qt, ctx->d_z, stride, ctx->cfg.gamma, ctx->mesh.roe,
                                         qfx, ctx->stream);
    }
    return cudaErrorInvalidValue;
  });
}

// Algorithmic bytes of one linear operator apply per unknown: read v and z,
// write the output (FP64 form 8 + 8 + 8; FP32-operator forms v FP32, z FP32,
// output FP64 or a float-float pair (8), or FP32 (4: the mixed form's Arnoldi
// steps with incomplete orthogonalisation)).
double jv_bytes_per_unknown(const expdg_ctx* ctx, bool out32 = false) {
  return ctx->f32op ? (out32 ? 12.0 : 16.0) : 24.0;
}

// L(qt) v -> out (no augmentation).  qt_T: linearisation state of qt in compute
// form (ctx->d_z, from linstate_into), v_T: input (FP32 in the FP32-operator
// forms, FP64 otherwise); out FP64 (or float-float in the float-float form).
cudaError_t jv_into(expdg_ctx* ctx, const void* qt_T, const void* v_T, Vec out, double alpha) {
  DGArgs a = ctx->mesh;
  set_alpha(a, alpha);
  a.q = qt_T;
  a.v = v_T;
  if (ctx->ff) {
    a.out_h = out.h;
    a.out_l = out.l;
  } else {
    a.out = out.d;
  }
  return run(ctx, EXPDG_K_JV, jv_bytes_per_unknown(ctx) * ctx->N, [&]() { return launch_lin(ctx, a); });
}

// while_waiting: host work done after the copy is queued and before the wait
// (the device is still busy with the queued launches).
template <class W>
expdg_status readback(expdg_ctx* ctx, W&& while_waiting) {
  const size_t off = offsetof(KState, red);
  CU(ctx, cudaMemcpyAsync(reinterpret_cast<char*>(ctx->h_ks) + off, reinterpret_cast<char*>(ctx->ks) + off,
                          sizeof(KState) - off, cudaMemcpyDeviceToHost, ctx->stream));
  while_waiting();
  CU(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->h_ks->status & 1) return fail(ctx, EXPDG_ENONPHYSICAL, "non-physical state (rho <= 0 or p <= 0)");
  return EXPDG_OK;
}
expdg_status readback(expdg_ctx* ctx) {
  return readback(ctx, [] {});
}

struct Replay {
  const expdg_trace_entry* e = nullptr;
  int n = 0;
};

constexpr size_t kPairMinUnknowns = 131072;


// w = sum_{i=0}^P phi_i(tau L(qt)) c_i  (c_i in ctx->c, has[i] false: zero).
// On the final sub-step the combination writes fin_out = fin_base + w instead
// of ctx->w (fin_out null: result left in ctx->w).
// use_hint: start the error checks of the first sub-step at m_prev, the m this
// stage accepted in the previous step (consecutive steps need similar m; a
// later acceptance is only more exact); every 8th step, and the step after an
// accepted probe, probes one check lower first (m_prev - 1 with paired checks,
// which evaluate H_{m-1} and H_m together, else max(m_step, m_prev - m_step)).
expdg_status phi_solve(expdg_ctx* ctx, const void* qt_T, double tau, const bool* has, int P, Vec fin_base,
                       Vec fin_out, int solve_id, const Replay& rp, expdg_stats* st,
                       std::vector<expdg_trace_entry>* trace, bool use_hint = false) {
  const size_t N = ctx->N, n_aug = N + P;
  const bool F = ctx->ff;
  const cudaStream_t s = ctx->stream;
  const expdg_config& cfg = ctx->cfg;
  // w(0) = c_0
  if (has[0]) {
    Vec x[1] = {ctx->c[0]};
    double a1[1] = {1.0};
    RUN(ctx, EXPDG_K_VECTOR, 16.0 * N, launch_lincomb(F, ctx->w, 1, x, a1, N, s));
  } else {
    if (F) {
      CU(ctx, cudaMemsetAsync(ctx->w.h, 0, N * sizeof(float), s));
      CU(ctx, cudaMemsetAsync(ctx->w.l, 0, N * sizeof(float), s));
    } else {
      CU(ctx, cudaMemsetAsync(ctx->w.d, 0, N * sizeof(double), s));
    }
  }
  std::vector<const expdg_trace_entry*> mine;
  if (rp.e)
    for (int k = 0; k < rp.n; ++k)
      if (rp.e[k].solve == solve_id) mine.push_back(&rp.e[k]);
  size_t krep = 0;
  double sv = 0.0, sigma = 1.0;
  int rejected = 0;
  while (sv < 1.0) {
    int m_fix = 0;
    double eta = 1.0;
    const bool replay = rp.e != nullptr;
    if (replay) {
      if (krep >= mine.size()) return fail(ctx, EXPDG_EINVAL, "replay trace ended before the solve finished");
      sigma = mine[krep]->sigma;
      m_fix = mine[krep]->m;
      eta = mine[krep]->eta;
      ++krep;
      if (m_fix < 0 || m_fix > cfg.m_max) return fail(ctx, EXPDG_EINVAL, "replayed m out of range");
    }
    // b_i = sigma^i sum_{j=0}^{P-i} s^j/j! c_{i+j}
    for (int i = 1; i <= P; ++i) {
      Vec xs[EXPDG_MAX_PHI + 1];
      double as[EXPDG_MAX_PHI + 1];
      int nx = 0;
      double fact = 1.0;
      for (int j = 0; j <= P - i; ++j) {
        if (j > 0) fact *= j;
        xs[nx] = has[i + j] ? ctx->c[i + j] : null_vec();
        as[nx] = std::pow(sigma, i) * std::pow(sv, j) / fact;
        ++nx;
      }
      RUN(ctx, EXPDG_K_VECTOR, 8.0 * (nx + 1) * N, launch_lincomb(F, ctx->b[i], nx, xs, as, N, s));
      // mixed form: the FP32 operator apply reads an FP32 copy of b_i
      if (ctx->f32op && !F) RUN(ctx, EXPDG_K_VECTOR, 12.0 * N, launch_to_f32(ctx->d_bf[i], ctx->b[i].d, N, s));
    }
    {
      Vec xs[EXPDG_MAX_PHI + 1];
      xs[0] = ctx->w;
      for (int i = 1; i <= P; ++i) xs[i] = ctx->b[i];
      // adaptive: the norms kernel also forms eta and beta on the device, so the
      // Arnoldi steps follow without a host round trip
      RUN(ctx, EXPDG_K_VECTOR, 8.0 * (P + 1) * N,
          launch_norms(F, ctx->ks, ctx->part, P + 1, xs, N, replay ? -1 : P, s));
    }
    expdg_status rs = EXPDG_OK;
    const bool last = (sv + sigma >= 1.0);
    const int iop = cfg.iop;
    double beta = -1.0;  // adaptive: in KState (the phi kernel reads it there)
    if (replay) {
      rs = readback(ctx);
      if (rs != EXPDG_OK) return rs;
      beta = std::sqrt(ctx->h_ks->red[0] + (P > 0 ? 1.0 / (eta * eta) : 0.0));
      if (beta == 0.0) {  // P == 0 and c_0 == 0: the result is zero
        sv += sigma;
        st->substeps++;
        if (trace) trace->push_back(expdg_trace_entry{solve_id, 0, sigma, eta});
        continue;
      }
      const double s0 = iop ? 1.0 / beta : 1.0;  // incomplete orthogonalisation: slot 0 holds beta v_0
      RUN(ctx, EXPDG_K_VECTOR, 16.0 * N, launch_start(F, ctx->ks, ctx->U, ctx->w, N, P, eta, s0, sigma * tau, 0, s));
    } else {
      // a zero start vector (P == 0, c_0 == 0) gives s0 = 0: the Arnoldi steps
      // break down at once and the combination adds zero
      RUN(ctx, EXPDG_K_VECTOR, 16.0 * N,
          launch_start(F, ctx->ks, ctx->U, ctx->w, N, P, 0.0, 0.0, sigma * tau, iop ? 1 : 2, s));
    }
    const int limit = replay ? m_fix : cfg.m_max;
    // checks at m_first, m_again, m_late and m_late + 2, then at the multiples of m_step
    int m_first = cfg.m_step, m_again = 0, m_late = 0;
    // Paired checks (the FP32-operator forms' change since m - 1, evaluated in
    // the check's launch) on problems of at least kPairMinUnknowns: there an
    // Arnoldi step costs more than the second exponential.  Below that, when
    // many small solves share the GPU, the extra cluster time outweighs the
    // saved steps.
    const bool f32 = ctx->f32op, mx = f32 && !F;
    const int kf = F ? KF_FF : (mx ? KF_MX : KF_F64);
    const bool pairs = f32 && !replay && N >= kPairMinUnknowns;
    const bool first_sub = (sv == 0.0 && rejected == 0);
    const int sid = solve_id & 1;
    bool probe = false;
    if (use_hint && first_sub && !replay && ctx->m_hint[sid] > 0) {
      probe = ctx->probe_next[sid] || (ctx->hint_uses[sid] % 8) == 0;
      ctx->hint_uses[sid]++;
      const int h = ctx->m_hint[sid];
      m_first = pairs ? std::max(1, h - (probe ? 1 : 0)) : std::max(cfg.m_step, h - (probe ? cfg.m_step : 0));
      m_again = h;
      if (pairs) m_late = h + 2;  // checks carry their own pair: cheap to retry
    }
    bool accepted = false;
    int m_acc = 0;
    double err = 0.0;
    // One Arnoldi step j on stream ss: operator apply, then the two
    // orthogonalisation passes.  The sub-step scalars come from KState (the
    // start kernel wrote them), so a step's launches are the same for every
    // sub-step and a run of steps can be replayed as a CUDA graph.
    const double vb = 8.0 * (double)n_aug;  // one vector: FP64 or float-float pair
    // an operator apply of an Arnoldi step: v, z and the output, plus the
    // augmentation vectors b_i (FP64, FP32 copies in the mixed form, float-float)
    const double jv_apply_bytes =
        (jv_bytes_per_unknown(ctx, mx && iop) + P * (mx ? 4.0 : 8.0)) * (double)N;
    // orthogonalisation passes: window slots read (8 bytes an entry), w' read
    // (FP32 top part in the mixed form's incomplete orthogonalisation), the
    // update's output written (plus its FP32 shadow in the mixed form)
    auto dots_bytes = [&](int jj) {
      if (!iop) return (jj + 2) * vb;
      const int nw = std::min(iop, jj + 1);
      return mx ? (nw + 0.5) * vb : (nw + 1) * vb;
    };
    auto update_bytes = [&](int jj) {
      if (!iop) return (jj + 4) * vb + (mx ? 0.5 * vb : 0.0);
      const int nw = std::min(iop, jj + 1);
      return (nw + 2) * vb;  // mixed: w' 4 + slot 8 + shadow 4 bytes
    };
    auto step_launches = [&](int j, cudaStream_t ss, bool counted) -> cudaError_t {
      DGArgs a = ctx->mesh;
      a.scal = &ctx->ks->jv;
      a.q = qt_T;
      a.z_early = 1;  // z was made before the solve's start kernel (a plain launch)
      const Vec vj = ctx->U.at(j), vo = ctx->U.at(j + 1);
      if (F) {
        a.v = vj.h;
        a.out_h = vo.h;
        a.out_l = vo.l;
      } else if (mx) {  // FP32 shadow in; FP32 out with incomplete orthogonalisation, else FP64
        a.v = vj.h;
        if (iop)
          a.out_h = vo.h;
        else
          a.out = vo.d;
      } else {
        a.v = vj.d;
        a.out = vo.d;
      }
      if (P > 0) {
        a.paug = P;
        if (F) {
          a.tail_h = vj.h + N;
          a.tail_l = vj.l + N;
          a.out_tail_h = vo.h + N;
          a.out_tail_l = vo.l + N;
        } else {
          a.tail_d = vj.d + N;
          a.out_tail_d = vo.d + N;
        }
        for (int i = 1; i <= P; ++i) {
          a.W_d[i] = ctx->b[i].d;
          a.W_h[i] = ctx->b[i].h;
          a.W_l[i] = ctx->b[i].l;
          a.W_f[i] = ctx->d_bf[i];
        }
      }
      const double bytes[3] = {jv_apply_bytes, dots_bytes(j), update_bytes(j)};
      auto l0 = [&]() { return launch_lin_on(ctx, a, ss); };
      auto l1 = [&]() {
        return iop ? launch_iom_dots(kf, iop, ctx->ks, ctx->part, ctx->U, j, N, n_aug, ss)
                   : launch_dots(F, ctx->ks, ctx->part, ctx->U, j, n_aug, ss);
      };
      auto l2 = [&]() {
        return iop ? launch_iom_update(kf, iop, ctx->ks, ctx->part, ctx->U, j, N, n_aug, ss)
                   : launch_update(F, ctx->ks, ctx->part, ctx->U, j, n_aug, ss);
      };
      cudaError_t e;
      if (counted) {  // direct launches, counted (and timed when profiling)
        if ((e = run(ctx, EXPDG_K_JV, bytes[0], l0)) != cudaSuccess) return e;
        if ((e = run(ctx, EXPDG_K_DOTS, bytes[1], l1)) != cudaSuccess) return e;
        return run(ctx, EXPDG_K_UPDATE, bytes[2], l2);
      }
      if ((e = l0()) != cudaSuccess) return e;
      if ((e = l1()) != cudaSuccess) return e;
      return l2();
    };
    auto due = [&](int m) {
      return replay ? (m == m_fix)
                    : (m == cfg.m_max || m == m_first || m == m_again ||
                       (m_late > 0 && (m == m_late || m == m_late + 2)) || (m > m_first && m % cfg.m_step == 0));
    };
    // Arnoldi steps j0 .. j1 - 1: one graph replay, or direct launches when
    // the range has no graph yet (it is captured while the host next waits
    // for the device, so a new range never waits for a capture)
    std::vector<std::pair<int, int>> to_capture;
    auto segment = [&](int j0, int j1) -> cudaError_t {
      cudaGraphExec_t g = ctx->prof_on ? nullptr : find_graph(ctx, j0, j1, P);
      if (!g && !ctx->prof_on && ctx->graphs_ok) to_capture.emplace_back(j0, j1);
      if (!g) {
        for (int jj = j0; jj < j1; ++jj) {
          const cudaError_t e = step_launches(jj, s, true);
          if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
      }
      for (int jj = j0; jj < j1; ++jj) {  // count the replayed launches like direct ones
        ctx->prof[EXPDG_K_JV].launches++;
        ctx->prof[EXPDG_K_JV].bytes += jv_apply_bytes;
        ctx->prof[EXPDG_K_DOTS].launches++;
        ctx->prof[EXPDG_K_DOTS].bytes += dots_bytes(jj);
        ctx->prof[EXPDG_K_UPDATE].launches++;
        ctx->prof[EXPDG_K_UPDATE].bytes += update_bytes(jj);
      }
      return cudaGraphLaunch(g, s);
    };
    int j = 0;
    while (j < limit) {
      int m = j + 1;  // next error check (due at m == limit at the latest)
      while (m < limit && !due(m)) ++m;
      CU(ctx, segment(j, m));
      st->krylov_iters += m - j;
      st->jv_applies += m - j;
      j = m;
      if (!due(m)) continue;
      // FP32-operator forms: the operator's rounding noise inflates Saad's
      // estimate, so a converged change since m - 1 also accepts (the check
      // evaluates both).  phi(H) in FP64, float-float in the float-float form.
      RUN(ctx, EXPDG_K_PHI, 8.0 * m * m,
          launch_phi(ctx->ks, m, beta, cfg.krylov_tol, replay ? 1 : 0, f32 ? 1 : 0, iop ? ctx->part : nullptr, kf,
                     iop ? iom_update_blocks(kf, iop, n_aug) : 0, F, pairs, s));
      // the combination follows the check at once and writes only if it
      // accepted, so an accepted check needs no second host round trip; its
      // bytes are counted once the decision is known
      const bool fin = last && fin_out.d != nullptr;
      RUN(ctx, EXPDG_K_COMBINE, 0.0,
          launch_combine(F, ctx->ks, ctx->U, fin ? fin_base : null_vec(), fin ? fin_out : ctx->w, N, true, s));
      rs = readback(ctx, [&] {
        for (const auto& r : to_capture) segment_graph(ctx, r.first, r.second, P, step_launches);
        to_capture.clear();
      });
      if (rs != EXPDG_OK) return rs;
      if (!replay) eta = ctx->h_ks->eta;
      if (ctx->h_ks->accept) {
        accepted = true;
        m_acc = ctx->h_ks->m_eff;
        err = ctx->h_ks->err;
        ctx->prof[EXPDG_K_COMBINE].bytes += 8.0 * (m_acc + (fin ? 2 : 1)) * N;
        break;
      }
    }
    if (!accepted) {
      st->rejected++;
      if (++rejected > cfg.max_substeps)
        return fail(ctx, EXPDG_EKRYLOV, "Krylov solve did not converge within the sub-step budget");
      sigma *= 0.5;
      continue;
    }
    if (use_hint && first_sub && !replay) {
      ctx->m_hint[sid] = m_acc;
      ctx->probe_next[sid] = probe && m_acc == m_first;  // m may still fall: probe again next step
    }
    sv += sigma;
    st->substeps++;
    st->err_est = std::fmax(st->err_est, err);
    if (trace) trace->push_back(expdg_trace_entry{solve_id, m_acc, sigma, eta});
    if (!replay) {
      if (m_acc <= cfg.m_max / 2) sigma *= 2.0;
      sigma = std::fmin(sigma, 1.0 - sv);
    }
  }
  return EXPDG_OK;
}

expdg_status validate(const expdg_config* c) {
  if (!c) return EXPDG_EINVAL;
  if (c->dim < 1 || c->dim > 3) return EXPDG_EINVAL;
  if (c->p < 1 || c->p > EXPDG_MAX_ORDER) return EXPDG_EINVAL;
  if (c->eq != EXPDG_BURGERS && c->eq != EXPDG_EULER) return EXPDG_EINVAL;
  if (c->eq == EXPDG_BURGERS && c->dim != 1) return EXPDG_EINVAL;
  for (int d = 0; d < c->dim; ++d) {
    if (c->ne[d] < 1) return EXPDG_EINVAL;
    if (!(c->hi[d] > c->lo[d])) return EXPDG_EINVAL;
  }
  if (c->eq == EXPDG_EULER && !(c->gamma > 1.0)) return EXPDG_EINVAL;
  if (c->scheme != EXPDG_EPI2 && c->scheme != EXPDG_EXPRB32 && c->scheme != EXPDG_EXPRB42) return EXPDG_EINVAL;
  if (c->prec != EXPDG_FP64 && c->prec != EXPDG_MIXED && c->prec != EXPDG_MIXED_FF) return EXPDG_EINVAL;
  if (!(c->krylov_tol > 0.0)) return EXPDG_EINVAL;
  if (c->m_max < 1 || c->m_max > EXPDG_MAX_KRYLOV) return EXPDG_EINVAL;
  if (c->m_step < 1) return EXPDG_EINVAL;
  if (c->max_substeps < 0) return EXPDG_EINVAL;
  if (c->iop < 0 || c->iop > EXPDG_MAX_IOP) return EXPDG_EINVAL;
  if (!(c->kappa >= 0.0) || !std::isfinite(c->kappa)) return EXPDG_EINVAL;
  if (c->bc != EXPDG_BC_PERIODIC && c->bc != EXPDG_BC_DIRICHLET) return EXPDG_EINVAL;
  if ((c->kappa > 0.0 || c->bc != EXPDG_BC_PERIODIC) && c->eq != EXPDG_BURGERS) return EXPDG_EINVAL;
  if (c->flux != EXPDG_FLUX_LF && c->flux != EXPDG_FLUX_ROE) return EXPDG_EINVAL;
  if (c->flux == EXPDG_FLUX_ROE && c->eq != EXPDG_EULER) return EXPDG_EINVAL;
  if (c->tile < EXPDG_TILE_AUTO || c->tile > EXPDG_TILE_TC1) return EXPDG_EINVAL;
  return EXPDG_OK;
}

// Copy a caller array (host or device) of n doubles into device memory;
// returns the device pointer to use (the caller's own if already on device).
const double* in_dev(expdg_ctx* ctx, const double* p, double* scratch, size_t n, cudaError_t* e) {
  *e = cudaSuccess;
  if (p == nullptr || is_device_ptr(ctx, p)) return p;
  *e = cudaMemcpyAsync(scratch, p, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  return scratch;
}

// One step of the configured scheme, q (device FP64) in place.
expdg_status step_dev(expdg_ctx* ctx, double* q, double dt, const Replay& rp, expdg_stats* st,
                      std::vector<expdg_trace_entry>* trace) {
  const bool F = ctx->ff;
  const size_t N = ctx->N;
  const cudaStream_t s = ctx->stream;
  CU(ctx, cudaMemsetAsync(&ctx->ks->status, 0, sizeof(int), s));
  // Linearisation state of the Jacobian point q, shared by every stage.
  CU(ctx, linstate_into(ctx, q, true));  // and q as float-float pairs for R(q)
  const void* qt_T = ctx->d_z;
  bool has[EXPDG_MAX_PHI + 1] = {false, false, false, false};
  const int scheme = ctx->cfg.scheme;
  if (scheme == EXPDG_EPI2) {
    CU(ctx, residual_into(ctx, q, ctx->c[1], dt, ctx->f32op));
    st->residual_applies++;
    has[1] = true;
    return phi_solve(ctx, qt_T, dt, has, 1, dvec(q), dvec(q), 0, rp, st, trace, true);
  }
  // EXPRB32 / EXPRB42 share: R^n, stage 1, D_{n,2} = R(q2) - R^n - L (q2 - q)
  CU(ctx, residual_into(ctx, q, ctx->rn, 1.0, ctx->f32op));
  st->residual_applies++;
  const double a1 = (scheme == EXPDG_EXPRB32) ? dt : 0.75 * dt;
  {
    Vec x[1] = {ctx->rn};
    double a[1] = {a1};
    RUN(ctx, EXPDG_K_VECTOR, 16.0 * N, launch_lincomb(F, ctx->c[1], 1, x, a, N, s));
  }
  has[1] = true;
  expdg_status r = phi_solve(ctx, qt_T, a1, has, 1, dvec(q), dvec(ctx->d_q2), 0, rp, st, trace, true);
  if (r != EXPDG_OK) return r;
  // t1 = R(q2)
  CU(ctx, residual_into(ctx, ctx->d_q2, ctx->t1, 1.0));
  st->residual_applies++;
  // t2 = q2 - q (FP64), t3 = L(q) t2
  {
    Vec x[2] = {dvec(ctx->d_q2), dvec(q)};
    double a[2] = {1.0, -1.0};
    RUN(ctx, EXPDG_K_VECTOR, 24.0 * N, launch_lincomb(false, dvec(ctx->d_t2), 2, x, a, N, s));
  }
  if (ctx->f32op) {  // the FP32 operator reads an FP32 input
    RUN(ctx, EXPDG_K_VECTOR, 12.0 * N, launch_to_f32(ctx->d_q32b, ctx->d_t2, N, s));
    CU(ctx, jv_into(ctx, qt_T, ctx->d_q32b, ctx->t3, 1.0));
  } else {
    CU(ctx, jv_into(ctx, qt_T, ctx->d_t2, ctx->t3, 1.0));
  }
  st->jv_applies++;
  const double cD = (scheme == EXPDG_EXPRB32) ? 2.0 * dt : (32.0 / 9.0) * dt;
  {
    Vec x[3] = {ctx->t1, ctx->rn, ctx->t3};
    double a[3] = {cD, -cD, -cD};
    RUN(ctx, EXPDG_K_VECTOR, 32.0 * N, launch_lincomb(F, ctx->c[3], 3, x, a, N, s));
  }
  bool has2[EXPDG_MAX_PHI + 1] = {false, false, false, true};
  if (scheme == EXPDG_EXPRB32) {
    // q^{n+1} = q2 + 2 dt phi_3(dt L) D
    return phi_solve(ctx, qt_T, dt, has2, 3, dvec(ctx->d_q2), dvec(q), 1, rp, st, trace, true);
  }
  // EXPRB42: q^{n+1} = q + dt phi_1(dt L) R^n + 32/9 dt phi_3(dt L) D
  {
    Vec x[1] = {ctx->rn};
    double a[1] = {dt};
    RUN(ctx, EXPDG_K_VECTOR, 16.0 * N, launch_lincomb(F, ctx->c[1], 1, x, a, N, s));
  }
  has2[1] = true;
  return phi_solve(ctx, qt_T, dt, has2, 3, dvec(q), dvec(q), 1, rp, st, trace, true);
}

void write_trace(const std::vector<expdg_trace_entry>& tr, expdg_trace_entry* out, int cap, int* n) {
  if (n) *n = (int)tr.size();
  if (!out) return;
  for (int k = 0; k < (int)tr.size() && k < cap; ++k) out[k] = tr[k];
}

}  // namespace

extern "C" {

const char* expdg_version(void) { return kVersion; }

void expdg_default_config(expdg_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->dim = 2;
  c->p = 4;
  c->ne[0] = c->ne[1] = c->ne[2] = 64;
  for (int d = 0; d < 3; ++d) {
    c->lo[d] = 0.0;
    c->hi[d] = 10.0;
  }
  c->eq = EXPDG_EULER;
  c->gamma = 1.4;
  c->scheme = EXPDG_EPI2;
  c->prec = EXPDG_FP64;
  c->krylov_tol = 1e-10;
  c->m_max = 64;
  c->m_step = 5;
  c->max_substeps = 32;
}

size_t expdg_context_bytes(const expdg_config* cfg) {
  if (validate(cfg) != EXPDG_OK) return 0;
  const bool ff = cfg->prec == EXPDG_MIXED_FF, f32 = cfg->prec != EXPDG_FP64;
  size_t nelem = 1, np = 1;
  for (int d = 0; d < cfg->dim; ++d) {
    nelem *= (size_t)cfg->ne[d];
    np *= (size_t)(cfg->p + 1);
  }
  const size_t m = (cfg->eq == EXPDG_BURGERS) ? 1 : (size_t)cfg->dim + 2;
  const size_t N = m * nelem * np;
  const size_t ld = ((N + EXPDG_MAX_PHI + 63) / 64) * 64;
  const size_t gran = (size_t)2 << 20;
  auto r = [&](size_t b) { return ((b + gran - 1) / gran) * gran; };
  size_t total = 5 * r(N * sizeof(double));                 // q, q2, t2, in, out
  if (f32) total += r(N * sizeof(float));                            // FP32 operand
  if (f32) total += r(2 * N * sizeof(float));                         // float-float state
  if (f32 && !ff) total += EXPDG_MAX_PHI * r(N * sizeof(float));     // FP32 copies of b_1..b_P
  total += r(N * (f32 ? sizeof(float) : sizeof(double)));    // linearisation state
  const size_t nvec = 2 * (EXPDG_MAX_PHI + 1) + 4;          // c, b, w, rn, t1, t3
  total += nvec * (ff ? 2 * r(N * sizeof(float)) : r(N * sizeof(double)));
  const size_t nb = ld * (size_t)(cfg->m_max + 1);
  total += ff ? 2 * r(nb * sizeof(float)) : r(nb * sizeof(double));
  if (f32 && !ff) total += r(nb * sizeof(float));                     // FP32 shadow planes
  total += r(sizeof(KState)) + r(reduction_scratch_entries() * sizeof(double));
  return total;
}

// Tile class of the FP32 operator apply (mixed and float-float forms) for
// this context: the one asked for, or (EXPDG_TILE_AUTO) the fastest of the
// three on the context's own mesh, timed with CUDA events over five applies
// each after two warm-up applies, on zero data (the apply's time does not
// depend on the values).  The default class is kept unless another is 3 %
// faster.  Results are cached per mesh shape and form for the process.
std::mutex g_tile_mu;
std::map<std::vector<long>, int> g_tile_cache;

cudaError_t choose_tile(expdg_ctx* ctx) {
  const expdg_config& c = ctx->cfg;
  ctx->mesh.tile = 0;
  if (!ctx->f32op) return cudaSuccess;
  if (c.tile != EXPDG_TILE_AUTO) {
    ctx->mesh.tile = c.tile - 1;
    return cudaSuccess;
  }
  const std::vector<long> key = {c.dim, c.p,     c.eq,     c.flux,   c.bc,    c.kappa != 0.0 ? 1 : 0,
                                 c.ne[0], c.ne[1], c.ne[2], ctx->lin_form};
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tile_cache.find(key);
    if (it != g_tile_cache.end()) {
      ctx->mesh.tile = it->second;
      return cudaSuccess;
    }
  }
  const cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemsetAsync(ctx->d_z, 0, ctx->N * sizeof(float), s);
  DGArgs a = ctx->mesh;
  a.q = ctx->d_z;
  if (ctx->ff) {
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->U.h, 0, ctx->N * sizeof(float), s);
    a.v = ctx->U.h;
    a.out_h = ctx->U.h + ctx->ld;
    a.out_l = ctx->U.l + ctx->ld;
  } else {  // mixed form: the FP32 shadow plane in and out, as in its Arnoldi steps
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->U.h, 0, ctx->N * sizeof(float), s);
    a.v = ctx->U.h;
    a.out_h = ctx->U.h + ctx->ld;
  }
  if (e != cudaSuccess) return e;
  set_alpha(a, 1.0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  int best = 0;
  float best_ms = 0.0f;
  for (int tk = 0; tk < 3 && e == cudaSuccess; ++tk) {
    if (tk > 0 && tile_elems_per_block(ctx->NP, tk) == tile_elems_per_block(ctx->NP, 0)) continue;  // same kernel
    a.tile = tk;
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = launch_lin(ctx, a);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = launch_lin(ctx, a);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (tk == 0 || ms < 0.97f * best_ms)) {
      best = tk;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  ctx->mesh.tile = best;
  std::lock_guard<std::mutex> lk(g_tile_mu);
  g_tile_cache[key] = best;
  return cudaSuccess;
}

expdg_status expdg_create(const expdg_config* cfg, expdg_ctx** out) {
  if (!out) return EXPDG_EINVAL;
  *out = nullptr;
  if (validate(cfg) != EXPDG_OK) return EXPDG_EINVAL;
  expdg_ctx* ctx = new expdg_ctx();
  ctx->cfg = *cfg;
  for (int d = cfg->dim; d < 3; ++d) {
    ctx->cfg.ne[d] = 1;
    ctx->cfg.lo[d] = 0.0;
    ctx->cfg.hi[d] = 1.0;
  }
  cudaError_t e = cudaGetDevice(&ctx->dev);
  if (e != cudaSuccess) {
    delete ctx;
    return EXPDG_ECUDA;
  }
  ctx->ff = (cfg->prec == EXPDG_MIXED_FF);
  ctx->f32op = (cfg->prec != EXPDG_FP64);
  ctx->lin_form = ctx->ff ? DG_F32_FF : (ctx->f32op ? DG_F32_MX : DG_F64);
  const int p = cfg->p;
  ctx->M = (cfg->eq == EXPDG_BURGERS) ? 1 : cfg->dim + 2;
  ctx->NP = 1;
  for (int d = 0; d < cfg->dim; ++d) ctx->NP *= (p + 1);
  ctx->nelem = 1;
  for (int d = 0; d < cfg->dim; ++d) ctx->nelem *= (size_t)cfg->ne[d];
  if (ctx->nelem > (size_t)0x7fffffff / (size_t)ctx->NP) {
    delete ctx;
    return EXPDG_EINVAL;
  }
  ctx->N = (size_t)ctx->M * ctx->nelem * ctx->NP;
  ctx->ld = ((ctx->N + EXPDG_MAX_PHI + 63) / 64) * 64;  // 256-byte aligned vectors
  double D[(MAXP + 1) * (MAXP + 1)];
  build_lgl(p, ctx->lgl_r, ctx->lgl_w, D);
  fill_tab(ctx->tab, D, p, 1.0 / ctx->lgl_w[0]);
  DGArgs& m = ctx->mesh;
  std::memset(&m, 0, sizeof(m));
  for (int d = 0; d < 3; ++d) {
    m.ne[d] = ctx->cfg.ne[d];
    m.two_over_h[d] = make_cst(2.0 / ((ctx->cfg.hi[d] - ctx->cfg.lo[d]) / ctx->cfg.ne[d]));
  }
  m.nelem = (int)ctx->nelem;
  m.gamma = make_cst(cfg->gamma);
  m.stride = ctx->nelem * ctx->NP;
  m.kappa = make_cst(cfg->kappa);
  m.viscous = cfg->kappa != 0.0 ? 1 : 0;
  m.dirichlet = (cfg->bc == EXPDG_BC_DIRICHLET) ? 1 : 0;
  m.roe = (cfg->flux == EXPDG_FLUX_ROE) ? 1 : 0;

  const size_t N = ctx->N;
#define ALLOC(call)                         \
  do {                                      \
    if ((e = (call)) != cudaSuccess) {      \
      expdg_destroy(ctx);                   \
      cudaGetLastError();                   \
      return e == cudaErrorMemoryAllocation ? EXPDG_ENOMEM : EXPDG_ECUDA; \
    }                                       \
  } while (0)
  ALLOC(dalloc(ctx, &ctx->d_q, N));
  ALLOC(dalloc(ctx, &ctx->d_q2, N));
  ALLOC(dalloc(ctx, &ctx->d_t2, N));
  ALLOC(dalloc(ctx, &ctx->d_in, N));
  ALLOC(dalloc(ctx, &ctx->d_out, N));
  if (ctx->f32op) ALLOC(dalloc(ctx, &ctx->d_q32b, N));
  if (ctx->f32op) ALLOC(dalloc(ctx, &ctx->d_qfx, 2 * N));
  if (ctx->f32op && !ctx->ff)
    for (int i = 1; i <= EXPDG_MAX_PHI; ++i) ALLOC(dalloc(ctx, &ctx->d_bf[i], N));
  if (ctx->f32op) {
    float* z = nullptr;
    ALLOC(dalloc(ctx, &z, N));
    ctx->d_z = z;
  } else {
    double* z = nullptr;
    ALLOC(dalloc(ctx, &z, N));
    ctx->d_z = z;
  }
  for (int i = 0; i <= EXPDG_MAX_PHI; ++i) {
    ALLOC(alloc_vec(ctx, &ctx->c[i], N));
    ALLOC(alloc_vec(ctx, &ctx->b[i], N));
  }
  ALLOC(alloc_vec(ctx, &ctx->w, N));
  ALLOC(alloc_vec(ctx, &ctx->rn, N));
  ALLOC(alloc_vec(ctx, &ctx->t1, N));
  ALLOC(alloc_vec(ctx, &ctx->t3, N));
  ctx->U.ld = ctx->ld;
  const size_t nb = ctx->ld * (size_t)(cfg->m_max + 1);
  if (ctx->ff) {
    ALLOC(dalloc(ctx, &ctx->U.h, nb));
    ALLOC(dalloc(ctx, &ctx->U.l, nb));
  } else {
    ALLOC(dalloc(ctx, &ctx->U.d, nb));
    if (ctx->f32op) ALLOC(dalloc(ctx, &ctx->U.h, nb));  // mixed form: FP32 shadow planes
  }
  ALLOC(dalloc(ctx, &ctx->ks, 1));
  double* part = nullptr;
  ALLOC(dalloc(ctx, &part, reduction_scratch_entries()));
  ctx->part = part;
  void* hk = nullptr;
  ALLOC(cudaMallocHost(&hk, sizeof(KState)));
  ctx->h_ks = static_cast<KState*>(hk);
  std::memset(ctx->h_ks, 0, sizeof(KState));
  ALLOC(cudaStreamSynchronize(0));  // the zero-fills above are complete
  ALLOC(choose_tile(ctx));  // CTA size of the mixed-form operator apply

#undef ALLOC
  *out = ctx;
  return EXPDG_OK;
}

void expdg_destroy(expdg_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (void* p : ctx->allocs) cudaFree(p);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->h_ks) cudaFreeHost(ctx->h_ks);
  delete ctx;
}

expdg_status expdg_set_stream(expdg_ctx* ctx, void* stream) {
  if (!ctx) return EXPDG_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return EXPDG_OK;
}

size_t expdg_num_unknowns(const expdg_ctx* ctx) { return ctx ? ctx->N : 0; }
int expdg_tile_in_use(const expdg_ctx* ctx) { return ctx ? ctx->mesh.tile + 1 : 0; }
int expdg_num_fields(const expdg_ctx* ctx) { return ctx ? ctx->M : 0; }
size_t expdg_num_elements(const expdg_ctx* ctx) { return ctx ? ctx->nelem : 0; }
int expdg_nodes_per_element(const expdg_ctx* ctx) { return ctx ? ctx->NP : 0; }

namespace {
// x_d = lo_d + h_d (e_d + (r_i + 1)/2) in the canonical layout [d][e][n].
void fill_node_coords(const expdg_config& c, const double* r, double* xyz) {
  const int n1 = c.p + 1;
  size_t nelem = 1, np = 1;
  for (int d = 0; d < c.dim; ++d) {
    nelem *= (size_t)c.ne[d];
    np *= (size_t)n1;
  }
  for (int d = 0; d < c.dim; ++d) {
    const double h = (c.hi[d] - c.lo[d]) / c.ne[d];
    for (size_t e = 0; e < nelem; ++e) {
      size_t t = e;
      int ec[3] = {0, 0, 0};
      for (int k = 0; k < c.dim; ++k) {
        ec[k] = (int)(t % c.ne[k]);
        t /= c.ne[k];
      }
      for (size_t n = 0; n < np; ++n) {
        int ii[3] = {0, 0, 0};
        size_t tn = n;
        for (int k = 0; k < c.dim; ++k) {
          ii[k] = (int)(tn % n1);
          tn /= n1;
        }
        xyz[((size_t)d * nelem + e) * np + n] = c.lo[d] + h * (ec[d] + (r[ii[d]] + 1.0) / 2.0);
      }
    }
  }
}
}  // namespace

expdg_status expdg_node_coords(const expdg_ctx* ctx, double* xyz) {
  if (!ctx || !xyz) return EXPDG_EINVAL;
  fill_node_coords(ctx->cfg, ctx->lgl_r, xyz);
  return EXPDG_OK;
}

expdg_status expdg_config_node_coords(const expdg_config* cfg, double* xyz) {
  if (validate(cfg) != EXPDG_OK || !xyz) return EXPDG_EINVAL;
  double r[MAXP + 1], w[MAXP + 1], D[(MAXP + 1) * (MAXP + 1)];
  build_lgl(cfg->p, r, w, D);
  fill_node_coords(*cfg, r, xyz);
  return EXPDG_OK;
}

expdg_status expdg_set_source(expdg_ctx* ctx, const double* s) {
  if (!ctx) return EXPDG_EINVAL;
  if (!s) {
    ctx->has_src = false;
    return EXPDG_OK;
  }
  if (!ctx->d_src) {
    cudaError_t e = dalloc(ctx, &ctx->d_src, ctx->N);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, e == cudaErrorMemoryAllocation ? EXPDG_ENOMEM : EXPDG_ECUDA, "source allocation");
    }
  }
  if (check_ptrs(ctx, {s}) != EXPDG_OK) return EXPDG_EINVAL;
  const cudaMemcpyKind kind = is_device_ptr(ctx, s) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CU(ctx, cudaMemcpyAsync(ctx->d_src, s, ctx->N * sizeof(double), kind, ctx->stream));
  CU(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->has_src = true;
  return EXPDG_OK;
}

expdg_status expdg_residual(expdg_ctx* ctx, const double* q, double* r) {
  if (!ctx || !q || !r) return fail(ctx, EXPDG_EINVAL, "null argument");
  if (check_ptrs(ctx, {q, r}) != EXPDG_OK) return EXPDG_EINVAL;
  cudaError_t e;
  const double* qd = in_dev(ctx, q, ctx->d_in, ctx->N, &e);
  CU(ctx, e);
  const bool rdev = is_device_ptr(ctx, r);
  double* rd = rdev ? r : ctx->d_out;
  CU(ctx, cudaMemsetAsync(&ctx->ks->status, 0, sizeof(int), ctx->stream));
  if (ctx->ff) {
    CU(ctx, residual_into(ctx, qd, ctx->t1, 1.0));
    RUN(ctx, EXPDG_K_VECTOR, 16.0 * ctx->N, launch_ff_to_f64(rd, ctx->t1, ctx->N, ctx->stream));
  } else {
    CU(ctx, residual_into(ctx, qd, dvec(rd), 1.0));
  }
  if (!rdev) CU(ctx, cudaMemcpyAsync(r, rd, ctx->N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return readback(ctx);
}

expdg_status expdg_jv(expdg_ctx* ctx, const double* qt, const double* v, double* out) {
  if (!ctx || !qt || !v || !out) return fail(ctx, EXPDG_EINVAL, "null argument");
  if (check_ptrs(ctx, {qt, v, out}) != EXPDG_OK) return EXPDG_EINVAL;
  cudaError_t e;
  const double* qd = in_dev(ctx, qt, ctx->d_in, ctx->N, &e);
  CU(ctx, e);
  const double* vd = in_dev(ctx, v, ctx->d_t2, ctx->N, &e);
  CU(ctx, e);
  const bool odev = is_device_ptr(ctx, out);
  double* od = odev ? out : ctx->d_out;
  CU(ctx, linstate_into(ctx, qd));
  if (ctx->ff) {
    RUN(ctx, EXPDG_K_VECTOR, 12.0 * ctx->N, launch_to_f32(ctx->d_q32b, vd, ctx->N, ctx->stream));
    CU(ctx, jv_into(ctx, ctx->d_z, ctx->d_q32b, ctx->t1, 1.0));
    RUN(ctx, EXPDG_K_VECTOR, 16.0 * ctx->N, launch_ff_to_f64(od, ctx->t1, ctx->N, ctx->stream));
  } else if (ctx->f32op) {  // mixed form: FP32 input, FP64 output
    RUN(ctx, EXPDG_K_VECTOR, 12.0 * ctx->N, launch_to_f32(ctx->d_q32b, vd, ctx->N, ctx->stream));
    CU(ctx, jv_into(ctx, ctx->d_z, ctx->d_q32b, dvec(od), 1.0));
  } else {
    CU(ctx, jv_into(ctx, ctx->d_z, vd, dvec(od), 1.0));
  }
  if (!odev) CU(ctx, cudaMemcpyAsync(out, od, ctx->N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CU(ctx, cudaStreamSynchronize(ctx->stream));
  return EXPDG_OK;
}

expdg_status expdg_phi(expdg_ctx* ctx, const double* qt, double tau, const double* const* c, int P, double* out,
                       expdg_stats* stats, const expdg_trace_entry* replay, int nreplay, expdg_trace_entry* trace,
                       int trace_cap, int* ntrace) {
  if (!ctx || !qt || !out || P < 0 || P > EXPDG_MAX_PHI) return fail(ctx, EXPDG_EINVAL, "bad argument");
  if (!std::isfinite(tau)) return fail(ctx, EXPDG_EINVAL, "tau must be finite");
  if (check_ptrs(ctx, {qt, out}) != EXPDG_OK) return EXPDG_EINVAL;
  for (int i = 0; c && i <= P; ++i)
    if (check_ptrs(ctx, {c[i]}) != EXPDG_OK) return EXPDG_EINVAL;
  const size_t N = ctx->N;
  const cudaStream_t s = ctx->stream;
  cudaError_t e;
  const double* qd = in_dev(ctx, qt, ctx->d_q, N, &e);
  CU(ctx, e);
  bool has[EXPDG_MAX_PHI + 1] = {false, false, false, false};
  for (int i = 0; i <= P; ++i) {
    if (!c || !c[i]) continue;
    has[i] = true;
    const double* ci = in_dev(ctx, c[i], ctx->d_in, N, &e);
    CU(ctx, e);
    if (ctx->ff) {
      RUN(ctx, EXPDG_K_VECTOR, 16.0 * N, launch_f64_to_ff(ctx->c[i], ci, N, s));
    } else {
      CU(ctx, cudaMemcpyAsync(ctx->c[i].d, ci, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
  }
  CU(ctx, linstate_into(ctx, qd));
  const void* qt_T = ctx->d_z;
  const bool odev = is_device_ptr(ctx, out);
  double* od = odev ? out : ctx->d_out;
  expdg_stats st{};
  std::vector<expdg_trace_entry> tr;
  Replay rp;
  rp.e = replay;
  rp.n = nreplay;
  expdg_status r = phi_solve(ctx, qt_T, tau, has, P, null_vec(), dvec(od), 0, rp, &st, &tr);
  if (r != EXPDG_OK) return r;
  if (!odev) CU(ctx, cudaMemcpyAsync(out, od, N * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(ctx, cudaStreamSynchronize(s));
  if (stats) *stats = st;
  write_trace(tr, trace, trace_cap, ntrace);
  return EXPDG_OK;
}

expdg_status expdg_step(expdg_ctx* ctx, double* q, double dt, expdg_stats* stats, const expdg_trace_entry* replay,
                        int nreplay, expdg_trace_entry* trace, int trace_cap, int* ntrace) {
  if (!ctx || !q) return fail(ctx, EXPDG_EINVAL, "null argument");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, EXPDG_EINVAL, "the step size must be finite and > 0");
  if (check_ptrs(ctx, {q}) != EXPDG_OK) return EXPDG_EINVAL;
  const size_t N = ctx->N;
  const bool qdev = is_device_ptr(ctx, q);
  double* qd = qdev ? q : ctx->d_q;
  if (!qdev) CU(ctx, cudaMemcpyAsync(qd, q, N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  expdg_stats st{};
  std::vector<expdg_trace_entry> tr;
  Replay rp;
  rp.e = replay;
  rp.n = nreplay;
  expdg_status r = step_dev(ctx, qd, dt, rp, &st, &tr);
  if (r != EXPDG_OK) return r;
  if (!qdev) CU(ctx, cudaMemcpyAsync(q, qd, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  r = readback(ctx);
  if (r != EXPDG_OK) return r;
  if (stats) *stats = st;
  write_trace(tr, trace, trace_cap, ntrace);
  return EXPDG_OK;
}

expdg_status expdg_advance(expdg_ctx* ctx, double* q, double dt, int nsteps, expdg_stats* stats) {
  if (!ctx || !q || nsteps < 0) return fail(ctx, EXPDG_EINVAL, "bad argument");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, EXPDG_EINVAL, "the step size must be finite and > 0");
  if (check_ptrs(ctx, {q}) != EXPDG_OK) return EXPDG_EINVAL;
  const size_t N = ctx->N;
  const bool qdev = is_device_ptr(ctx, q);
  double* qd = qdev ? q : ctx->d_q;
  if (!qdev) CU(ctx, cudaMemcpyAsync(qd, q, N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  expdg_stats st{};
  Replay rp;
  // a solve's decisions depend only on its own inputs, not on earlier calls
  ctx->m_hint[0] = ctx->m_hint[1] = 0;
  ctx->hint_uses[0] = ctx->hint_uses[1] = 0;
  ctx->probe_next[0] = ctx->probe_next[1] = false;
  for (int k = 0; k < nsteps; ++k) {
    expdg_status r = step_dev(ctx, qd, dt, rp, &st, nullptr);
    if (r != EXPDG_OK) return r;
  }
  if (!qdev) CU(ctx, cudaMemcpyAsync(q, qd, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  expdg_status r = readback(ctx);
  if (r != EXPDG_OK) return r;
  if (stats) *stats = st;
  return EXPDG_OK;
}

expdg_status expdg_profile_enable(expdg_ctx* ctx, int on) {
  if (!ctx) return EXPDG_EINVAL;
  CU(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->prof_on = on != 0;
  for (auto& p : ctx->prof) p = expdg_kernel_prof{0, 0.0, 0.0};
  ctx->recs.clear();
  ctx->ev_used = 0;
  return EXPDG_OK;
}

expdg_status expdg_profile_get(expdg_ctx* ctx, expdg_kernel_prof* out, int reset) {
  if (!ctx || !out) return EXPDG_EINVAL;
  CU(ctx, cudaStreamSynchronize(ctx->stream));
  for (const auto& r : ctx->recs) {
    float ms = 0.f;
    CU(ctx, cudaEventElapsedTime(&ms, r.a, r.b));
    ctx->prof[r.cls].ms += ms;
  }
  ctx->recs.clear();
  ctx->ev_used = 0;
  for (int k = 0; k < EXPDG_K_COUNT; ++k) out[k] = ctx->prof[k];
  if (reset)
    for (auto& p : ctx->prof) p = expdg_kernel_prof{0, 0.0, 0.0};
  return EXPDG_OK;
}

const char* expdg_last_error(const expdg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

}  // extern "C"
