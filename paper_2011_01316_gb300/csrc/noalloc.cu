// expdg_residual_noalloc: the residual R(q) without a context and without any
// device allocation, for callers that cannot allocate device memory.
//
// Its scratch - the float-float copy of the state (mixed and float-float
// forms), the float-float output of the float-float form, and the
// non-physical-state flag of every form -
// lives in the file-scope arrays below.  Every GPU that loads this library
// holds them (about 8 MiB) until the process exits.
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tables.h"

namespace {

constexpr size_t kMaxUnknowns = (size_t)1 << 19;  // EXPDG_NOALLOC_MAX_UNKNOWNS
constexpr int kMaxDevices = 64;

// [0, 2 kMax): float-float state (interleaved pairs); [2 kMax, 3 kMax): residual
// hi; [3 kMax, 4 kMax): residual lo
static __device__ __align__(256) float g_scratch[4 * kMaxUnknowns];
static __device__ __align__(256) int g_status[64];

// Device addresses of the arrays, per device ordinal (the host-side names of
// g_scratch / g_status are stand-ins, not device addresses).  Looked up once
// per device, with that device current, under a std::call_once per device, so
// first calls from several host threads do not race on the cache.
struct Addr {
  float* scratch;
  int* status;
  cudaError_t err;
};
Addr g_addr[kMaxDevices];
std::once_flag g_once[kMaxDevices];

cudaError_t device_addresses(int dev, Addr** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  Addr& a = g_addr[dev];
  std::call_once(g_once[dev], [&a] {
    void* p = nullptr;
    a.err = cudaGetSymbolAddress(&p, g_scratch);
    a.scratch = static_cast<float*>(p);
    if (a.err == cudaSuccess) {
      a.err = cudaGetSymbolAddress(&p, g_status);
      a.status = static_cast<int*>(p);
    }
  });
  if (a.err != cudaSuccess) return a.err;
  *out = &a;
  return cudaSuccess;
}

// Memory the current device reaches directly: its own device memory, or
// managed memory.  Host memory and another device's memory are rejected (the
// kernels would dereference them without access).
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at{};
  if (p == nullptr || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" expdg_status expdg_residual_noalloc(const expdg_config* cfg, const double* q, double* r,
                                               void* cuda_stream) {
  using namespace expdg;
  if (!cfg || !q || !r) return EXPDG_EINVAL;
  const int dim = cfg->dim, p = cfg->p;
  if (dim < 1 || dim > 3 || p < 1 || p > EXPDG_MAX_ORDER) return EXPDG_EINVAL;
  if (cfg->eq != EXPDG_BURGERS && cfg->eq != EXPDG_EULER) return EXPDG_EINVAL;
  if (cfg->eq == EXPDG_BURGERS && dim != 1) return EXPDG_EINVAL;
  if (cfg->eq == EXPDG_EULER && !(cfg->gamma > 1.0)) return EXPDG_EINVAL;
  if (cfg->prec != EXPDG_FP64 && cfg->prec != EXPDG_MIXED && cfg->prec != EXPDG_MIXED_FF) return EXPDG_EINVAL;
  if (!(cfg->kappa >= 0.0) || (cfg->bc != EXPDG_BC_PERIODIC && cfg->bc != EXPDG_BC_DIRICHLET)) return EXPDG_EINVAL;
  if ((cfg->kappa > 0.0 || cfg->bc != EXPDG_BC_PERIODIC) && cfg->eq != EXPDG_BURGERS) return EXPDG_EINVAL;
  if (cfg->flux != EXPDG_FLUX_LF && (cfg->flux != EXPDG_FLUX_ROE || cfg->eq != EXPDG_EULER)) return EXPDG_EINVAL;
  size_t nelem = 1;
  int np = 1;
  for (int d = 0; d < dim; ++d) {
    if (cfg->ne[d] < 1 || !(cfg->hi[d] > cfg->lo[d])) return EXPDG_EINVAL;
    nelem *= (size_t)cfg->ne[d];
    np *= p + 1;
  }
  const int m = (cfg->eq == EXPDG_BURGERS) ? 1 : dim + 2;
  if (nelem > (size_t)0x7fffffff / (size_t)np) return EXPDG_EINVAL;
  const size_t N = (size_t)m * nelem * np;
  const bool ffr = cfg->prec != EXPDG_FP64;  // float-float residual: needs the scratch
  const bool ffo = cfg->prec == EXPDG_MIXED_FF;  // its float-float output (else FP64, into r)
  if (ffr && N > kMaxUnknowns) return EXPDG_EINVAL;  // beyond the static scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EXPDG_ECUDA;
  if (!on_device(q, dev) || !on_device(r, dev)) return EXPDG_EINVAL;

  Addr* ad = nullptr;
  if (device_addresses(dev, &ad) != cudaSuccess) return EXPDG_ECUDA;
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  Tab tab{};
  double rr[MAXP + 1], ww[MAXP + 1], D[(MAXP + 1) * (MAXP + 1)];
  build_lgl(p, rr, ww, D);
  fill_tab(tab, D, p, 1.0 / ww[0]);
  DGArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int d = 0; d < 3; ++d) {
    const bool used = d < dim;
    a.ne[d] = used ? cfg->ne[d] : 1;
    a.two_over_h[d] = make_cst(used ? 2.0 / ((cfg->hi[d] - cfg->lo[d]) / cfg->ne[d]) : 2.0);
  }
  a.nelem = (int)nelem;
  a.gamma = make_cst(cfg->gamma);
  a.kappa = make_cst(cfg->kappa);
  a.viscous = cfg->kappa != 0.0 ? 1 : 0;
  a.dirichlet = (cfg->bc == EXPDG_BC_DIRICHLET) ? 1 : 0;
  a.roe = (cfg->flux == EXPDG_FLUX_ROE) ? 1 : 0;
  a.stride = nelem * np;
  a.alpha = 1.0;
  a.alpha_h = 1.0f;
  a.alpha_l = 0.0f;
  a.status = ad->status;

  // the status word keeps the previous call's value: clear it first
  if (cudaMemsetAsync(ad->status, 0, sizeof(int), s) != cudaSuccess) return EXPDG_ECUDA;
  float* qfx = ad->scratch;
  float* rh = ad->scratch + 2 * kMaxUnknowns;
  float* rl = ad->scratch + 3 * kMaxUnknowns;
  cudaError_t e = cudaSuccess;
  if (ffr) {  // float-float residual, as expdg_residual computes it in the FP32-operator forms
    e = launch_f64_to_fx(qfx, q, N, s);
    a.q = qfx;
    if (ffo) {
      a.out_h = rh;
      a.out_l = rl;
    } else {
      a.out = r;
    }
    if (e == cudaSuccess) {
      if (dim == 1)
        e = launch_dg_fx_1d(cfg->eq, p, a, tab, s);
      else if (dim == 2)
        e = launch_dg_fx_2d(cfg->eq, p, a, tab, s);
      else
        e = launch_dg_fx_3d(cfg->eq, p, a, tab, s);
    }
  } else {  // the FP64 residual (FP64 form): in place, no scratch
    a.q = q;
    a.out = r;
    if (dim == 1)
      e = launch_dg_1d(false, DG_F64, cfg->eq, p, a, tab, s);
    else if (dim == 2)
      e = launch_dg_2d(false, DG_F64, cfg->eq, p, a, tab, s);
    else
      e = launch_dg_3d(false, DG_F64, cfg->eq, p, a, tab, s);
  }
  if (e == cudaSuccess && ffo) {
    Vec v{};
    v.h = rh;
    v.l = rl;
    e = launch_ff_to_f64(r, v, N, s);
  }
  if (e != cudaSuccess) return EXPDG_ECUDA;
  int flag = 0;
  if (cudaMemcpyAsync(&flag, ad->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return EXPDG_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return EXPDG_ECUDA;
  return (flag & 1) ? EXPDG_ENONPHYSICAL : EXPDG_OK;
}
