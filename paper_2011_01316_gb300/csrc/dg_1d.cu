// DG operator kernels instantiated for dimension 1.
#include "jv32.cuh"

namespace expdg {

cudaError_t launch_dg_1d(bool linear, int form, int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  if (eq == EXPDG_BURGERS) return launch_dg_dim<1, EXPDG_BURGERS>(linear, form, p, a, t, s);
  if (eq == EXPDG_EULER && a.roe) return launch_dg_roe_1d(linear, form, p, a, t, s);
  if (eq == EXPDG_EULER) return launch_dg_dim<1, EXPDG_EULER>(linear, form, p, a, t, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_linstate_1d(int eq, bool fp32, const double* q, void* z, size_t stride, double gamma, int roe,
                               float* qfx, cudaStream_t s) {
  if (eq == EXPDG_BURGERS) return launch_linstate_dim<1, EXPDG_BURGERS>(fp32, q, z, stride, gamma, roe, qfx, s);
  if (eq == EXPDG_EULER) return launch_linstate_dim<1, EXPDG_EULER>(fp32, q, z, stride, gamma, roe, qfx, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_dg_fx_1d(int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  if (eq == EXPDG_BURGERS) return launch_dg_fx_dim<1, EXPDG_BURGERS>(p, a, t, s);
  if (eq == EXPDG_EULER && a.roe) return launch_dg_roe_fx_1d(p, a, t, s);
  if (eq == EXPDG_EULER) return launch_dg_fx_dim<1, EXPDG_EULER>(p, a, t, s);
  return cudaErrorInvalidValue;
}

}  // namespace expdg
