// DG operator kernels instantiated for dimension 3.
#include "jv32.cuh"

namespace expdg {

cudaError_t launch_dg_3d(bool linear, int form, int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  if (eq == EXPDG_EULER && a.roe) return launch_dg_roe_3d(linear, form, p, a, t, s);
  if (eq == EXPDG_EULER) return launch_dg_dim<3, EXPDG_EULER>(linear, form, p, a, t, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_linstate_3d(int eq, bool fp32, const double* q, void* z, size_t stride, double gamma, int roe,
                               float* qfx, cudaStream_t s) {
  if (eq == EXPDG_EULER) return launch_linstate_dim<3, EXPDG_EULER>(fp32, q, z, stride, gamma, roe, qfx, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_dg_fx_3d(int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  if (eq == EXPDG_EULER && a.roe) return launch_dg_roe_fx_3d(p, a, t, s);
  if (eq == EXPDG_EULER) return launch_dg_fx_dim<3, EXPDG_EULER>(p, a, t, s);
  return cudaErrorInvalidValue;
}

}  // namespace expdg
