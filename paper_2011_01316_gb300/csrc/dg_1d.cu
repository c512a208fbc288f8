// DG operator kernels instantiated for dimension 1.
#include "dg_impl.cuh"

namespace expdg {

cudaError_t launch_dg_1d(bool linear, bool fp32, int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  if (eq == EXPDG_BURGERS) return launch_dg_dim<1, EXPDG_BURGERS>(linear, fp32, p, a, t, s);
  if (eq == EXPDG_EULER) return launch_dg_dim<1, EXPDG_EULER>(linear, fp32, p, a, t, s);
  return cudaErrorInvalidValue;
}

}  // namespace expdg
