// DG operator kernels instantiated for dimension 3.
#include "dg_impl.cuh"

namespace expdg {

cudaError_t launch_dg_3d(bool linear, bool fp32, int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s) {

  if (eq == EXPDG_EULER) return launch_dg_dim<3, EXPDG_EULER>(linear, fp32, p, a, t, s);
  return cudaErrorInvalidValue;
}

}  // namespace expdg
