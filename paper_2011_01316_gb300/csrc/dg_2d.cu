// DG operator kernels instantiated for dimension 2.
#include "dg_impl.cuh"

namespace expdg {

cudaError_t launch_dg_2d(bool linear, bool fp32, int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s) {

  if (eq == EXPDG_EULER) return launch_dg_dim<2, EXPDG_EULER>(linear, fp32, p, a, t, s);
  return cudaErrorInvalidValue;
}

}  // namespace expdg
