// DG operator kernels with the Roe flux (Euler), instantiated for dimension 2.
#include "jv32.cuh"

namespace expdg {

cudaError_t launch_dg_roe_2d(bool linear, int form, int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  return launch_dg_dim<2, EXPDG_EULER, true>(linear, form, p, a, t, s);
}

cudaError_t launch_dg_roe_fx_2d(int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  return launch_dg_fx_dim<2, EXPDG_EULER, true>(p, a, t, s);
}

}  // namespace expdg
