// Level-kernel family: estimator EST_APPROX, exact precision XP_F32, approximate arithmetic AP_FX64.
#include "kernels.h"
#include "level_kernel.cuh"

namespace mlmc {
cudaError_t launch_approx_fx64(int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                      const LaunchArgs &a, int *occ) {
  return launch_family<EST_APPROX, XP_F32, AP_FX64>(scheme, pc, grid, block, smem, st, a, occ);
}
}  // namespace mlmc
