// Level-kernel family: estimator EST_EXACT, exact precision XP_F32, approximate arithmetic AP_NONE.
#include "kernels.h"
#include "level_kernel.cuh"

namespace mlmc {
cudaError_t launch_exact_f32(int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                      const LaunchArgs &a, int *occ) {
  return launch_family<EST_EXACT, XP_F32, AP_NONE>(scheme, pc, grid, block, smem, st, a, occ);
}
}  // namespace mlmc
