// Level-kernel family: estimator EST_APPROX, binary16 increments with S in FP32 (AP_F16S).
#include "kernels.h"
#include "level_kernel.cuh"

namespace mlmc {
cudaError_t launch_approx_f16s(int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                      const LaunchArgs &a, int *occ) {
  return launch_family<EST_APPROX, XP_F32, AP_F16S, 1>(scheme, pc, grid, block, smem, st, a, occ);
}
}  // namespace mlmc
