// Level-kernel family: estimator EST_CORR, bfloat16 increments with S in FP32 (AP_BF16S).
#include "kernels.h"
#include "level_kernel.cuh"

namespace mlmc {
cudaError_t launch_corr_bf16s(int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                      const LaunchArgs &a, int *occ) {
  return launch_family<EST_CORR, XP_F32, AP_BF16S, 1>(scheme, pc, grid, block, smem, st, a, occ);
}
}  // namespace mlmc
