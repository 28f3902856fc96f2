// Level-kernel family: estimator EST_APPROX, bfloat16 increments with S in FP32 (AP_BF16S), packed draws (three lockstep samples per Philox word).
#include "kernels.h"
#include "level_kernel.cuh"

namespace mlmc {
cudaError_t launch_approx_bf16s_p3(int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                      const LaunchArgs &a, int *occ) {
  return launch_family<EST_APPROX, XP_F32, AP_BF16S, 3>(scheme, pc, grid, block, smem, st, a, occ);
}
}  // namespace mlmc
