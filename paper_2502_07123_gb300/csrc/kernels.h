// Launch entry points of the level-kernel families (one translation unit each).
#pragma once
#include <cuda_runtime.h>

namespace mlmc {
struct LaunchArgs;
// Launch one level kernel of the family for (scheme, payoff class).  With
// occ != nullptr nothing is launched: *occ receives the resident CTAs per SM of
// the device-scheduled kernel (level_kernel_dyn) for this block and smem size.
#define MLMC_FAMILY(name)                                                                                      \
  cudaError_t name(int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st, const LaunchArgs &a, \
                   int *occ);
MLMC_FAMILY(launch_exact_f32)
MLMC_FAMILY(launch_exact_f64)
MLMC_FAMILY(launch_approx_fixed)
MLMC_FAMILY(launch_approx_f16)
MLMC_FAMILY(launch_approx_bf16)
MLMC_FAMILY(launch_corr_fixed)
MLMC_FAMILY(launch_corr_f16)
MLMC_FAMILY(launch_corr_bf16)
MLMC_FAMILY(launch_approx_fx32)
MLMC_FAMILY(launch_approx_fx64)
MLMC_FAMILY(launch_corr_fx32)
MLMC_FAMILY(launch_corr_fx64)
MLMC_FAMILY(launch_approx_fixed_p3)
MLMC_FAMILY(launch_approx_f16_p3)
MLMC_FAMILY(launch_approx_bf16_p3)
MLMC_FAMILY(launch_approx_fx32_p3)
MLMC_FAMILY(launch_approx_fx64_p3)
// families 17 / 24: merged nested launch of families 15, 8 and 10 (Euler-Maruyama,
// terminal payoffs; per-item kind in ItemDesc::kind); 24: pre-scaled sum1 form
cudaError_t launch_nested_fx32(int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               const LaunchArgs &a, int *occ, bool pre);
// families 18-23: binary16 / bfloat16 increments with S in FP32
MLMC_FAMILY(launch_approx_f16s)
MLMC_FAMILY(launch_approx_bf16s)
MLMC_FAMILY(launch_corr_f16s)
MLMC_FAMILY(launch_corr_bf16s)
MLMC_FAMILY(launch_approx_f16s_p3)
MLMC_FAMILY(launch_approx_bf16s_p3)
#undef MLMC_FAMILY
}  // namespace mlmc
