// Merged nested launch (approximate packed, approximate one sample per thread
// and correction chunks in one grid) for the 32-bit fast fixed-point datapath,
// Euler-Maruyama, terminal payoffs.
#include "kernels.h"
#include "level_kernel.cuh"

namespace mlmc {
cudaError_t launch_nested_fx32(int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               const LaunchArgs &a, int *occ) {
  if (scheme != 0 || pc != PC_TERMINAL || occ || a.dyn || a.dump) return cudaErrorInvalidValue;
  auto k = nested_kernel<AP_FX32, 0, PC_TERMINAL>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}
}  // namespace mlmc
