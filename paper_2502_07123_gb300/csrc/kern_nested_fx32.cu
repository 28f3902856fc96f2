// Merged nested launch (approximate packed, approximate one sample per thread
// and correction chunks in one grid) for the 32-bit fast fixed-point datapath,
// Euler-Maruyama, terminal payoffs; pre: the pre-scaled sum1 form (family 24).
#include "kernels.h"
#include "level_kernel.cuh"

namespace mlmc {
cudaError_t launch_nested_fx32(int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               const LaunchArgs &a, int *occ, bool pre) {
  if (scheme != 0 || pc != PC_TERMINAL || occ || a.dyn || a.dump) return cudaErrorInvalidValue;
  auto k = pre ? nested_kernel<AP_FX32, 0, PC_TERMINAL, true> : nested_kernel<AP_FX32, 0, PC_TERMINAL, false>;
  // above 48 KB of dynamic plus static shared memory (the static part holds
  // up to about 8.6 KB: the inverse-Normal cubics) the kernel must opt in
  if (smem > 32 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}
}  // namespace mlmc
