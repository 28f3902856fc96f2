// mlmc_exact_normal_f32: the FP32 exact Normal of the level kernels
// (exact_normal_f32, Sec. 3.1) for caller-given words J.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "host_api.h"
#include "mlmc.h"

using namespace mlmc;

namespace {

__global__ void exact_normal_kernel(const uint32_t *J, float *z, uint64_t n) {
  __shared__ float4 tab[PHI_INV_PARTS];
  for (int k = threadIdx.x; k < PHI_INV_PARTS; k += blockDim.x) tab[k] = k_phi_inv[k];
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    z[i] = exact_normal_f32(J[i], tab);
}

}  // namespace

using namespace mlmc_host;

extern "C" {

mlmc_status mlmc_exact_normal_f32(const uint32_t *J, float *z, uint64_t n, void *stream) {
  MLMC_API_LOCK();
  if (n == 0) return MLMC_OK;
  if (!J || !z) return MLMC_EINVAL;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  const uint64_t blocks = (n + 255) / 256;
  exact_normal_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(J, z, n);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
    return MLMC_ECUDA;
  return MLMC_OK;
}

}  // extern "C"
