// Table-construction and helper launches (tables.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "item.h"

namespace mlmc {

enum Rep : int { REP_FP64 = 0, REP_FP32 = 1, REP_FP16 = 2, REP_BF16 = 3, REP_FIXED = 4 };

struct RoundKeys;
cudaError_t launch_m1_table(int d, double *out, cudaStream_t st);
cudaError_t launch_m1_convert(const double *z, int n, int rep, int fZ, void *out, cudaStream_t st);
cudaError_t launch_m1_signed(const double *z, int d, int rep, int fZ, void *out, cudaStream_t st);
cudaError_t launch_table_values(int method, int d, int rep, int fZ, const void *tab, double *out,
                                cudaStream_t st);
cudaError_t launch_philox(const uint4 *ctr, uint64_t n, const RoundKeys &rk, uint4 *out, cudaStream_t st);

}  // namespace mlmc
