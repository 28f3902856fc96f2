// Device construction of the approximate inverse-CDF tables (Sec. 3.1 and
// 3.3) and a Philox evaluation kernel used for parity checks.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "device_common.cuh"
#include "tables.h"

namespace mlmc {

// Method 1 (Sec. 3.1): Z_k = 2^d * integral of Phi^{-1} over [k 2^-d, (k+1) 2^-d]
// = 2^d (phi(a) - phi(b)) with a = Phi^{-1}(k 2^-d), b = Phi^{-1}((k+1) 2^-d),
// evaluated as 2^d phi(b) expm1((b - a)(b + a) / 2) to avoid cancellation
// (phi(a) = phi(b) exp((b^2 - a^2)/2)); phi(Phi^{-1}(0)) = 0 for k = 0.
__global__ void m1_table_kernel(int d, double *out) {
  const int half = 1 << (d - 1);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= half) return;
  const double scale = ldexp(1.0, d);
  const double b = (k + 1 == half) ? 0.0 : normcdfinv((double)(k + 1) / scale);
  const double inv_sqrt_2pi = 0.39894228040143267794;
  const double phib = exp(-0.5 * b * b) * inv_sqrt_2pi;
  double v;
  if (k == 0) {
    v = -scale * phib;
  } else {
    const double a = normcdfinv((double)k / scale);
    v = scale * phib * expm1(0.5 * (b - a) * (b + a));
  }
  out[k] = v;
}

// Representations of the Method-1 table used by the kernels.
__global__ void m1_convert_kernel(const double *z, int n, int rep, int fZ, void *out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double v = z[k];
  switch (rep) {
    case REP_FP32: ((float *)out)[k] = (float)v; break;
    case REP_FP16: ((uint16_t *)out)[k] = __half_as_ushort(__double2half(v)); break;
    case REP_BF16: ((uint16_t *)out)[k] = __bfloat16_as_ushort(__double2bfloat16(v)); break;
    case REP_FIXED: ((int32_t *)out)[k] = (int32_t)floor(ldexp(v, fZ) + 0.5); break;
    default: ((double *)out)[k] = v; break;
  }
}

// Method-1 table over all 2^d values of j (the top d bits of J), as the level
// kernels index it: entry j < 2^(d-1) is the rounded Z_j, entry j >= 2^(d-1)
// the negated rounded Z_{2^d-1-j} (the mirrored interval, Sec. 3.1).
__global__ void m1_signed_kernel(const double *z, int d, int rep, int fZ, void *out) {
  const int half = 1 << (d - 1);
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 2 * half) return;
  const bool neg = j >= half;
  const double v = z[neg ? 2 * half - 1 - j : j];
  switch (rep) {
    case REP_FP16: {
      const __half h = __double2half(v);
      ((uint16_t *)out)[j] = __half_as_ushort(neg ? __hneg(h) : h);
      break;
    }
    case REP_BF16: {
      const __nv_bfloat16 h = __double2bfloat16(v);
      ((uint16_t *)out)[j] = __bfloat16_as_ushort(neg ? __hneg(h) : h);
      break;
    }
    case REP_FIXED: {
      const int32_t q = (int32_t)floor(ldexp(v, fZ) + 0.5);
      ((int32_t *)out)[j] = neg ? -q : q;
      break;
    }
    default: {
      const float f = (float)v;
      ((float *)out)[j] = neg ? -f : f;
      break;
    }
  }
}

// Values of every table index as the level kernels see them (for parity tests).
__global__ void table_values_kernel(int method, int d, int rep, int fZ, const void *tab, double *out) {
  const int n = 1 << (d - 1);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  if (method == 1) {
    switch (rep) {
      case REP_FP32: out[k] = ((const float *)tab)[k]; break;
      case REP_FP16: out[k] = __half2float(__ushort_as_half(((const uint16_t *)tab)[k])); break;
      case REP_BF16: out[k] = __bfloat162float(__ushort_as_bfloat16(((const uint16_t *)tab)[k])); break;
      case REP_FIXED: out[k] = ldexp((double)((const int32_t *)tab)[k], -fZ); break;
      default: out[k] = ((const double *)tab)[k]; break;
    }
    return;
  }
  const M3Coef *m3 = (const M3Coef *)tab;
  const int c = m3_class((uint32_t)k);
  if (rep == REP_FIXED) {
    const int64_t t = m3->A[c] + m3->B[c] * (int64_t)k;
    const int sh = M3_FRAC - fZ;
    out[k] = ldexp((double)((t + ((int64_t)1 << (sh - 1))) >> sh), -fZ);
    return;
  }
  const float v = fmaf(m3->b[c], (float)k, m3->a[c]);
  if (rep == REP_FP16) out[k] = __half2float(__float2half_rn(v));
  else if (rep == REP_BF16) out[k] = __bfloat162float(__float2bfloat16_rn(v));
  else out[k] = v;
}

__global__ void philox_kernel(const uint4 *ctr, uint64_t n, RoundKeys rk, uint4 *out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], rk);
}

cudaError_t launch_m1_table(int d, double *out, cudaStream_t st) {
  const int n = 1 << (d - 1);
  m1_table_kernel<<<(n + 127) / 128, 128, 0, st>>>(d, out);
  return cudaGetLastError();
}
cudaError_t launch_m1_convert(const double *z, int n, int rep, int fZ, void *out, cudaStream_t st) {
  m1_convert_kernel<<<(n + 127) / 128, 128, 0, st>>>(z, n, rep, fZ, out);
  return cudaGetLastError();
}
cudaError_t launch_m1_signed(const double *z, int d, int rep, int fZ, void *out, cudaStream_t st) {
  const int n = 1 << d;
  m1_signed_kernel<<<(n + 127) / 128, 128, 0, st>>>(z, d, rep, fZ, out);
  return cudaGetLastError();
}
cudaError_t launch_table_values(int method, int d, int rep, int fZ, const void *tab, double *out,
                                cudaStream_t st) {
  const int n = 1 << (d - 1);
  table_values_kernel<<<(n + 127) / 128, 128, 0, st>>>(method, d, rep, fZ, tab, out);
  return cudaGetLastError();
}
cudaError_t launch_philox(const uint4 *ctr, uint64_t n, const RoundKeys &rk, uint4 *out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctr, n, rk, out);
  return cudaGetLastError();
}

}  // namespace mlmc
