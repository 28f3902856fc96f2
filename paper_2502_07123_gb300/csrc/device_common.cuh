// Device building blocks of the level kernels: Philox4x32-10, the exact and
// approximate Normal maps of Sec. 3, fixed-point re-quantisation (Sec. 4.1)
// and 128-bit integer accumulation.
#pragma once
#include "phi_inv_table.h"
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "item.h"

namespace mlmc {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each with two
// 32x32->64 products by the published multipliers; the round keys
// (key + r * Weyl increment) are precomputed on the host.
constexpr uint32_t PHILOX_M0 = 0xD2511F53u;
constexpr uint32_t PHILOX_M1 = 0xCD9E8D57u;
constexpr uint32_t PHILOX_W0 = 0x9E3779B9u;
constexpr uint32_t PHILOX_W1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys &rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)PHILOX_M0 * c.x;
    const uint64_t p1 = (uint64_t)PHILOX_M1 * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk.k[2 * r], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ rk.k[2 * r + 1], (uint32_t)p0);
  }
  return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4 &w, int k) {
  return k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
}

// Exact Normal Z = Phi^{-1}(2^-32 (J + 1/2)) in single precision (Sec. 3.1).
// The upper half uses Phi^{-1}(1 - u) = -Phi^{-1}(u): with J' = J or ~J below
// 2^31, u = 2^-32 (J' + 1/2) (J' rounded to nearest as a float) lies in
// [2^-33, 1/2].  Phi^{-1}(u) is the cubic of u's part (phi_inv_table.h; tab:
// that table in shared memory): u's exponent and the top four bits of its
// significand pick one of 512 parts of [2^-33, 1/2) (the 513th is u = 1/2),
// the other 19 bits are the position t in [0, 1) within it.  Error: about
// 1e-7 (1 + |Z|), unbiased (round to nearest).
__device__ __forceinline__ float exact_normal_f32(uint32_t J, const float4 *tab) {
  const uint32_t m = (uint32_t)((int32_t)J >> 31);
  const float u = fmaf(__uint2float_rn(J ^ m), 0x1p-32f, 0x1p-33f);
  const uint32_t b = __float_as_uint(u);
  const float4 c = tab[(b >> 19) - (94u << 4)];   // exponent field of 2^-33 is 94
  const float t = __uint_as_float(((b << 4) & 0x7FFFF0u) | 0x3F800000u) - 1.0f;
  const float z = fmaf(fmaf(fmaf(c.w, t, c.z), t, c.y), t, c.x);
  return __int_as_float(__float_as_int(z) ^ (int)(m & 0x80000000u));
}

__device__ __forceinline__ double exact_normal_f64(uint32_t J) {
  const uint32_t m = (uint32_t)((int32_t)J >> 31);
  const double u = ((double)(J ^ m) + 0.5) * 0x1p-32;
  const double z = normcdfinv(u);
  return m ? -z : z;
}

// Table index of the approximate Normal (Sec. 3.1): j = top d bits of J; the
// upper half (leading bit of j set) mirrors the index and flips the sign, so
// Z~ is the mean of Phi^{-1} over the 2^-d interval containing U.
struct ApproxIndex {
  uint32_t idx;
  bool neg;
};
__device__ __forceinline__ ApproxIndex approx_index(uint32_t J, int d) {
  const uint32_t j = J >> (32 - d);
  const uint32_t m = 0u - (j >> (d - 1));
  return ApproxIndex{(j ^ m) & ((1u << (d - 1)) - 1u), m != 0u};
}

// Method-3 class of a table index: {0,1} -> 0, [2^c, 2^(c+1)) -> c.
__device__ __forceinline__ int m3_class(uint32_t idx) {
  return 31 - __clz(idx | 1u);
}

// Fixed point: exact re-expression and rounding (ties toward +inf), saturation.
__device__ __forceinline__ int64_t requant(int64_t x, const Requant &q) {
  const int64_t y = (int64_t)((uint64_t)x << q.ls) + q.radd;
  return y >> q.rs;
}
__device__ __forceinline__ int64_t saturate(int64_t x, int64_t lim, uint32_t &sat) {
  const int64_t y = x > lim ? lim : (x < -lim ? -lim : x);
  sat |= (uint32_t)(y != x);
  return y;
}

// Half-precision helpers: one IEEE rounding per operation, never fused.
template <class H> struct HalfOps;
template <> struct HalfOps<__half> {
  static __device__ __forceinline__ __half mul(__half a, __half b) { return __hmul_rn(a, b); }
  static __device__ __forceinline__ __half add(__half a, __half b) { return __hadd_rn(a, b); }
  static __device__ __forceinline__ __half sub(__half a, __half b) { return __hsub_rn(a, b); }
  static __device__ __forceinline__ float to_f(__half a) { return __half2float(a); }
  static __device__ __forceinline__ __half from_bits(uint16_t b) { return __ushort_as_half(b); }
  static __device__ __forceinline__ __half from_f(float x) { return __float2half_rn(x); }
  static __device__ __forceinline__ __half neg(__half a) { return __hneg(a); }
};
template <> struct HalfOps<__nv_bfloat16> {
  static __device__ __forceinline__ __nv_bfloat16 mul(__nv_bfloat16 a, __nv_bfloat16 b) { return __hmul_rn(a, b); }
  static __device__ __forceinline__ __nv_bfloat16 add(__nv_bfloat16 a, __nv_bfloat16 b) { return __hadd_rn(a, b); }
  static __device__ __forceinline__ __nv_bfloat16 sub(__nv_bfloat16 a, __nv_bfloat16 b) { return __hsub_rn(a, b); }
  static __device__ __forceinline__ float to_f(__nv_bfloat16 a) { return __bfloat162float(a); }
  static __device__ __forceinline__ __nv_bfloat16 from_bits(uint16_t b) { return __ushort_as_bfloat16(b); }
  static __device__ __forceinline__ __nv_bfloat16 from_f(float x) { return __float2bfloat16_rn(x); }
  static __device__ __forceinline__ __nv_bfloat16 neg(__nv_bfloat16 a) { return __hneg(a); }
};

// Paired (x2) form: one instruction rounds both halves of a 32-bit register,
// each exactly as the scalar operation of HalfOps would.
template <class H> struct HalfOps2;
template <> struct HalfOps2<__half> {
  using T = __half2;
  static __device__ __forceinline__ T mul(T a, T b) { return __hmul2_rn(a, b); }
  static __device__ __forceinline__ T add(T a, T b) { return __hadd2_rn(a, b); }
  static __device__ __forceinline__ T sub(T a, T b) { return __hsub2_rn(a, b); }
  static __device__ __forceinline__ T pack(__half lo, __half hi) { return __halves2half2(lo, hi); }
  static __device__ __forceinline__ T splat(__half a) { return __half2half2(a); }
  static __device__ __forceinline__ __half lo(T a) { return __low2half(a); }
  static __device__ __forceinline__ __half hi(T a) { return __high2half(a); }
};
template <> struct HalfOps2<__nv_bfloat16> {
  using T = __nv_bfloat162;
  static __device__ __forceinline__ T mul(T a, T b) { return __hmul2_rn(a, b); }
  static __device__ __forceinline__ T add(T a, T b) { return __hadd2_rn(a, b); }
  static __device__ __forceinline__ T sub(T a, T b) { return __hsub2_rn(a, b); }
  static __device__ __forceinline__ T pack(__nv_bfloat16 lo, __nv_bfloat16 hi) { return __halves2bfloat162(lo, hi); }
  static __device__ __forceinline__ T splat(__nv_bfloat16 a) { return __bfloat162bfloat162(a); }
  static __device__ __forceinline__ __nv_bfloat16 lo(T a) { return __low2bfloat16(a); }
  static __device__ __forceinline__ __nv_bfloat16 hi(T a) { return __high2bfloat16(a); }
};

// 128-bit unsigned accumulation of squares of int64 values.
__device__ __forceinline__ void add_u128(uint64_t &lo, uint64_t &hi, uint64_t alo, uint64_t ahi) {
  const uint64_t nlo = lo + alo;
  hi += ahi + (uint64_t)(nlo < lo);
  lo = nlo;
}
__device__ __forceinline__ void add_square(uint64_t &lo, uint64_t &hi, int64_t y) {
  const uint64_t a = (uint64_t)(y < 0 ? -y : y);
  add_u128(lo, hi, a * a, __umul64hi(a, a));
}

}  // namespace mlmc
