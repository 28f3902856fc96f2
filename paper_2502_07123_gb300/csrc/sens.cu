// Error-model statistics of one MLMC level on the GPU (Sec. 4.2-4.3): for
// the discounted level difference DeltaP = P_f - P_c of a European call under
// Euler-Maruyama with exact FP64 Normals (stream 0, the correction
// estimator's uniforms), the sensitivities xbar = d DeltaP / d x of every
// intermediate variable of Algorithm 1 -- con1 (and the coarse constant for
// 2h), con2, Z_j, mul1_k, sum1_k, mul2_k, S_k on both paths, and S0 -- their
// second moments per variable type (V_indep, eq. optimistic) and per instance
// (V_corr, eq. pessimistic), the maxima |x| per type (exponents, Sec. 4.1),
// and the mean and variance of DeltaP.
//
// The reverse sweep of Algorithm 1 has a closed form for this graph: with
// S_{k+1} = S_k (1 + sum1_k), d S_n / d S_{k+1} = S_n / S_{k+1}, so every
// sensitivity is a_f S_n (resp. a_c S^c_m) times a per-step factor
// (1 / S_{k+1}, 1 / (1 + sum1_k), Z_k / (1 + sum1_k), ...), where
// a_f = e^{-rT} 1[S_n > K] and a_c = -e^{-rT} 1[S^c_m > K].  A thread
// therefore needs no tape: pass 1 runs the sample forward and accumulates the
// per-step factor sums (which give the per-type second moments once S_n and
// S^c_m are known); pass 2 regenerates the same uniforms, forms each
// instance's sensitivity and adds its square, summed over the warp, into the
// warp's own shared-memory row (deterministic order).  Per-CTA partials are
// summed in CTA order by sens_finalize_kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "host_api.h"
#include "item.h"
#include "mlmc.h"

using namespace mlmc;

namespace {

constexpr int SENS_THREADS = 128;
constexpr int SENS_WARPS = SENS_THREADS / 32;
constexpr int SENS_MAX_LEVEL = 10;
// per-instance rows kept on the device: S-type (= mul2 except S0), sum1-type (= mul1), Z
constexpr int SENS_ROWS = 3;
enum { T_Z = 0, T_CON1 = 1, T_CON2 = 2, T_MUL1 = 3, T_SUM1 = 4, T_MUL2 = 5, T_S = 6 };

struct SensConsts {
  double con1, con1c, con2, S0, K, disc;
  int level, n, m, ni;
  uint64_t first, N;
  uint32_t ctr2, ctr3;
};

// Per-CTA partial: per-type sums of squared sensitivities, maxima, DeltaP sums,
// and the per-sample scalar instances (con1 fine / coarse, con2, S0).
struct SensPartial {
  double A[7];
  double maxabs[7];
  double sdp, sdp2;
  double c1f, c1c, c2, s0;
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// Exact FP64 Normal of fine step k of sample s (stream 0); `q` / `w` cache the
// last Philox call of this thread.
struct Draws {
  uint64_t q = ~0ULL;
  uint4 w;
  __device__ __forceinline__ double z(const SensConsts &c, const RoundKeys &rk, uint64_t s, int k) {
    const uint64_t wi = (s << c.level) + (uint64_t)k;
    const uint64_t qq = wi >> 2;
    if (qq != q) {
      q = qq;
      w = philox4x32_10(make_uint4((uint32_t)qq, (uint32_t)(qq >> 32), c.ctr2, c.ctr3), rk);
    }
    return exact_normal_f64(word_of(w, (int)(wi & 3)));
  }
};

__global__ void __launch_bounds__(SENS_THREADS) sens_kernel(const SensConsts c, const RoundKeys rk, int iters,
                                                            SensPartial *part, double *inst_part) {
  extern __shared__ double srow[];   // [warp][SENS_ROWS][ni]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ni = c.ni, n = c.n, m = c.m;
  double *row = srow + (size_t)warp * SENS_ROWS * ni;
  for (int i = lane; i < SENS_ROWS * ni; i += 32) row[i] = 0.0;
  __syncwarp();
  double A[7] = {0, 0, 0, 0, 0, 0, 0}, mx[7] = {0, 0, 0, 0, 0, 0, 0};
  double sdp = 0.0, sdp2 = 0.0, c1f = 0.0, c1c = 0.0, c2s = 0.0, s0s = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (int it = 0; it < iters; ++it) {
    const uint64_t rel = (uint64_t)it * stride + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = rel < c.N;
    const uint64_t s = c.first + (valid ? rel : 0);
    // ---- pass 1: forward, factor sums ----
    Draws dr;
    double S = c.S0, Sc = c.S0, zprev = 0.0;
    double inv2S = 0.0, u2 = 0.0, u1 = 0.0, zu = 0.0;
    double inv2Sc = 0.0, v2 = 0.0, v1 = 0.0, zcv = 0.0, uv = 0.0, uprev = 0.0;
    double mz = 0.0, m1 = 0.0, ms1 = 0.0, mm2 = 0.0, mS = c.S0;
    for (int k = 0; k < n; ++k) {
      const double z = dr.z(c, rk, s, k);
      const double mul1 = c.con2 * z;
      const double sum1 = c.con1 + mul1;
      const double mul2 = S * sum1;
      S = S + mul2;
      const double u = 1.0 / (1.0 + sum1);
      inv2S += 1.0 / (S * S);
      u2 += u * u;
      u1 += u;
      zu += z * u;
      mz = fmax(mz, fabs(z)); m1 = fmax(m1, fabs(mul1)); ms1 = fmax(ms1, fabs(sum1));
      mm2 = fmax(mm2, fabs(mul2)); mS = fmax(mS, fabs(S));
      if (m > 0 && (k & 1)) {
        const double zc = zprev + z;
        const double mul1c = c.con2 * zc;
        const double sum1c = c.con1c + mul1c;
        const double mul2c = Sc * sum1c;
        Sc = Sc + mul2c;
        const double v = 1.0 / (1.0 + sum1c);
        inv2Sc += 1.0 / (Sc * Sc);
        v2 += v * v;
        v1 += v;
        zcv += zc * v;
        uv += v * (uprev + u);
        m1 = fmax(m1, fabs(mul1c)); ms1 = fmax(ms1, fabs(sum1c));
        mm2 = fmax(mm2, fabs(mul2c)); mS = fmax(mS, fabs(Sc));
      }
      zprev = z;
      uprev = u;
    }
    const double Pf = c.disc * (S > c.K ? S - c.K : 0.0);
    const double Pc = m > 0 ? c.disc * (Sc > c.K ? Sc - c.K : 0.0) : 0.0;
    const double F = valid && S > c.K ? c.disc * S : 0.0;
    const double G = valid && m > 0 && Sc > c.K ? -c.disc * Sc : 0.0;
    if (valid) {
      const double dp = Pf - Pc;
      sdp += dp;
      sdp2 += dp * dp;
      mx[T_Z] = fmax(mx[T_Z], mz); mx[T_MUL1] = fmax(mx[T_MUL1], m1); mx[T_SUM1] = fmax(mx[T_SUM1], ms1);
      mx[T_MUL2] = fmax(mx[T_MUL2], mm2); mx[T_S] = fmax(mx[T_S], mS);
    }
    const double sS0 = (F + G) / c.S0;
    A[T_S] += F * F * inv2S + G * G * inv2Sc + sS0 * sS0;
    A[T_MUL2] += F * F * inv2S + G * G * inv2Sc;
    A[T_SUM1] += F * F * u2 + G * G * v2;
    A[T_MUL1] += F * F * u2 + G * G * v2;
    const double a1f = F * u1, a1c = G * v1, a2 = F * zu + G * zcv;
    A[T_CON1] += a1f * a1f + a1c * a1c;
    A[T_CON2] += a2 * a2;
    A[T_Z] += c.con2 * c.con2 * (F * F * u2 + 2.0 * F * G * uv + 2.0 * G * G * v2);
    c1f += a1f * a1f; c1c += a1c * a1c; c2s += a2 * a2; s0s += sS0 * sS0;
    // ---- pass 2: per-instance squares (same uniforms), summed over the warp ----
    Draws dr2;
    S = c.S0; Sc = c.S0; zprev = 0.0; uprev = 0.0;
    for (int k = 0; k < n; ++k) {
      const double z = dr2.z(c, rk, s, k);
      const double sum1 = c.con1 + c.con2 * z;
      S = S + S * sum1;
      const double u = 1.0 / (1.0 + sum1);
      const double xs = F / S, xu = F * u;
      const double ws = warp_sum(xs * xs), wu = warp_sum(xu * xu);
      if (lane == 0) { row[k] += ws; row[ni + k] += wu; }
      if (m > 0 && (k & 1)) {
        const double zc = zprev + z;
        const double sum1c = c.con1c + c.con2 * zc;
        Sc = Sc + Sc * sum1c;
        const double v = 1.0 / (1.0 + sum1c);
        const int kc = k >> 1;
        const double ys = G / Sc, yv = G * v;
        const double za = c.con2 * (F * uprev + G * v), zb = c.con2 * (F * u + G * v);
        const double w1 = warp_sum(ys * ys), w2 = warp_sum(yv * yv), w3 = warp_sum(za * za), w4 = warp_sum(zb * zb);
        if (lane == 0) {
          row[n + kc] += w1; row[ni + n + kc] += w2;
          row[2 * ni + k - 1] += w3; row[2 * ni + k] += w4;
        }
      } else if (m == 0) {
        const double zb = c.con2 * F * u;
        const double w4 = warp_sum(zb * zb);
        if (lane == 0) row[2 * ni + k] += w4;
      }
      zprev = z;
      uprev = u;
    }
  }
  // ---- CTA reduction (warp order) ----
  __shared__ SensPartial wp[SENS_WARPS];
  SensPartial p;
  for (int t = 0; t < 7; ++t) { p.A[t] = warp_sum(A[t]); p.maxabs[t] = warp_max(mx[t]); }
  p.sdp = warp_sum(sdp); p.sdp2 = warp_sum(sdp2);
  p.c1f = warp_sum(c1f); p.c1c = warp_sum(c1c); p.c2 = warp_sum(c2s); p.s0 = warp_sum(s0s);
  if (lane == 0) wp[warp] = p;
  __syncthreads();
  if (threadIdx.x == 0) {
    SensPartial t = wp[0];
    for (int w = 1; w < SENS_WARPS; ++w) {
      for (int q = 0; q < 7; ++q) { t.A[q] += wp[w].A[q]; t.maxabs[q] = fmax(t.maxabs[q], wp[w].maxabs[q]); }
      t.sdp += wp[w].sdp; t.sdp2 += wp[w].sdp2;
      t.c1f += wp[w].c1f; t.c1c += wp[w].c1c; t.c2 += wp[w].c2; t.s0 += wp[w].s0;
    }
    t.maxabs[T_CON1] = fmax(fabs(c.con1), m > 0 ? fabs(c.con1c) : 0.0);
    t.maxabs[T_CON2] = fabs(c.con2);
    part[blockIdx.x] = t;
  }
  double *out = inst_part + (size_t)blockIdx.x * SENS_ROWS * ni;
  for (int i = threadIdx.x; i < SENS_ROWS * ni; i += blockDim.x) {
    double x = 0.0;
    for (int w = 0; w < SENS_WARPS; ++w) x += srow[(size_t)w * SENS_ROWS * ni + i];
    out[i] = x;
  }
}

// Sum the CTA partials in CTA order: block 0 the scalars, the others one
// per-instance entry per thread.
__global__ void sens_finalize_kernel(const SensPartial *part, const double *inst_part, int n_ctas, int ni,
                                     SensPartial *res, double *inst) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    SensPartial t = part[0];
    for (int b = 1; b < n_ctas; ++b) {
      for (int q = 0; q < 7; ++q) { t.A[q] += part[b].A[q]; t.maxabs[q] = fmax(t.maxabs[q], part[b].maxabs[q]); }
      t.sdp += part[b].sdp; t.sdp2 += part[b].sdp2;
      t.c1f += part[b].c1f; t.c1c += part[b].c1c; t.c2 += part[b].c2; t.s0 += part[b].s0;
    }
    *res = t;
  }
  const int i = (blockIdx.x - 1) * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 || i >= SENS_ROWS * ni) return;
  double x = 0.0;
  for (int b = 0; b < n_ctas; ++b) x += inst_part[(size_t)b * SENS_ROWS * ni + i];
  inst[i] = x;
}

}  // namespace

extern "C" mlmc_status mlmc_sensitivities(int level, uint64_t N, const mlmc_params *p, uint64_t seed,
                                          uint64_t first_sample, mlmc_sensitivity *out, double *inst_out) {
  MLMC_API_LOCK();
  using namespace mlmc_host;
  if (!out || !p || !params_ok(p) || level < 0 || level > SENS_MAX_LEVEL || N == 0) return MLMC_EINVAL;
  if (p->payoff != MLMC_EURO || p->scheme != MLMC_EULER) return MLMC_EINVAL;
  if (N > (1ULL << 40) || first_sample > (1ULL << (60 - level)) - N) return MLMC_EINVAL;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  SensConsts c;
  std::memset(&c, 0, sizeof c);
  const double h = std::ldexp(p->T, -level);
  c.con1 = p->r * h;
  c.con1c = p->r * (2.0 * h);
  c.con2 = p->sigma * std::sqrt(h);
  c.S0 = p->S0;
  c.K = p->K;
  c.disc = std::exp(-p->r * p->T);
  c.level = level;
  c.n = 1 << level;
  c.m = level > 0 ? c.n / 2 : 0;
  c.ni = c.n + c.m + 1;
  c.first = first_sample;
  c.N = N;
  c.ctr2 = (uint32_t)level;   // stream 0
  c.ctr3 = p->request_id;
  RoundKeys rk;
  make_round_keys(seed, rk);
  const int n_ctas = (int)std::min<uint64_t>((uint64_t)2 * ctx_num_sms(),
                                             (N + SENS_THREADS - 1) / SENS_THREADS);
  const uint64_t per = (uint64_t)n_ctas * SENS_THREADS;
  const int iters = (int)((N + per - 1) / per);
  const size_t smem = sizeof(double) * SENS_WARPS * SENS_ROWS * (size_t)c.ni;
  cudaStream_t st = ctx_stream();
  SensPartial *d_part = nullptr, *d_res = nullptr;
  double *d_ip = nullptr, *d_inst = nullptr;
  const size_t rows = (size_t)SENS_ROWS * c.ni;
  if (cudaMalloc(&d_part, sizeof(SensPartial) * n_ctas) != cudaSuccess ||
      cudaMalloc(&d_res, sizeof(SensPartial)) != cudaSuccess ||
      cudaMalloc(&d_ip, sizeof(double) * rows * n_ctas) != cudaSuccess ||
      cudaMalloc(&d_inst, sizeof(double) * rows) != cudaSuccess) {
    cudaFree(d_part); cudaFree(d_res); cudaFree(d_ip); cudaFree(d_inst);
    return MLMC_ENOMEM;
  }
  mlmc_status rs = MLMC_OK;
  SensPartial h_res;
  std::vector<double> rowsum(rows);
  do {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(sens_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      rs = MLMC_ECUDA;
      break;
    }
    sens_kernel<<<n_ctas, SENS_THREADS, smem, st>>>(c, rk, iters, d_part, d_ip);
    sens_finalize_kernel<<<1 + (unsigned)((rows + 127) / 128), 128, 0, st>>>(d_part, d_ip, n_ctas, c.ni, d_res,
                                                                             d_inst);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h_res, d_res, sizeof h_res, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(rowsum.data(), d_inst, sizeof(double) * rows, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rs = MLMC_ECUDA;
  } while (0);
  cudaFree(d_part); cudaFree(d_res); cudaFree(d_ip); cudaFree(d_inst);
  if (rs != MLMC_OK) return rs;
  // per-instance second moments, type-major 7 x ni
  const int ni = c.ni, n = c.n, m = c.m;
  std::vector<double> E((size_t)7 * ni, 0.0);
  const double inv = 1.0 / (double)N;
  for (int i = 0; i < n + m; ++i) {
    E[(size_t)T_S * ni + i] = rowsum[i] * inv;
    E[(size_t)T_MUL2 * ni + i] = rowsum[i] * inv;
    E[(size_t)T_SUM1 * ni + i] = rowsum[ni + i] * inv;
    E[(size_t)T_MUL1 * ni + i] = rowsum[ni + i] * inv;
  }
  for (int j = 0; j < n; ++j) E[(size_t)T_Z * ni + j] = rowsum[2 * ni + j] * inv;
  E[(size_t)T_S * ni + n + m] = h_res.s0 * inv;
  E[(size_t)T_CON1 * ni + 0] = h_res.c1f * inv;
  E[(size_t)T_CON1 * ni + 1] = h_res.c1c * inv;
  E[(size_t)T_CON2 * ni + 0] = h_res.c2 * inv;
  std::memset(out, 0, sizeof *out);
  for (int t = 0; t < 7; ++t) {
    out->A[t] = h_res.A[t] * inv;
    out->maxabs[t] = h_res.maxabs[t];
    double b = 0.0;
    for (int i = 0; i < ni; ++i) b += std::sqrt(E[(size_t)t * ni + i]);
    out->B[t] = b;
  }
  out->mean = h_res.sdp * inv;
  out->var = std::max(0.0, h_res.sdp2 * inv - out->mean * out->mean);
  out->n = N;
  out->n_instances = ni;
  if (inst_out) std::memcpy(inst_out, E.data(), sizeof(double) * E.size());
  return MLMC_OK;
}
