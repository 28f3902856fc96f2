// Work items: parameter checks, per-level fixed-point formats and constants
// (Algorithm 1, Sec. 4.1), the proof that selects the fast fixed-point
// datapath, kernel families and the launch-shape table, and the (cached)
// build of one ItemDesc with its chunking into CTAs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "item.h"
#include "kernels.h"
#include "reduce.cuh"
#include "mlmc.h"
#include "tables.h"
#include "host_api.h"

using namespace mlmc;

namespace mlmc_host {

// Work items already built, by everything their constants depend on (params,
// the level's format, level, variant, stream); the sample range is set per call.
struct CachedItem {
  BuiltItem b;
  double disc;
  int unit, exact_int;
};
std::unordered_map<std::string, CachedItem> g_item_cache;
void item_cache_clear() {
  g_item_cache.clear();
  plan_cache_clear();
}

double g_cost[4] = {8.0, 1.0, 0.5, 1.5};
const double g_cost_default[4] = {8.0, 1.0, 0.5, 1.5};

// Launch shape per (kernel family, scheme, payoff class, level class): CTA
// threads and fine path-steps per thread.  Defaults 128 / 256 until
// mlmc_autotune installs measured choices.
constexpr int TUNE_THREADS = 128, TUNE_SPT = 256;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune;
uint64_t g_tune_gen = 0;

int level_class(int level) { return level <= 1 ? level : (level <= 4 ? 2 : (level <= 7 ? 3 : 4)); }

void tuning_for(int family, int scheme, int pc, int level, int *threads, int *spt) {
  auto f = g_tune.find(std::make_tuple(family, scheme, pc, level_class(level)));
  *threads = f == g_tune.end() ? TUNE_THREADS : f->second.first;
  *spt = f == g_tune.end() ? TUNE_SPT : f->second.second;
}

// ---------------------------------------------------------------------------
// parameters, formats and constants
// ---------------------------------------------------------------------------

bool params_ok(const mlmc_params *p) {
  if (!p) return false;
  if (!(std::isfinite(p->S0) && std::isfinite(p->K) && std::isfinite(p->r) && std::isfinite(p->sigma) &&
        std::isfinite(p->T)))
    return false;
  if (!(p->S0 > 0.0) || p->K < 0.0 || p->sigma < 0.0 || !(p->T > 0.0)) return false;
  if (p->payoff < 0 || p->payoff > 3 || p->scheme < 0 || p->scheme > 1) return false;
  if (p->icdf_method < 1 || p->icdf_method > 3) return false;
  if (p->icdf_bits < 2 || p->icdf_bits > 14) return false;
  if (p->icdf_method == 2 && !m2_shape_ok(p->icdf_bits, m2_fields_of(p))) return false;   // n | d, >= 2 bits each
  if (p->icdf_method != 2 && p->icdf_fields != 0) return false;
  if (p->formats && p->n_formats < 0) return false;
  if (p->rng_pack != 0 && p->rng_pack != 1) return false;
  return true;
}

int m2_fields_of(const mlmc_params *p) { return p->icdf_fields ? p->icdf_fields : 2; }

// Lanes per pack of an approximate-only estimator (packed draws need 3 fields of d bits).
bool approx_only_variant(int v) {
  return v == MLMC_FIXED_APPROX || v == MLMC_FP16_APPROX || v == MLMC_BF16_APPROX || v == MLMC_FP16S_APPROX ||
         v == MLMC_BF16S_APPROX;
}

int pack_lanes(const mlmc_params *p, int variant) {
  const bool approx_only = approx_only_variant(variant);
  if (!approx_only || !p->rng_pack) return 1;
  return 32 / p->icdf_bits == 3 ? 3 : 0;  // 0: packing requested but unsupported for this d
}

int bitlen(double x, int f) {
  if (x <= 0.0) return 1 - f;
  return std::max((int)std::floor(std::log2(x)) + 1, 1 - f);
}
// e such that x rounded to f fractional bits stays below 2^e: x + 2^-(f+1) < 2^e
int bitlen_rounded(double x, int f) { return bitlen(x + std::ldexp(1.0, -(f + 1)), f); }

void default_format(const mlmc_params *p, int level, mlmc_format *out) {
  const double r = p->r, sig = p->sigma, T = p->T, S0 = p->S0, K = p->K;
  const double h = T / (double)(1LL << level);
  int f[7] = {12, 16 + level, 14 + level, 12 + level, 12 + level, 12 + level, 14 + level};
  for (int i = 0; i < 7; ++i) f[i] = std::min(24, std::max(10, f[i]));
  // S keeps at most 21 fractional bits (the 32-bit datapath holds e_S + f_S <= 30
  // for the test case), mul2 no more than S
  f[F_S] = std::min(f[F_S], 21);
  f[F_MUL2] = std::min(f[F_MUL2], f[F_S]);
  const double mul1_bound = std::max(16.0 * sig * std::sqrt(h), 128.0 * sig * sig * h);
  int e[7];
  e[F_Z] = 3;
  e[F_CON1] = bitlen_rounded(std::max(std::fabs(r) * 2.0 * h, 0.5 * sig * sig * h), f[F_CON1]);
  e[F_CON2] = bitlen_rounded(sig * std::sqrt(h), f[F_CON2]);
  e[F_MUL1] = bitlen(mul1_bound, f[F_MUL1]);
  e[F_SUM1] = bitlen(std::fabs(r) * 2.0 * h + mul1_bound, f[F_SUM1]);
  const double smax = std::max(S0 * std::exp(std::fabs(r) * T + 6.0 * sig * std::sqrt(T)), K);
  e[F_S] = bitlen_rounded(smax, f[F_S]);
  if (e[F_S] + f[F_S] > 30) {
    // a wide S (high volatility, long maturity) gives up fractional bits down to
    // 10 so that S keeps to 30 bits and the 32-bit datapath
    f[F_S] = std::max(10, 30 - e[F_S]);
    f[F_MUL2] = std::min(f[F_MUL2], f[F_S]);
    e[F_S] = bitlen_rounded(smax, f[F_S]);
  }
  e[F_MUL2] = e[F_S] + e[F_SUM1];
  for (int i = 0; i < 7; ++i) { out->e[i] = (int8_t)e[i]; out->f[i] = (int8_t)f[i]; }
}

Requant make_rq(int from, int to) {
  Requant q;
  if (to >= from) { q.ls = to - from; q.rs = 0; q.radd = 0; }
  else { q.ls = 0; q.rs = from - to; q.radd = (int64_t)1 << (q.rs - 1); }
  return q;
}

// rd of a real constant to f fractional bits, within e integer bits.
mlmc_status const_fixed(double x, int e, int f, int64_t *out) {
  const double s = std::ldexp(x, f);
  if (!(std::fabs(s) < 4503599627370496.0)) return MLMC_EOVERFLOW;
  const double n = std::floor(s + 0.5);
  if (std::fabs(n) > std::ldexp(1.0, e + f) - 1.0) return MLMC_EOVERFLOW;
  *out = (int64_t)n;
  return MLMC_OK;
}

// Ranges the int32 / int64 datapath of the level kernel can hold exactly.
bool format_ok_gpu(const mlmc_format &F, bool milstein, int d) {
  int e[7], f[7];
  for (int i = 0; i < 7; ++i) { e[i] = F.e[i]; f[i] = F.f[i]; }
  for (int i = 0; i < 7; ++i) {
    if (f[i] < 0 || f[i] > 40) return false;
    const int w = e[i] + f[i];
    if (w < 1) return false;
    if (i < F_MUL2 && w > 31) return false;
    if (w > 62) return false;
  }
  if (f[F_Z] > 28) return false;  // Method-3 evaluation shifts by M3_FRAC - f_Z >= 2; 2 f_Z < 63
  (void)d;
  const int F1 = std::max(f[F_CON1], f[F_MUL1]);
  const int F2 = std::max(f[F_S], f[F_MUL2]);
  const int zc = e[F_Z] + 1 + f[F_Z];                       // coarse z: one more integer bit
  if ((e[F_CON2] + f[F_CON2]) + zc > 62) return false;      // con2 * z
  if (e[F_CON2] + e[F_Z] + 1 + f[F_MUL1] > 62) return false; // left re-quantisation of that product
  if (e[F_CON1] + 1 + F1 > 60 || e[F_MUL1] + F1 > 60) return false;  // aligned sum1 terms (3 of them)
  if (std::max(e[F_CON1] + 1, e[F_MUL1]) + 2 + f[F_SUM1] > 62) return false;
  if (milstein && (e[F_CON1] + f[F_CON1]) + 2 * zc > 62) return false;  // con3 * (z^2 - m)
  if ((e[F_S] + f[F_S]) + (e[F_SUM1] + f[F_SUM1]) > 62) return false;   // S * sum1
  if (e[F_S] + e[F_SUM1] + f[F_MUL2] > 62) return false;
  if (e[F_S] + F2 > 61 || e[F_MUL2] + F2 > 61) return false;           // aligned S + mul2
  return true;
}

int family_of(int variant) {
  // 0 exact f32, 1 exact f64, 2 approx fixed, 3 approx f16, 4 approx bf16, 5 corr fixed, 6 corr f16, 7 corr bf16,
  // 18 / 19 approx f16 / bf16 with FP32 S, 20 / 21 corr f16 / bf16 with FP32 S
  switch (variant) {
    case MLMC_FP32_EXACT: return 0;
    case MLMC_FP64_EXACT: return 1;
    case MLMC_FIXED_APPROX: return 2;
    case MLMC_FP16_APPROX: return 3;
    case MLMC_BF16_APPROX: return 4;
    case MLMC_NESTED_CORR_FIXED: return 5;
    case MLMC_NESTED_CORR_FP16: return 6;
    case MLMC_NESTED_CORR_BF16: return 7;
    case MLMC_FP16S_APPROX: return 18;
    case MLMC_BF16S_APPROX: return 19;
    case MLMC_NESTED_CORR_FP16S: return 20;
    default: return 21;
  }
}
// The chunk kind of an item in the merged nested kernel (families 17 / 24): the
// 32-bit fixed-point families with Euler-Maruyama and a terminal payoff,
// 15 approximate packed (0), 8 approximate one sample per thread (1),
// 10 correction (2); -1 for every other item (and for enumerated ones).
int merged_kind(const BuiltItem &b) {
  // enumerated items (exact low levels) keep their own launch: the merged
  // kernel's group code reads Philox words only
  if (b.scheme != MLMC_EULER || b.pc != PC_TERMINAL || b.it.dump || b.it.enumerate) return -1;
  return b.family == 15 ? 0 : (b.family == 8 ? 1 : (b.family == 10 ? 2 : -1));
}

int cost_kind_of(int variant) {
  if (variant == MLMC_FP64_EXACT) return 0;
  if (variant == MLMC_FP32_EXACT) return 1;
  if (approx_only_variant(variant)) return 2;
  return 3;
}

cudaError_t launch_by_family(int fam, int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             const LaunchArgs &a, int *occ) {
  switch (fam) {
    case 12: return launch_approx_fixed_p3(scheme, pc, grid, block, smem, st, a, occ);
    case 13: return launch_approx_f16_p3(scheme, pc, grid, block, smem, st, a, occ);
    case 14: return launch_approx_bf16_p3(scheme, pc, grid, block, smem, st, a, occ);
    case 15: return launch_approx_fx32_p3(scheme, pc, grid, block, smem, st, a, occ);
    case 16: return launch_approx_fx64_p3(scheme, pc, grid, block, smem, st, a, occ);
    case 17: return launch_nested_fx32(scheme, pc, grid, block, smem, st, a, occ, false);
    case 24: return launch_nested_fx32(scheme, pc, grid, block, smem, st, a, occ, true);
    case 18: return launch_approx_f16s(scheme, pc, grid, block, smem, st, a, occ);
    case 19: return launch_approx_bf16s(scheme, pc, grid, block, smem, st, a, occ);
    case 20: return launch_corr_f16s(scheme, pc, grid, block, smem, st, a, occ);
    case 21: return launch_corr_bf16s(scheme, pc, grid, block, smem, st, a, occ);
    case 22: return launch_approx_f16s_p3(scheme, pc, grid, block, smem, st, a, occ);
    case 23: return launch_approx_bf16s_p3(scheme, pc, grid, block, smem, st, a, occ);
    case 8: return launch_approx_fx32(scheme, pc, grid, block, smem, st, a, occ);
    case 9: return launch_approx_fx64(scheme, pc, grid, block, smem, st, a, occ);
    case 10: return launch_corr_fx32(scheme, pc, grid, block, smem, st, a, occ);
    case 11: return launch_corr_fx64(scheme, pc, grid, block, smem, st, a, occ);
    case 0: return launch_exact_f32(scheme, pc, grid, block, smem, st, a, occ);
    case 1: return launch_exact_f64(scheme, pc, grid, block, smem, st, a, occ);
    case 2: return launch_approx_fixed(scheme, pc, grid, block, smem, st, a, occ);
    case 3: return launch_approx_f16(scheme, pc, grid, block, smem, st, a, occ);
    case 4: return launch_approx_bf16(scheme, pc, grid, block, smem, st, a, occ);
    case 5: return launch_corr_fixed(scheme, pc, grid, block, smem, st, a, occ);
    case 6: return launch_corr_f16(scheme, pc, grid, block, smem, st, a, occ);
    default: return launch_corr_bf16(scheme, pc, grid, block, smem, st, a, occ);
  }
}

int64_t radd_of(int k) { return k > 0 ? (int64_t)1 << (k - 1) : 0; }

// floor(v / 2^k) for a 128-bit value (k >= 0)
__int128 floor_shift(__int128 v, int k) { return v >> k; }

// Decide whether the fast fixed-point datapath computes exactly the values of
// the general one for this format: every rounding is a right shift, and the
// magnitudes of mul1, mul3, sum1 (from the table bound) and of mul2 (given
// |S| <= lim_S) can never reach their saturation limits, so that only S needs
// a run-time range check.  Fills ff and tells whether S needs 64 bits.
//
// Terms are aligned on the finer of the two grids of each sum (con1 and mul1
// on F1 = max(f_con1, f_mul1); S and mul2 on max(f_S, f_mul2)), as Algorithm 1's
// exact alignment does.  When mul2 is finer than S (k = f_mul2 - f_S > 0),
// S + mul2 is rounded back to S's format by a second shift; with floor shifts
// and an unsaturated mul2 the two roundings are one:
//   floor((floor((P + r2) / 2^rs2) + 2^(k-1)) / 2^k)
//     = floor((P + r2 + 2^(k-1) 2^rs2) / 2^(rs2 + k)),    P = S sum1,
// so the step adds that single shift of P to S (rs2 + k = f_sum1).
bool fast_fixed(const int e[7], const int f[7], int64_t con1, int64_t con1c, int64_t con2, int64_t con3,
                int64_t zmax, bool milstein, int64_t nsteps, FastFixed &ff, bool &s64) {
  typedef __int128 I;
  const int fZ = f[F_Z];
  const int F1 = std::max(f[F_CON1], f[F_MUL1]);
  if (f[F_SUM1] > F1) return false;   // a finer sum1 is a left shift, not a rounding
  const int rs1 = f[F_CON2] + fZ - f[F_MUL1];
  const int rs3 = f[F_CON1] + 2 * fZ - f[F_MUL1];
  const int rs_sum1 = F1 - f[F_SUM1];
  const int rs2 = f[F_S] + f[F_SUM1] - f[F_MUL2];
  if (rs1 < 0 || rs3 < 0 || rs2 < 0 || rs1 > 62 || rs3 > 62 || rs2 > 62 || rs_sum1 > 30) return false;
  const int shC1 = F1 - f[F_CON1];                    // con1 onto the sum1 accumulation grid
  const int shF1 = F1 - f[F_MUL1];                    // mul1, mul3 onto it
  const int shS = std::max(f[F_S] - f[F_MUL2], 0);    // mul2 onto S's grid (S the finer)
  const int k2 = std::max(f[F_MUL2] - f[F_S], 0);     // S + mul2 back to S's grid (mul2 the finer)
  if (shC1 > 30 || shF1 > 30 || shS > 30 || rs2 + k2 > 62) return false;
  auto lim = [&](int v) { return ((I)1 << (e[v] + f[v])) - 1; };
  // coarse increments are sums of two table values; level 0 (one step) has no
  // coarse path, so its increments are single table values
  const I zc = nsteps > 1 ? 2 * (I)zmax : (I)zmax;
  const I r1 = radd_of(rs1), r3 = radd_of(rs3), rsum = radd_of(rs_sum1), r2 = radd_of(rs2);
  if ((I)con2 * zc + r1 >= ((I)1 << 62)) return false;
  const I m1a = floor_shift((I)con2 * zc + r1, rs1), m1b = floor_shift(-(I)con2 * zc + r1, rs1);
  const I mul1_abs = std::max(m1a, -m1b);
  if (mul1_abs > lim(F_MUL1)) return false;
  I mul3_abs = 0;
  if (milstein) {
    const I one = (I)1 << (2 * fZ);
    const I zz_max = zc * zc - one, zz_min = -2 * one;
    // Z~^2 - m in 32 bits (the kernel forms con3 (Z~^2 - m) as one 32x32 product)
    if (zc * zc >= ((I)1 << 31) - 1 || 2 * one >= ((I)1 << 31)) return false;
    if ((I)con3 * zz_max + r3 >= ((I)1 << 62) || zc * zc >= ((I)1 << 62)) return false;
    const I a = floor_shift((I)con3 * zz_max + r3, rs3), b = floor_shift((I)con3 * zz_min + r3, rs3);
    mul3_abs = std::max(a < 0 ? -a : a, b < 0 ? -b : b);
    if (mul3_abs > lim(F_MUL1)) return false;
  }
  const I c1 = (I)con1 * ((I)1 << shC1), c1c = (I)con1c * ((I)1 << shC1);
  const I c1max = std::max(c1 < 0 ? -c1 : c1, c1c < 0 ? -c1c : c1c);
  const I acc_abs = c1max + rsum + (mul1_abs + mul3_abs) * ((I)1 << shF1);
  if (acc_abs >= ((I)1 << 31) - 1) return false;
  const I sum1_abs = floor_shift(acc_abs, rs_sum1) + 1;
  if (sum1_abs > lim(F_SUM1)) return false;
  const I limS = lim(F_S);
  // the rounding constant of the step's single shift (r2 alone when k2 = 0)
  const I radd2 = r2 + (k2 > 0 ? ((I)1 << (k2 - 1)) * ((I)1 << rs2) : 0);
  if (limS * sum1_abs + radd2 >= ((I)1 << 62)) return false;
  const I mul2_abs = floor_shift(limS * sum1_abs + r2, rs2) + 1;   // the format's mul2
  if (mul2_abs > lim(F_MUL2)) return false;
  // what the step adds to S, in S's units
  const I add_abs = k2 > 0 ? floor_shift(limS * sum1_abs + radd2, rs2 + k2) + 1 : mul2_abs * ((I)1 << shS);
  if (k2 == 0 && mul2_abs >= ((I)1 << 31)) return false;
  if (add_abs >= ((I)1 << 31)) return false;
  const I snew = limS + add_abs;
  if (snew >= ((I)1 << 62)) return false;
  s64 = !(snew < ((I)1 << 31) - 1);
  ff.con2 = (int32_t)con2;
  ff.con3 = (int32_t)con3;
  ff.con1r = (int32_t)(c1 + rsum);
  ff.con1cr = (int32_t)(c1c + rsum);
  ff.mulF1 = 1 << shF1;
  ff.rs1 = rs1; ff.rs3 = rs3; ff.rs_sum1 = rs_sum1; ff.rs2 = rs2 + k2;
  ff.mulS = 1 << shS;
  ff.radd1 = (int64_t)r1; ff.radd3 = (int64_t)r3; ff.radd2 = (int64_t)radd2;
  // the pre-scaled product: sum1 2^(32 - rs2) and radd2 2^(32 - rs2) in range,
  // |S| < 2^31 (32-bit S) so the 64-bit product cannot overflow
  const int rs2t = rs2 + k2;
  ff.pre_ok = rs2t >= 1 && rs2t <= 31 && sum1_abs < ((I)1 << (rs2t - 1)) && radd2 < ((I)1 << 31);
  ff.mfine = (int64_t)1 << (2 * fZ);
  ff.mcoarse = (int64_t)2 << (2 * fZ);
  ff.limS = (int64_t)limS;
  // Lazy saturation of the 32-bit datapath (approximate-only kernels): S runs
  // unclamped, its running maximum is compared with lim_S once per pack, and a
  // pack that went above is simulated again with the clamps.  The values are
  // those of the clamped datapath as long as no path can pass below -lim_S
  // while it stays at or below +lim_S:
  //  * sum1 >= -1 (sum1_min below): from S_k >= 0 a step ends at or above
  //    -mulS (S + S sum1 >= 0, minus one unit of mul2);
  //  * from S_k < 0 the magnitude grows at most to |S_k| (1 + a) + mulS,
  //    a = max |sum1|, so B_{k+1} = B_k (1 + a) + mulS bounds it from B_0 = 0
  //    (S_0 > 0) and B_n <= lim_S after the path's n steps suffices;
  //  * the first value above +lim_S cannot wrap (snew < 2^31 above).
  // The lazy run tracks max S only after the odd fine steps (and on the coarse
  // path), against limT: a fine step takes |S| to at most |S| (1 + A) + mulS,
  // A = max |sum1| 2^-f_sum1 (mulS = 1 when mul2 is finer than S), so S <= limT
  // before a step keeps it within lim_S after it; with S_0 <= limT (build_item
  // checks) every even-index fine S is tracked and every odd-index one follows.
  ff.limT = (int64_t)(((limS - (I)ff.mulS) << f[F_SUM1]) / (((I)1 << f[F_SUM1]) + sum1_abs));
  ff.lazy = 0;
  if (!s64) {
    const I c1min = std::min(c1, c1c);
    const I sum1_min = floor_shift(c1min + rsum - (mul1_abs + mul3_abs) * ((I)1 << shF1), rs_sum1);
    if (sum1_min >= -((I)1 << f[F_SUM1])) {
      const long double a = std::ldexp((long double)sum1_abs, -f[F_SUM1]);
      const long double n = (long double)nsteps, mS = (long double)ff.mulS;
      const long double Bn = a > 0.0L ? mS * (std::pow(1.0L + a, n) - 1.0L) / a : mS * n;
      // a factor-2 margin on the long double evaluation
      if (std::isfinite((double)Bn) && 2.0L * Bn <= (long double)limS) ff.lazy = 1;
    }
  }
  return true;
}

// Largest |table value| in Z's fixed-point format, as the kernels evaluate it.
int64_t table_zmax_fixed(const double *Z, int d, int method, int fZ, int fields) {
  int64_t zmax = 0;
  if (method == 2) {
    const M2Table *t;
    if (m2_build(d, fields, &t) != MLMC_OK) return INT64_MAX;
    for (int j = 0; j < (1 << d); ++j)
      zmax = std::max<int64_t>(zmax, std::llabs(std::llround(std::ldexp(m2_value(*t, d, j, REP_FIXED, fZ), fZ))));
    return zmax;
  }
  if (method == 1) {
    for (int k = 0; k < (1 << (d - 1)); ++k)
      zmax = std::max<int64_t>(zmax, std::llabs((int64_t)std::floor(std::ldexp(Z[k], fZ) + 0.5)));
    return zmax;
  }
  M3Coef c;
  m3_fit(Z, d, c);
  const int sh = M3_FRAC - fZ;
  for (int k = 0; k < (1 << (d - 1)); ++k) {
    const int cls = k < 2 ? 0 : 31 - __builtin_clz((unsigned)k);
    const int64_t t = c.A[cls] + c.B[cls] * (int64_t)k;
    zmax = std::max<int64_t>(zmax, std::llabs((t + ((int64_t)1 << (sh - 1))) >> sh));
  }
  return zmax;
}



// Level-0 approximate items of the 32-bit fast datapath (families 8 and 15)
// with a terminal payoff take their sample values from the per-index table
// (tab_y0), unless they write per-sample records.  Only lazy items: S_0 <=
// limT there, so no index's one fine step leaves lim_S and no sample counts a
// saturation (the items that may saturate keep the clamped step code).
int tab_y0_of(const BuiltItem &b, const void *dump) {
  return (b.family == 8 || b.family == 15) && b.it.level == 0 && b.pc == PC_TERMINAL && b.it.ff.lazy && !dump ? 1
                                                                                                              : 0;
}

// Split an item's sample groups into chunks of `threads` x groups_per_thread.
mlmc_status chunk_built(BuiltItem &b, int threads, int spt, int num_sms, bool floor) {
  ItemDesc &it = b.it;
  uint32_t gpt = 1;
  const uint64_t spg = steps_per_group(it.level);
  const uint64_t nch = chunk_count(it.g1 - it.g0, spg, b.kp, threads, spt, num_sms, &gpt, floor);
  if (nch > 0x7fffffffULL) return MLMC_EINVAL;
  it.groups_per_thread = gpt;
  it.n_chunks = (uint32_t)nch;
  b.chunk_cost = (double)gpt * (double)threads * (double)spg * b.kp * b.cost_step;
  return MLMC_OK;
}

// Packed draws of an item with fewer packs than one wave of resident threads
// run one sample per thread: latency rather than throughput bounds such items.
bool lane_split(uint64_t N, int num_sms) {
  const uint64_t wave = 6ULL * 128ULL * (uint64_t)std::max(1, num_sms);
  return N > 0 && (N + 2) / 3 < wave;
}

// N is bounded before the subtraction, so that the test cannot wrap.
bool sample_range_ok(int level, uint64_t first, uint64_t N) {
  const uint64_t words = 1ULL << (60 - level);
  return N <= (1ULL << 58) && N <= words && first <= words - N;
}

mlmc_status build_item(const mlmc_work &w, int out_index, void *dump, BuiltItem &b, double &disc, int &unit,
                       int &exact_int, TableSource &src) {
  const mlmc_params *p = w.params;
  if (!params_ok(p)) return MLMC_EINVAL;
  if (w.level < 0 || w.level > 20 || w.variant < 0 || w.variant > 11) return MLMC_EINVAL;
  if (w.stream < -1 || w.stream > 255) return MLMC_EINVAL;
  const int lev = w.level;
  // word index s 2^l + i and the group index must stay below 2^62
  if (!sample_range_ok(lev, w.first_sample, w.N)) return MLMC_EINVAL;
  ItemDesc &it = b.it;
  std::memset(&it, 0, sizeof it);
  const int v = w.variant;
  const bool approx = !(v == MLMC_FP32_EXACT || v == MLMC_FP64_EXACT);
  const int stream = w.stream >= 0 ? w.stream : (approx_only_variant(v) ? 1 : 0);
  it.first = w.first_sample;
  it.N = w.N;
  it.level = lev;
  it.nlog = lev;
  it.payoff = p->payoff;
  it.scheme = p->scheme;
  it.method = p->icdf_method;
  it.d = p->icdf_bits;
  it.ctr2 = (uint32_t)lev | ((uint32_t)stream << 8);
  it.ctr3 = p->request_id;
  it.out_index = (uint32_t)out_index;
  it.dump = dump;
  if (w.flags & ~MLMC_WORK_ENUMERATE) return MLMC_EINVAL;
  const bool enumerate = (w.flags & MLMC_WORK_ENUMERATE) != 0;
  int KP = pack_lanes(p, v);
  if (enumerate) {
    // every combination of table cells once: approximate-only, levels 0-1, samples [0, 2^(d 2^l))
    const bool approx_only = approx_only_variant(v);
    const int bits = p->icdf_bits << lev;
    if (!approx_only || lev > 1 || bits > 24 || w.first_sample != 0 || w.N != (1ULL << bits)) return MLMC_EINVAL;
    KP = 1;
    it.enumerate = 1;
  }
  if (KP == 0) return MLMC_EINVAL;
  if (KP == 3 && lev >= 2 && lane_split(w.N, src.num_sms())) {
    // few samples: one sample per thread (three times the threads), the same
    // packed draws (sample s reads lane s mod 3 of pack s / 3)
    KP = 1;
    it.lanes = 3;
  }
  // sample groups (chunking into CTAs: chunk_built)
  const uint64_t spc = samples_per_group(lev, KP);
  it.g0 = w.first_sample / spc;
  it.g1 = w.N == 0 ? it.g0 : (w.first_sample + w.N + spc - 1) / spc;
  // groups whose samples all lie in [first, first + N)
  it.gf0 = (w.first_sample + spc - 1) / spc;
  it.gf1 = (w.first_sample + w.N) / spc;
  if (it.gf1 < it.gf0) it.gf1 = it.gf0;
  b.kp = KP;
  b.cost_step = g_cost[cost_kind_of(v)];
  // exact-path constants (the same FP64 expressions as the fixed-point ones)
  const double h = std::ldexp(p->T, -lev);
  const double rh = p->r * h, rh2 = p->r * (2.0 * h), sqh = std::sqrt(h);
  const double c2 = p->sigma * sqh, c3 = 0.5 * p->sigma * p->sigma * h;
  it.c1d = rh; it.c2d = c2; it.c1cd = rh2; it.c3d = c3; it.S0d = p->S0; it.Kd = p->K;
  it.c1f = (float)rh; it.c2f = (float)c2; it.c1cf = (float)rh2; it.c3f = (float)c3;
  it.S0f = (float)p->S0; it.Kf = (float)p->K;
  disc = std::exp(-p->r * p->T);
  unit = 0;
  exact_int = 0;
  b.smem = 0;
  bool fast = false, fast64 = false;
  if (approx) {
    const bool fixed = (v == MLMC_FIXED_APPROX || v == MLMC_NESTED_CORR_FIXED);
    const bool bf = (v == MLMC_BF16_APPROX || v == MLMC_NESTED_CORR_BF16 || v == MLMC_BF16S_APPROX ||
                     v == MLMC_NESTED_CORR_BF16S);
    const int rep = fixed ? REP_FIXED : (bf ? REP_BF16 : REP_FP16);
    int fZ = 0;
    if (fixed) {
      mlmc_format F;
      if (p->formats && lev < p->n_formats) F = p->formats[lev];
      else if (p->formats) return MLMC_EINVAL;
      else default_format(p, lev, &F);
      if (!format_ok_gpu(F, p->scheme == MLMC_MILSTEIN, p->icdf_bits)) return MLMC_EINVAL;
      int e[7], f[7];
      for (int i = 0; i < 7; ++i) { e[i] = F.e[i]; f[i] = F.f[i]; }
      fZ = f[F_Z];
      FixedConsts &fx = it.fx;
      int64_t con1, con1c, con2, con3, S0q, Kq;
      mlmc_status s = MLMC_OK;
      if ((s = const_fixed(rh, e[F_CON1], f[F_CON1], &con1)) != MLMC_OK) return s;
      if ((s = const_fixed(rh2, e[F_CON1] + 1, f[F_CON1], &con1c)) != MLMC_OK) return s;
      if ((s = const_fixed(c2, e[F_CON2], f[F_CON2], &con2)) != MLMC_OK) return s;
      if ((s = const_fixed(c3, e[F_CON1], f[F_CON1], &con3)) != MLMC_OK) return s;
      if ((s = const_fixed(p->S0, e[F_S], f[F_S], &S0q)) != MLMC_OK) return s;
      if ((s = const_fixed(p->K, e[F_S], f[F_S], &Kq)) != MLMC_OK) return s;
      const int F1 = std::max(f[F_CON1], f[F_MUL1]);
      const int F2 = std::max(f[F_S], f[F_MUL2]);
      fx.con1A = con1 * ((int64_t)1 << (F1 - f[F_CON1]));
      fx.con1cA = con1c * ((int64_t)1 << (F1 - f[F_CON1]));
      fx.con2 = (int32_t)con2;
      fx.con3 = (int32_t)con3;
      fx.S0 = S0q;
      fx.K = Kq;
      for (int i = 0; i < 7; ++i) fx.lim[i] = ((int64_t)1 << (e[i] + f[i])) - 1;
      fx.q_mul1 = make_rq(f[F_CON2] + f[F_Z], f[F_MUL1]);
      fx.q_mul3 = make_rq(f[F_CON1] + 2 * f[F_Z], f[F_MUL1]);
      fx.sh_mul1_F1 = F1 - f[F_MUL1];
      fx.q_sum1 = make_rq(F1, f[F_SUM1]);
      fx.q_mul2 = make_rq(f[F_S] + f[F_SUM1], f[F_MUL2]);
      fx.sh_S_F2 = F2 - f[F_S];
      fx.sh_mul2_F2 = F2 - f[F_MUL2];
      fx.q_S = make_rq(F2, f[F_S]);
      fx.fZ2 = 2 * f[F_Z];
      fx.fS = f[F_S];
      // the table must fit Z's format
      int64_t zmax = 0;
      if ((s = src.zmax_fixed(p->icdf_method, p->icdf_bits, fZ, m2_fields_of(p), &zmax)) != MLMC_OK) return s;
      if ((double)zmax > std::ldexp(1.0, e[F_Z] + fZ) - 1.0) return MLMC_EOVERFLOW;
      unit = f[F_S] + (p->payoff == MLMC_ASIAN ? lev + 1 : 0);
      bool s64 = false;
      fast = fast_fixed(e, f, con1, con1c, con2, con3, zmax, p->scheme == MLMC_MILSTEIN, (int64_t)1 << lev, it.ff,
                        s64);
      fast64 = s64;
      if (fast && it.ff.lazy && S0q > it.ff.limT) it.ff.lazy = 0;   // the thinned check needs S_0 <= limT
      // the 32-bit datapath keeps (Z~, fine sum1) pairs in shared memory (2^d x 8
      // bytes: d <= 12) and rounds products by one funnel shift (shifts below 32)
      if (fast && !fast64 &&
          (p->icdf_bits > 12 || it.ff.rs1 > 31 || it.ff.rs2 > 31 ||
           (p->scheme == MLMC_MILSTEIN && it.ff.rs3 > 31)))
        fast64 = true;
      if (fast && !fast64) {
        // the 32-bit datapath sums a group's squared terminal payoff differences in
        // 64 bits: |Y| <= max(lim_S, 2^f_S), so spc samples need spc ymax^2 < 2^64
        const double ymax = std::max(std::ldexp(1.0, e[F_S] + f[F_S]), std::ldexp(1.0, f[F_S]));
        if (!((double)spc * ymax * ymax < 0x1p64)) fast64 = true;
      }
    } else {
      uint16_t (*cv)(double) = bf ? bf16_bits : half_bits;
      it.h_c1 = cv(rh);
      it.h_c1c = cv(rh2);
      it.h_c2 = cv(c2);
      it.h_c3 = cv(c3);
      it.h_S0 = cv(p->S0);
      unit = 24;
    }
    const void *tab = nullptr;
    mlmc_status s = src.device_table(p->icdf_method, p->icdf_bits, rep, fZ, m2_fields_of(p), &tab);
    if (s != MLMC_OK) return s;
    it.ztab = tab;
    b.smem = p->icdf_method != 3 ? (size_t)(1 << p->icdf_bits) * (fixed ? 4 : 2) : sizeof(M3Coef);
    exact_int = approx_only_variant(v) ? 1 : 0;
    if (p->icdf_method == 2 && !exact_int) {
      // Method 2 coupling: the correction's exact path reads the interval ranks
      const uint16_t *perm = nullptr;
      if ((s = src.m2_perm(p->icdf_bits, m2_fields_of(p), &perm)) != MLMC_OK) return s;
      it.perm = perm;
      b.smem += sizeof(uint16_t) << p->icdf_bits;
    }
  }
  it.unit = unit;
  it.unit_scale = std::ldexp(1.0f, -unit);
  b.family = family_of(v);
  if (fast) {
    if (b.family == 2) b.family = fast64 ? 9 : 8;
    else if (b.family == 5) b.family = fast64 ? 11 : 10;
  }
  if (KP == 3) {
    // packed families: 12 fixed (general), 13 binary16, 14 bfloat16, 15 fixed 32-bit S, 16 fixed 64-bit S
    switch (b.family) {
      case 2: b.family = 12; break;
      case 3: b.family = 13; break;
      case 4: b.family = 14; break;
      case 8: b.family = 15; break;
      case 9: b.family = 16; break;
      case 18: b.family = 22; break;
      case 19: b.family = 23; break;
      default: return MLMC_EINVAL;
    }
  }
  if (b.family == 8 || b.family == 10 || b.family == 15) {
    // the 32-bit datapath's shared-memory table: (Z~_j, fine sum1_j) pairs for
    // every method (Method 3's lines are evaluated into it), then Method 2's ranks
    b.smem = ((size_t)8 << p->icdf_bits) + (it.perm ? (sizeof(uint16_t) << p->icdf_bits) : 0);
  }
  b.scheme = p->scheme;
  b.pc = p->payoff == MLMC_ASIAN ? PC_ASIAN : (p->payoff == MLMC_LOOKBACK ? PC_LOOKBACK : PC_TERMINAL);
  it.tab_y0 = tab_y0_of(b, dump);
  return MLMC_OK;
}

// build_item through the cache (flags 0): the constants, tables and family
// come from the first build of the same (params, format, level, variant,
// stream); the sample range and its groups are set for this call.
mlmc_status build_item_cached(const mlmc_work &w, int out_index, void *dump, BuiltItem &b, double &disc, int &unit,
                              int &exact_int) {
  const mlmc_params *p = w.params;
  if (w.flags != 0 || !params_ok(p) || w.level < 0 || w.level > 20)
    return build_item(w, out_index, dump, b, disc, unit, exact_int, ctx_tables());
  std::string key;
  key.reserve(96);
  auto put = [&](const void *x, size_t n) { key.append((const char *)x, n); };
  put(&p->S0, sizeof(double) * 5);
  put(&p->payoff, sizeof(int32_t) * 4);
  put(&p->request_id, sizeof(uint32_t));
  put(&p->rng_pack, sizeof(int32_t) * 2);   // rng_pack, icdf_fields
  const int has_fmt = p->formats ? (w.level < p->n_formats ? 1 : 2) : 0;
  put(&has_fmt, sizeof has_fmt);
  if (has_fmt == 1) put(&p->formats[w.level], sizeof(mlmc_format));
  put(&w.level, sizeof(int32_t) * 2);     // level, variant
  put(&w.stream, sizeof(int32_t));
  const int split = lane_split(w.N, g.num_sms) ? 1 : 0;   // the packed-draw layout depends on N
  put(&split, sizeof split);
  auto f = g_item_cache.find(key);
  if (f == g_item_cache.end()) {
    mlmc_status s = build_item(w, out_index, dump, b, disc, unit, exact_int, ctx_tables());
    if (s != MLMC_OK) return s;
    if (g_item_cache.size() > 8192) g_item_cache.clear();
    g_item_cache.emplace(key, CachedItem{b, disc, unit, exact_int});
    return MLMC_OK;
  }
  const int lev = w.level;
  if (!sample_range_ok(lev, w.first_sample, w.N)) return MLMC_EINVAL;
  b = f->second.b;
  disc = f->second.disc;
  unit = f->second.unit;
  exact_int = f->second.exact_int;
  ItemDesc &it = b.it;
  it.first = w.first_sample;
  it.N = w.N;
  it.out_index = (uint32_t)out_index;
  it.dump = dump;
  it.tab_y0 = tab_y0_of(b, dump);
  const uint64_t spc = samples_per_group(lev, b.kp);
  it.g0 = w.first_sample / spc;
  it.g1 = w.N == 0 ? it.g0 : (w.first_sample + w.N + spc - 1) / spc;
  it.gf0 = (w.first_sample + spc - 1) / spc;
  it.gf1 = (w.first_sample + w.N) / spc;
  if (it.gf1 < it.gf0) it.gf1 = it.gf0;
  b.cost_step = g_cost[cost_kind_of(w.variant)];
  return MLMC_OK;
}

void make_round_keys(uint64_t seed, RoundKeys &rk) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k[2 * r] = k0;
    rk.k[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

double cost_of_variant(int variant) { return g_cost[cost_kind_of(variant)]; }

}  // namespace mlmc_host

using namespace mlmc_host;

extern "C" {

mlmc_status mlmc_cost_model(int kind, double cost_per_step) {
  MLMC_API_LOCK();
  if (kind < 0 || kind > 3 || !std::isfinite(cost_per_step)) return MLMC_EINVAL;
  g_cost[kind] = cost_per_step > 0.0 ? cost_per_step : g_cost_default[kind];
  return MLMC_OK;
}

mlmc_status mlmc_default_format(const mlmc_params *p, int level, mlmc_format *out) {
  if (!params_ok(p) || !out || level < 0 || level > 20) return MLMC_EINVAL;
  default_format(p, level, out);
  return MLMC_OK;
}

}  // extern "C"
