// Device work-item descriptor and reduction records of the level kernels.
// Built on the host (items.cu) from the public mlmc_work / mlmc_params and
// copied to device memory once per plan.
#pragma once
#include <stdint.h>

namespace mlmc {

// estimator kinds (template parameter EST of the level kernel)
enum Est : int { EST_EXACT = 0, EST_APPROX = 1, EST_CORR = 2 };
// exact-path precision
enum Xp : int { XP_NONE = 0, XP_F32 = 1, XP_F64 = 2 };
// approximate-path arithmetic
// AP_FIXED is the general fixed-point datapath (64-bit, saturating every
// variable); AP_FX32 / AP_FX64 are the fast datapath for formats whose bounds
// the host has proven (32-bit values, S in 32 or 64 bits, only S range-checked).
// AP_F16S / AP_BF16S: binary16 / bfloat16 increments with S in FP32.
enum Ap : int { AP_NONE = 0, AP_FIXED = 1, AP_F16 = 2, AP_BF16 = 3, AP_FX32 = 4, AP_FX64 = 5, AP_F16S = 6, AP_BF16S = 7 };
// payoff classes that need different path functionals
enum PayClass : int { PC_TERMINAL = 0, PC_ASIAN = 1, PC_LOOKBACK = 2 };

// ((x << ls) + radd) >> rs with at most one of ls, rs non-zero: the exact
// re-expression of n 2^-from in 2^-to, rounded to nearest with ties toward +inf.
struct Requant {
  int32_t ls, rs;
  int64_t radd;
};

struct FixedConsts {
  int64_t con1A, con1cA;   // con1, con1_c aligned to the sum1 accumulation grid F1
  int32_t con2, con3;      // con2 (f_con2), con3 (f_con1)
  int64_t S0, K;           // in S's format
  int64_t lim[7];          // saturation limits 2^(e+f) - 1
  Requant q_mul1;          // con2 * z          : f_con2 + f_Z      -> f_mul1
  Requant q_mul3;          // con3 * (z^2 - m)  : f_con1 + 2 f_Z    -> f_mul1
  int32_t sh_mul1_F1;      // mul1 -> F1 (left shift)
  Requant q_sum1;          // F1 -> f_sum1
  Requant q_mul2;          // S * sum1          : f_S + f_sum1      -> f_mul2
  int32_t sh_S_F2, sh_mul2_F2;  // S, mul2 -> F2 (left shifts)
  Requant q_S;             // F2 -> f_S
  int32_t fZ2;             // 2 f_Z (Milstein: the constant m is m 2^(2 f_Z))
  int32_t fS;
};

// Constants of the fast fixed-point step (host-proven: no variable but S can
// leave its format; S is checked every step).  Every rounding adds its half
// unit before an arithmetic right shift; left alignments are multiplications.
struct FastFixed {
  int32_t con2, con3;
  int32_t con1r, con1cr;     // con1, con1_c on the sum1 accumulation grid F1 = max(f_con1, f_mul1),
                             // plus the rounding half unit of sum1
  int32_t mulF1;             // 2^(F1 - f_mul1): mul1, mul3 onto that grid
  int32_t rs1, rs3, rs_sum1; // rs_sum1 = F1 - f_sum1
  int32_t rs2;               // shift of S sum1: f_S + f_sum1 - f_mul2, or f_sum1 when mul2 is finer
                             // than S (the rounding of S + mul2 folded in)
  int32_t mulS;              // 2^(f_S - f_mul2) when S is the finer, else 1
  int64_t radd1, radd3, radd2;
  int64_t mfine, mcoarse;    // 1 and 2 in units 2^-2fZ (Milstein)
  int64_t limS;
  int64_t limT;              // lazy runs: S after an odd fine step (and the coarse S) at most limT
                             // keeps every fine S within lim_S (fast_fixed)
  int32_t lazy;              // 32-bit S may run unclamped, checked once per pack (fast_fixed)
  int32_t pre_ok;            // |sum1| < 2^(rs2 - 1): sum1 2^(32 - rs2) fits 32 bits, so the rounded
                             // product S sum1 is the high word of one 64-bit multiply-add
                             // (the merged nested kernel's pre-scaled form, family 24)
};

struct ItemDesc {
  // sample range and chunking
  uint64_t first, N;       // samples [first, first + N)
  uint64_t g0, g1;         // groups [g0, g1) covering the range
  uint64_t gf0, gf1;       // groups [gf0, gf1) lie entirely inside the sample range
  uint32_t groups_per_thread;
  uint32_t chunk_begin;    // first chunk (CTA) of this item within its launch
  uint32_t n_chunks;
  uint32_t out_index;      // index of this item's result record
  // method
  int32_t level, nlog;     // nlog = level (2^level fine steps)
  int32_t payoff, scheme, method, d;
  uint32_t ctr2, ctr3;     // Philox counter words 2 and 3: level | stream << 8, request
  int32_t unit;            // approximate payoff unit exponent
  int32_t enumerate;       // 1: table indices enumerate samples instead of Philox draws
  int32_t lanes;           // 3: packed draws with one sample per thread (sample s reads lane s mod 3
                           // of pack s / 3); levels >= 2, approximate-only, KP = 1 kernels
  int32_t kind;            // in a merged nested launch: 0 approximate packed, 1 approximate one
                           // sample per thread, 2 correction (nested_kernel)
  int32_t tab_y0;          // 1: a level-0 approximate item of the 32-bit fast datapath with a terminal
                           // payoff; its shared-memory table holds (Y_j, saturated_j), the sample value
                           // of every index j (its one fine step is a function of j alone)
  float unit_scale;        // 2^-unit (FP32, correction estimators)
  // exact path constants
  float c1f, c2f, c1cf, c3f, S0f, Kf;
  double c1d, c2d, c1cd, c3d, S0d, Kd;
  // approximate path
  FixedConsts fx;
  FastFixed ff;
  uint16_t h_c1, h_c1c, h_c2, h_c3, h_S0, h_pad;  // binary16 / bfloat16 bit patterns
  const void *ztab;        // device table for methods 1 and 2 (int32 / half bits), or method-3 coefficients
  const uint16_t *perm;    // method 2, correction estimators: interval rank pi(j) of every d-bit j
  // optional per-sample dump (device), indexed by sample - first
  void *dump;
};

// Per-CTA partial sums, written by the level kernel and summed in chunk order.
struct Partial {
  int64_t isum;
  uint64_t isum2_lo, isum2_hi;
  double dsum, dsum2;
  uint64_t nsat;
};

// Per-item result on the device (undiscounted).
struct DevSums {
  double dsum, dsum2;
  int64_t isum;
  uint64_t isum2_lo, isum2_hi;
  uint64_t nsat;
};

// Philox4x32-10 round keys (k0 + r W0, k1 + r W1), r = 0..9, precomputed on the host.
struct RoundKeys {
  uint32_t k[20];
};

// Item and chunk counts of a launch whose work is decided on the device (the
// engine's scheduler writes them before the launch; a CTA takes chunks
// blockIdx.x, blockIdx.x + gridDim.x, ...).
struct DynLaunch {
  uint32_t item_off;       // first item of the launch in LaunchArgs::items
  uint32_t n_items;
  uint32_t chunk0;         // global chunk index of the launch's first chunk
  uint32_t n_chunks;
};

// Launch-wide arguments of a level kernel (passed as a __grid_constant__ parameter).
struct LaunchArgs {
  const ItemDesc *items;   // the items of this launch, ordered by chunk_begin
  int n_items;
  uint32_t chunk0;         // global chunk index of blockIdx.x == 0
  Partial *partials;       // indexed by global chunk index
  RoundKeys rk;
  const DynLaunch *dyn;    // nullptr: one chunk per CTA, gridDim.x chunks
  // per item of the launch, zero between launches: the CTA that finishes an
  // item's last chunk sums its partials into out[out_index] (nullptr: a
  // separate kernel does)
  uint32_t *counters;
  DevSums *out;
  // nonzero: some item of the launch writes per-sample records (the launch
  // uses the kernel that holds the record-writing code)
  int dump;
};

#if defined(__CUDACC__)
#define MLMC_HD __host__ __device__
#else
#define MLMC_HD
#endif

// Sample groups.  A group is one Philox call's worth of packs (4 packs on level
// 0, 2 on level 1) or, from level 2, one pack over the 2^l / 4 calls of its
// path; a pack holds kp lockstep samples (kp = 3 with packed draws, else 1).
MLMC_HD inline uint64_t samples_per_group(int level, int kp) {
  return (uint64_t)kp * (level >= 2 ? 1u : (level == 1 ? 2u : 4u));
}
MLMC_HD inline uint64_t steps_per_group(int level) { return level >= 2 ? (1ULL << level) : 4ULL; }

// Chunking of an item of `groups` sample groups for CTAs of `threads` threads:
// about spt fine path-steps per thread (at least one group), but (with floor)
// no fewer than four CTAs per SM while the item has that many groups.  Returns
// the number of chunks (CTAs) and sets *gpt, the groups per thread.
MLMC_HD inline uint64_t chunk_count(uint64_t groups, uint64_t spg, int kp, int threads, int spt, int num_sms,
                                    uint32_t *gpt, bool floor = true) {
  uint64_t G = (uint64_t)spt / (spg * (uint64_t)kp);
  if (G < 1) G = 1;
  const uint64_t min_ctas = 4ULL * (uint64_t)(num_sms > 1 ? num_sms : 1);
  uint64_t cap = (groups + (uint64_t)threads * min_ctas - 1) / ((uint64_t)threads * min_ctas);
  if (cap < 1) cap = 1;
  if (floor && G > cap) G = cap;
  *gpt = (uint32_t)G;
  const uint64_t per_chunk = G * (uint64_t)threads;
  return (groups + per_chunk - 1) / per_chunk;
}

// Method-3 coefficient tables (Sec. 3.3): d-1 classes.
struct M3Coef {
  int64_t A[16], B[16];    // fixed point with M3_FRAC bits
  float a[16], b[16];
};
constexpr int M3_FRAC = 30;

}  // namespace mlmc
