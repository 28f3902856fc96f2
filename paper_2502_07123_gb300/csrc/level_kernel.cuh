// The MLMC level kernel: per-sample coupled fine/coarse GBM paths of one
// level (Sec. 2.1), exact Normals and/or table-based approximate Normals from
// the same uniform J (Sec. 3), the low-precision path in fixed point
// (Algorithm 1) or binary16/bfloat16, payoffs, the level difference / nested
// correction (eq. chap:nested_exp) and per-CTA sums of Y and Y^2.
//
// Layout: one CTA processes one chunk of one work item; each thread simulates
// groups of samples whose uniforms come from one Philox call per group (4
// packs per call on level 0, 2 on level 1, one pack over 2^l / 4 calls above;
// a pack is one sample, or three with packed draws), entirely in registers.  The approximate-Normal table of the item
// lives in shared memory.  The only global-memory traffic is the work-item
// descriptor, the table, one Partial record per CTA, the item's sums (written
// by the CTA that finishes its last chunk) and the optional dump.
#pragma once
#include <type_traits>

#include "device_common.cuh"
#include "mlmc.h"
#include "reduce.cuh"

namespace mlmc {

using mlmc_sample_rec = ::mlmc_sample;

// Words of "call" q when the table indices enumerate the samples (levels 0 and
// 1): sample s takes j_i = (s >> (d i)) mod 2^d at step i, placed in the top d
// bits; the word layout per call is the one of the Philox draws.
__device__ __forceinline__ uint4 enum_words(uint64_t q, int lev, int d) {
  const uint32_t mask = (1u << d) - 1u, sh = 32u - (uint32_t)d;
  if (lev == 0) {
    const uint32_t s = 4u * (uint32_t)q;
    return make_uint4((s & mask) << sh, ((s + 1u) & mask) << sh, ((s + 2u) & mask) << sh, ((s + 3u) & mask) << sh);
  }
  const uint32_t s0 = 2u * (uint32_t)q, s1 = s0 + 1u;
  return make_uint4((s0 & mask) << sh, ((s0 >> d) & mask) << sh, (s1 & mask) << sh, ((s1 >> d) & mask) << sh);
}

template <int XP> struct XType { using T = float; };
template <> struct XType<XP_F64> { using T = double; };
template <int AP> struct HType { using T = __half; };
template <> struct HType<AP_BF16> { using T = __nv_bfloat16; };
template <> struct HType<AP_BF16S> { using T = __nv_bfloat16; };

constexpr int MAX_THREADS = 256;
// Register budget: the approximate fixed-point Euler kernel with terminal payoffs
// (the bulk of the nested estimator) runs with 6 resident 128-thread CTAs per SM
// (80 registers per thread), measured faster than its natural ~100 registers.
// The matching correction kernel (static launch) takes the same budget, 80
// instead of 111 registers: alone it is 2% slower, but beside the approximate
// kernels of a work list its CTAs fit next to theirs and the step is 3% faster
// (its device-scheduled form would spill there and keeps its allocation).
// The approximate 32-bit fixed-point Asian kernels run 4 CTAs per SM (<= 128
// registers, measured 8-16% faster than their natural ~144).
// Every other instantiation keeps its natural allocation (a cap there spills).
constexpr int LAUNCH_THREADS = 128;
template <int EST, int AP, int SCHEME, int PC, bool DYN = false> struct MinCtas {
  static constexpr bool EM_TERMINAL_FX32 = AP == AP_FX32 && SCHEME == 0 && PC == PC_TERMINAL;
  static constexpr int value =
      (EM_TERMINAL_FX32 && (EST == EST_APPROX || (EST == EST_CORR && !DYN))) ? 6
      : ((EST == EST_APPROX && AP == AP_FX32 && PC == PC_ASIAN) ? 4 : 1);
};

// The inverse-Normal cubics of the FP32 exact path (phi_inv_table.h) in
// shared memory: 8 KB, the same for every item.  Kernels whose chunks run an
// FP32 exact path stage them once per CTA, before their first chunk's table
// (whose barrier makes them visible).
__device__ __forceinline__ float4 *phi_inv_smem() {
  __shared__ float4 s_phi_inv[PHI_INV_PARTS];
  return s_phi_inv;
}
__device__ __forceinline__ void stage_phi_inv() {
  float4 *d = phi_inv_smem();
  for (int k = threadIdx.x; k < PHI_INV_PARTS; k += blockDim.x) d[k] = k_phi_inv[k];
}
template <int EST, int XP>
struct NeedsPhi {
  static constexpr bool value = EST != EST_APPROX && XP == XP_F32;
};

// Bytes per entry of the shared-memory approximate-Normal table of a datapath:
// the 32-bit fast fixed-point datapath keeps (Z~_j, sum1 of a fine step) pairs.
template <int AP>
struct TabBytes {
  static constexpr size_t value = AP == AP_FX32 ? 8 : ((AP == AP_FIXED || AP == AP_FX64) ? 4 : 2);
};

// sum1 of one fast fixed-point step of Algorithm 1 from its Normal increment z:
// mul1 = rd(con2 z), [Milstein: mul3 = rd(con3 (z^2 - m))], sum1 = rd(con1 + mul1
// [+ mul3]).  c1r: con1 (fine) or con1_c (coarse) with sum1's rounding half unit;
// m: 1 (fine) or 2 (coarse) in units 2^-2fZ.  F32: the host proved every
// rounding shift below 32, so a product's rounded value is one funnel shift of
// its two words.
template <bool MIL, bool F32>
__device__ __forceinline__ int32_t ff_sum1(const FastFixed &ff, int32_t z, int32_t c1r, int64_t m) {
  int32_t mul1;
  const int64_t p1 = (int64_t)ff.con2 * z + ff.radd1;
  if constexpr (F32) mul1 = (int32_t)__funnelshift_r((uint32_t)p1, (uint32_t)((uint64_t)p1 >> 32), ff.rs1);
  else mul1 = (int32_t)(p1 >> ff.rs1);
  int32_t acc = c1r + mul1 * ff.mulF1;
  if constexpr (MIL) {
    // |Z~^2 - m| < 2^31 on this datapath (host-checked): one 32 x 32 product
    const int32_t zz = z * z - (int32_t)m;
    const int64_t p3 = (int64_t)ff.con3 * zz + ff.radd3;
    int32_t mul3;
    if constexpr (F32) mul3 = (int32_t)__funnelshift_r((uint32_t)p3, (uint32_t)((uint64_t)p3 >> 32), ff.rs3);
    else mul3 = (int32_t)(p3 >> ff.rs3);
    acc += mul3 * ff.mulF1;
  }
  return acc >> ff.rs_sum1;
}

// KP > 1 (approximate-only estimators): KP samples advance in lockstep, lane L
// reading bits [32 - d(L+1), 32 - dL) of the shared word (packed draws).
// MSEL: 0 the item uses a table lookup (Methods 1 and 2), 1 the line
// evaluation of Method 3, 2 either, chosen per step (only the per-sample
// dump instantiation); chosen once per chunk, so the hot step code has no
// branch on the method.
// PRE (merged nested kernel, family 24): the 32-bit fast datapath's sum1
// arrives multiplied by 2^(32 - rs2) (the host proved that it fits), so the
// rounded product rd(S sum1) is the high word of one 64-bit multiply-add: no
// funnel shift on the ALU pipe, which bounds that kernel.
// MERGED: the merged nested kernel's instantiation, which takes no enumerated
// items (the plan keeps those apart), so its group code has no enumeration
// branch.
template <int EST, int XP, int AP, int SCHEME, int PC, int KP = 1, int MSEL = 0, bool PRE = false,
          bool MERGED = false>
struct LevelSim {
  static_assert(KP == 1 || EST == EST_APPROX, "packed draws feed approximate-only estimators");
  static constexpr bool ENUMERATE = !MERGED;   // the group code reads enumerated words when asked
  static constexpr bool HAS_EXACT = (EST != EST_APPROX);
  static constexpr bool HAS_APPROX = (EST != EST_EXACT);
  static constexpr bool MIL = (SCHEME == 1);
  static constexpr bool FAST = (AP == AP_FX32 || AP == AP_FX64);
  static constexpr bool FIXED = (AP == AP_FIXED || FAST);
  static constexpr bool HALF = (AP == AP_F16 || AP == AP_BF16 || AP == AP_F16S || AP == AP_BF16S);
  // half increments with S (and its average and minimum) in FP32
  static constexpr bool S32 = (AP == AP_F16S || AP == AP_BF16S);
  // packed half draws: lanes 0 and 1 share paired (x2) registers, lane 2 is scalar
  static constexpr bool PAIR = HALF && KP == 3 && !S32;
  using AS = typename std::conditional<AP == AP_FX32, int32_t, int64_t>::type;  // fixed-point S
  // saturation flag of the fast datapath: OR of (clamped ^ unclamped) for a 32-bit S
  using SatT = typename std::conditional<AP == AP_FX32, uint32_t, bool>::type;
  // Approximate-only 32-bit datapath: when the host proved it exact (ff.lazy),
  // a group of packs first runs with S unclamped, tracking only its running
  // maximum hi; if hi stayed at or below lim_S no clamp would have acted and the
  // values are final, otherwise the group runs again on the clamped (EAGER)
  // datapath.
  static constexpr bool LAZY = (EST == EST_APPROX && AP == AP_FX32);
  static constexpr int KPV = KP;
  static constexpr int ESTV = EST;
  using X = typename XType<XP>::T;
  using H = typename HType<AP>::T;
  using HO = HalfOps<H>;
  using HO2 = HalfOps2<H>;
  using H2 = typename HO2::T;
  using HS = typename std::conditional<S32, float, H>::type;   // S of the half datapaths
  static __device__ __forceinline__ float sf(float x) { return x; }
  static __device__ __forceinline__ float sf(H x) { return HO::to_f(x); }

  // ---- per-item constants (registers) ----
  int level, nsteps, payoff, d, dshift, method;
  // FX32: byte offset of lane l's table entry = rotr(word, rot[l]) & off_mask
  int32_t pre2;            // PRE: 2^(32 - rs2), and radd2 times it
  int64_t radd2p;
  uint32_t rot[KP], off_mask;
  const uint16_t *perm_s;  // method 2 coupling of the exact path (shared memory), or nullptr
  const float4 *phi;       // FP32 exact path: the inverse-Normal cubics in shared memory
  uint32_t low_mask;
  X c1, c2, c1c, c3, S0, K;
  // fixed point
  FixedConsts fx;
  FastFixed ff;
  // half
  H hc1, hc1c, hc2, hc3;
  HS hS0;
  H2 pc1, pc1c, pc2, pc3;
  float K32;
  float unit_scale;
  const void *smem_tab;

  // ---- per-sample state (approximate state per lane) ----
  X S, Sc, zprev, accF, accC, minF, minC;
  AS aS[KP], aSc[KP], aminF[KP], aminC[KP];
  SatT satb[KP];
  AS hi;   // LAZY: running maximum of S over a group's lanes and steps (reset by the caller)
  int64_t aaccF[KP], aaccC[KP];
  int32_t azprev[KP];
  HS hS[KP], hSc[KP], hminF[KP], hminC[KP];
  H hzprev[KP];
  H2 pS, pSc, pzprev;   // lanes 0 and 1 when PAIR (hS[0..1] etc. then unused)
  float haccF[KP], haccC[KP];
  uint32_t sat[KP];

  __device__ __forceinline__ void load(const ItemDesc &it, const void *tab) {
    level = it.level;
    nsteps = 1 << it.level;
    payoff = it.payoff;
    d = it.d;
    dshift = 32 - it.d;
    method = it.method;
    if constexpr (XP == XP_F64) {
      c1 = it.c1d; c2 = it.c2d; c1c = it.c1cd; c3 = it.c3d; S0 = it.S0d; K = it.Kd;
    } else {
      c1 = it.c1f; c2 = it.c2f; c1c = it.c1cf; c3 = it.c3f; S0 = it.S0f; K = it.Kf;
    }
    if constexpr (FIXED) fx = it.fx;
    if constexpr (FAST) ff = it.ff;
    if constexpr (AP == AP_FX32 && PRE) {
      pre2 = 1 << (32 - it.ff.rs2);
      radd2p = (int64_t)((uint64_t)it.ff.radd2 << (32 - it.ff.rs2));
    }
    if constexpr (HALF) {
      hc1 = HO::from_bits(it.h_c1); hc1c = HO::from_bits(it.h_c1c);
      hc2 = HO::from_bits(it.h_c2); hc3 = HO::from_bits(it.h_c3);
      if constexpr (S32) hS0 = it.S0f;
      else hS0 = HO::from_bits(it.h_S0);
      K32 = it.Kf;
      if constexpr (PAIR) {
        pc1 = HO2::splat(hc1); pc1c = HO2::splat(hc1c); pc2 = HO2::splat(hc2); pc3 = HO2::splat(hc3);
      }
    }
    unit_scale = it.unit_scale;
    smem_tab = tab;
    if constexpr (AP == AP_FX32) {
      // lane l's field, bits [32 - d(l+1), 32 - d l) of the word, lands at bits [3, 3 + d)
#pragma unroll
      for (int l = 0; l < KP; ++l) rot[l] = (uint32_t)(32 - it.d * (l + 1) - 3) & 31u;
      off_mask = ((1u << it.d) - 1u) << 3;
    }
    perm_s = nullptr;
    if constexpr (HAS_EXACT && XP == XP_F32) phi = phi_inv_smem();
    low_mask = (1u << dshift) - 1u;
    if constexpr (EST == EST_CORR) {
      if (it.perm) perm_s = (const uint16_t *)((const unsigned char *)tab + ((size_t)1 << it.d) * TabBytes<AP>::value);
    }
  }

  __device__ __forceinline__ void begin() {
    if constexpr (HAS_EXACT) {
      S = S0; Sc = S0; zprev = X(0);
      accF = X(0.5) * S0; accC = accF; minF = S0; minC = S0;
    }
#pragma unroll
    for (int l = 0; l < KP; ++l) {
      if constexpr (FIXED) {
        aS[l] = (AS)fx.S0; aSc[l] = (AS)fx.S0; aaccF[l] = 0; aaccC[l] = 0; aminF[l] = aS[l]; aminC[l] = aS[l];
        azprev[l] = 0;
        satb[l] = SatT(0);
      }
      if constexpr (HALF) {
        hS[l] = hS0; hSc[l] = hS0; hzprev[l] = HO::from_f(0.0f); hminF[l] = hS0; hminC[l] = hS0;
        haccF[l] = __fmul_rn(0.5f, sf(hS0)); haccC[l] = haccF[l];
      }
      sat[l] = 0;
    }
    if constexpr (PAIR) {
      pS = HO2::splat(hS0); pSc = pS; pzprev = HO2::splat(HO::from_f(0.0f));
    }
  }
  // LAZY: did some S since hi was reset leave [-lim_S, lim_S]?  (The host
  // proved that it cannot leave below first.)
  __device__ __forceinline__ bool over() const { return hi > (AS)ff.limT; }

  // ---- exact path (FP32 / FP64) ----
  __device__ __forceinline__ X exact_inc(X z, X cc1, X mm) const {
    if constexpr (MIL) return fma(c3, fma(z, z, -mm), fma(c2, z, cc1));
    else return fma(c2, z, cc1);
  }

  // ---- fixed-point Algorithm-1 step ----
  __device__ __forceinline__ int64_t fx_step(int64_t s, int32_t z, int64_t con1A, int m, uint32_t &sat) {
    const int64_t mul1 = saturate(requant((int64_t)fx.con2 * z, fx.q_mul1), fx.lim[3], sat);
    int64_t acc = con1A + (int64_t)((uint64_t)mul1 << fx.sh_mul1_F1);
    if constexpr (MIL) {
      const int64_t zz = (int64_t)z * z - ((int64_t)m << fx.fZ2);
      const int64_t mul3 = saturate(requant((int64_t)fx.con3 * zz, fx.q_mul3), fx.lim[3], sat);
      acc += (int64_t)((uint64_t)mul3 << fx.sh_mul1_F1);
    }
    const int64_t sum1 = saturate(requant(acc, fx.q_sum1), fx.lim[4], sat);
    const int64_t mul2 = saturate(requant(s * sum1, fx.q_mul2), fx.lim[5], sat);
    const int64_t s2 = (int64_t)((uint64_t)s << fx.sh_S_F2) + (int64_t)((uint64_t)mul2 << fx.sh_mul2_F2);
    return saturate(requant(s2, fx.q_S), fx.lim[6], sat);
  }

  // ---- fast fixed-point Algorithm-1 step (same values as fx_step while S stays in range) ----
  // The S update of a step whose sum1 is known: mul2 = rd(S sum1), S = rd(S + mul2).
  // TRACK (lazy runs): count this S in the pack's maximum (fast_fixed's limT)
  template <bool EAGER, bool TRACK = true>
  __device__ __forceinline__ AS ff_apply(AS s, int32_t sum1, SatT &satb) {
    if constexpr (AP == AP_FX32 && PRE) {
      const int64_t p2 = (int64_t)s * sum1 + radd2p;
      const int32_t mul2 = (int32_t)((uint64_t)p2 >> 32);
      s = (int32_t)((uint32_t)s + (uint32_t)mul2 * (uint32_t)ff.mulS);
    } else if constexpr (AP == AP_FX32) {
      const int64_t p2 = (int64_t)s * sum1 + ff.radd2;
      const int32_t mul2 = (int32_t)__funnelshift_r((uint32_t)p2, (uint32_t)((uint64_t)p2 >> 32), ff.rs2);
      s = (int32_t)((uint32_t)s + (uint32_t)mul2 * (uint32_t)ff.mulS);
    } else {
      const int32_t mul2 = (int32_t)((int64_t)((uint64_t)s * (uint64_t)(int64_t)sum1 + (uint64_t)ff.radd2) >> ff.rs2);
      s = (int64_t)((uint64_t)s + (uint64_t)((int64_t)mul2 * ff.mulS));
    }
    if constexpr (LAZY && !EAGER) {
      if constexpr (TRACK) hi = max(hi, s);
      return s;
    }
    // saturation of S (the only variable the host could not bound)
    const AS lim = (AS)ff.limS;
    const AS c = min(max(s, -lim), lim);
    if constexpr (AP == AP_FX32) satb |= (uint32_t)(c ^ s);
    else satb |= (c != s);
    return c;
  }
  template <bool EAGER>
  __device__ __forceinline__ AS ff_step(AS s, int32_t z, int32_t c1r, int64_t m, SatT &satb) {
    if constexpr (AP == AP_FX32 && PRE) return ff_apply<EAGER>(s, ff_sum1<MIL, true>(ff, z, c1r, m) * pre2, satb);
    else return ff_apply<EAGER>(s, ff_sum1<MIL, AP == AP_FX32>(ff, z, c1r, m), satb);
  }
  // FX32: (Z~, sum1 of a fine step) of lane l of word w, from the shared-memory pairs
  // (the table sits at the start of the dynamic shared memory: addressing it
  // there, rather than through smem_tab, leaves the base to the load's
  // immediate offset, one add fewer per lookup)
  __device__ __forceinline__ int2 fx32_entry(uint32_t w, int l) const {
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    const uint32_t off = __funnelshift_r(w, w, rot[l]) & off_mask;
    return *(const int2 *)(smem_dyn + off);
  }

  // ---- half-precision step (one rounding per operation) ----
  // With S32 only the increment sum1 is in half precision; S is updated in
  // FP32 (mul2 = fl32(S sum1), S = fl32(S + mul2)).
  __device__ __forceinline__ HS h_step(HS s, H z, H cc1, H mh) const {
    const H mul1 = HO::mul(hc2, z);
    H sum1 = HO::add(cc1, mul1);
    if constexpr (MIL) {
      const H sq = HO::mul(z, z);
      const H sqm = HO::sub(sq, mh);
      const H mul3 = HO::mul(hc3, sqm);
      sum1 = HO::add(sum1, mul3);
    }
    if constexpr (S32) {
      return __fadd_rn(s, __fmul_rn(s, HO::to_f(sum1)));
    } else {
      const H mul2 = HO::mul(s, sum1);
      return HO::add(s, mul2);
    }
  }
  // the same step on two lanes at once
  __device__ __forceinline__ H2 h2_step(H2 s, H2 z, H2 cc1, H2 mh) const {
    const H2 mul1 = HO2::mul(pc2, z);
    H2 sum1 = HO2::add(cc1, mul1);
    if constexpr (MIL) {
      const H2 sq = HO2::mul(z, z);
      const H2 sqm = HO2::sub(sq, mh);
      const H2 mul3 = HO2::mul(pc3, sqm);
      sum1 = HO2::add(sum1, mul3);
    }
    const H2 mul2 = HO2::mul(s, sum1);
    return HO2::add(s, mul2);
  }
  // lane l's half state (fine / coarse)
  __device__ __forceinline__ HS lane_S(int l) const {
    if constexpr (PAIR) { if (l == 0) return HO2::lo(pS); if (l == 1) return HO2::hi(pS); }
    return hS[l];
  }
  __device__ __forceinline__ HS lane_Sc(int l) const {
    if constexpr (PAIR) { if (l == 0) return HO2::lo(pSc); if (l == 1) return HO2::hi(pSc); }
    return hSc[l];
  }
  __device__ __forceinline__ static void lane_min(HS &mn, HS x) { mn = sf(x) < sf(mn) ? x : mn; }

  // Approximate Normal of J in Z's fixed-point format: Method 1 reads the
  // signed table at j = top d bits of J; Method 3 evaluates the class line.
  __device__ __forceinline__ int32_t fixed_z(uint32_t J) const {
    if constexpr (MSEL == 0) return ((const int32_t *)smem_tab)[J >> dshift];
    if constexpr (MSEL == 2) {
      if (method != 3) return ((const int32_t *)smem_tab)[J >> dshift];
    }
    const ApproxIndex ai = approx_index(J, d);
    int32_t v;
    {
      const M3Coef *m3 = (const M3Coef *)smem_tab;
      const int c = m3_class(ai.idx);
      const int64_t t = m3->A[c] + m3->B[c] * (int64_t)ai.idx;
      const int sh = M3_FRAC - fx.fZ2 / 2;
      v = (int32_t)((t + ((int64_t)1 << (sh - 1))) >> sh);
    }
    return ai.neg ? -v : v;
  }

  __device__ __forceinline__ H half_z(uint32_t J) const {
    if constexpr (MSEL == 0) return HO::from_bits(((const uint16_t *)smem_tab)[J >> dshift]);
    if constexpr (MSEL == 2) {
      if (method != 3) return HO::from_bits(((const uint16_t *)smem_tab)[J >> dshift]);
    }
    const ApproxIndex ai = approx_index(J, d);
    H v;
    {
      const M3Coef *m3 = (const M3Coef *)smem_tab;
      const int c = m3_class(ai.idx);
      v = HO::from_f(fmaf(m3->b[c], (float)ai.idx, m3->a[c]));
    }
    return ai.neg ? HO::neg(v) : v;
  }

  // One fine step i driven by J, and the coarse step after odd i (levels >= 1).
  // PAR: parity of i when known at compile time (0 even, 1 odd), -1 otherwise.
  template <bool COARSE, int PAR = -1, bool EAGER = true>
  __device__ __forceinline__ void step(uint32_t J, int i) {
    const bool odd = PAR >= 0 ? (PAR == 1) : ((i & 1) != 0);
    if constexpr (HAS_EXACT) {
      // Method 2 (Sec. 3.2): the exact path takes the uniform in the interval
      // pi(j) that the approximate value of j is ranked at, with J's low bits
      const uint32_t Je = perm_s ? (((uint32_t)perm_s[J >> dshift] << dshift) | (J & low_mask)) : J;
      X z;
      if constexpr (XP == XP_F64) z = exact_normal_f64(Je);
      else z = exact_normal_f32(Je, phi);
      if constexpr (PC == PC_ASIAN) { if (i > 0) accF = accF + S; }
      S = fma(S, exact_inc(z, c1, X(1)), S);
      if constexpr (PC == PC_LOOKBACK) minF = fmin(minF, S);
      if constexpr (COARSE) {
        if (odd) {
          const X zc = zprev + z;
          if constexpr (PC == PC_ASIAN) { if (i > 1) accC = accC + Sc; }
          Sc = fma(Sc, exact_inc(zc, c1c, X(2)), Sc);
          if constexpr (PC == PC_LOOKBACK) minC = fmin(minC, Sc);
        } else {
          zprev = z;
        }
      }
    }
    if constexpr (PAIR) {
      // Algorithm-1 arithmetic of lanes 0 and 1 in paired instructions; lane 2 alone
      const H z0 = half_z(J), z1 = half_z(J << d), z2 = half_z(J << (2 * d));
      const H2 z01 = HO2::pack(z0, z1);
      if constexpr (PC == PC_ASIAN) {
        if (i > 0) {
          haccF[0] = __fadd_rn(haccF[0], HO::to_f(HO2::lo(pS)));
          haccF[1] = __fadd_rn(haccF[1], HO::to_f(HO2::hi(pS)));
          haccF[2] = __fadd_rn(haccF[2], HO::to_f(hS[2]));
        }
      }
      pS = h2_step(pS, z01, pc1, HO2::splat(HO::from_f(1.0f)));
      hS[2] = h_step(hS[2], z2, hc1, HO::from_f(1.0f));
      if constexpr (PC == PC_LOOKBACK) {
        lane_min(hminF[0], HO2::lo(pS)); lane_min(hminF[1], HO2::hi(pS)); lane_min(hminF[2], hS[2]);
      }
      if constexpr (COARSE) {
        if (odd) {
          const H2 zc01 = HO2::add(pzprev, z01);
          const H zc2 = HO::add(hzprev[2], z2);
          if constexpr (PC == PC_ASIAN) {
            if (i > 1) {
              haccC[0] = __fadd_rn(haccC[0], HO::to_f(HO2::lo(pSc)));
              haccC[1] = __fadd_rn(haccC[1], HO::to_f(HO2::hi(pSc)));
              haccC[2] = __fadd_rn(haccC[2], HO::to_f(hSc[2]));
            }
          }
          pSc = h2_step(pSc, zc01, pc1c, HO2::splat(HO::from_f(2.0f)));
          hSc[2] = h_step(hSc[2], zc2, hc1c, HO::from_f(2.0f));
          if constexpr (PC == PC_LOOKBACK) {
            lane_min(hminC[0], HO2::lo(pSc)); lane_min(hminC[1], HO2::hi(pSc)); lane_min(hminC[2], hSc[2]);
          }
        } else {
          pzprev = z01;
          hzprev[2] = z2;
        }
      }
    } else if constexpr (AP == AP_FX32) {
      // the fine step's sum1 comes with Z~ from the table; the coarse step forms
      // its own from Z~_2k + Z~_2k+1
#pragma unroll
      for (int l = 0; l < KP; ++l) {
        const int2 e = fx32_entry(J, l);
        if constexpr (PC == PC_ASIAN) { if (i > 0) aaccF[l] += aS[l]; }
        // lazy runs track S after the odd fine steps only (limT); with the parity
        // unknown at compile time, after every step (more is as exact)
        constexpr bool TRACK_FINE = PAR == 1 || (PAR == -1 && COARSE);
        aS[l] = ff_apply<EAGER, TRACK_FINE>(aS[l], e.y, satb[l]);
        if constexpr (PC == PC_LOOKBACK) aminF[l] = aS[l] < aminF[l] ? aS[l] : aminF[l];
        if constexpr (COARSE) {
          if (odd) {
            if constexpr (PC == PC_ASIAN) { if (i > 1) aaccC[l] += aSc[l]; }
            aSc[l] = ff_step<EAGER>(aSc[l], azprev[l] + e.x, ff.con1cr, ff.mcoarse, satb[l]);
            if constexpr (PC == PC_LOOKBACK) aminC[l] = aSc[l] < aminC[l] ? aSc[l] : aminC[l];
          } else {
            azprev[l] = e.x;
          }
        }
      }
    } else if constexpr (HAS_APPROX) {
#pragma unroll
      for (int l = 0; l < KP; ++l) {
        const uint32_t Jl = l == 0 ? J : (J << (d * l));  // this lane's field at the top
        if constexpr (FIXED) {
          const int32_t z = fixed_z(Jl);
          if constexpr (PC == PC_ASIAN) { if (i > 0) aaccF[l] += aS[l]; }
          if constexpr (FAST) aS[l] = ff_step<EAGER>(aS[l], z, ff.con1r, ff.mfine, satb[l]);
          else aS[l] = fx_step(aS[l], z, fx.con1A, 1, sat[l]);
          if constexpr (PC == PC_LOOKBACK) aminF[l] = aS[l] < aminF[l] ? aS[l] : aminF[l];
          if constexpr (COARSE) {
            if (odd) {
              if constexpr (PC == PC_ASIAN) { if (i > 1) aaccC[l] += aSc[l]; }
              if constexpr (FAST) aSc[l] = ff_step<EAGER>(aSc[l], azprev[l] + z, ff.con1cr, ff.mcoarse, satb[l]);
              else aSc[l] = fx_step(aSc[l], azprev[l] + z, fx.con1cA, 2, sat[l]);
              if constexpr (PC == PC_LOOKBACK) aminC[l] = aSc[l] < aminC[l] ? aSc[l] : aminC[l];
            } else {
              azprev[l] = z;
            }
          }
        } else {
          const H z = half_z(Jl);
          if constexpr (PC == PC_ASIAN) { if (i > 0) haccF[l] = __fadd_rn(haccF[l], sf(hS[l])); }
          hS[l] = h_step(hS[l], z, hc1, HO::from_f(1.0f));
          if constexpr (PC == PC_LOOKBACK) lane_min(hminF[l], hS[l]);
          if constexpr (COARSE) {
            if (odd) {
              const H zc = HO::add(hzprev[l], z);
              if constexpr (PC == PC_ASIAN) { if (i > 1) haccC[l] = __fadd_rn(haccC[l], sf(hSc[l])); }
              hSc[l] = h_step(hSc[l], zc, hc1c, HO::from_f(2.0f));
              if constexpr (PC == PC_LOOKBACK) lane_min(hminC[l], hSc[l]);
            } else {
              hzprev[l] = z;
            }
          }
        }
      }
    }
  }

  // ---- payoffs ----
  __device__ __forceinline__ X exact_payoff(X x, X acc, X mn, int steps) const {
    if constexpr (PC == PC_TERMINAL) {
      if (payoff == 1) return x > K ? X(1) : X(0);
      const X dd = x - K;
      return dd > X(0) ? dd : X(0);
    } else if constexpr (PC == PC_ASIAN) {
      // one explicit multiply-add: every instantiation rounds the average alike
      const X avg = fma(X(0.5), x, acc) * (X(1) / X(steps));
      const X dd = avg - K;
      return dd > X(0) ? dd : X(0);
    } else {
      return x - mn;
    }
  }
  // PAY: the terminal payoff when known at compile time (0 European, 1 digital), -1 otherwise
  template <int PAY = -1>
  __device__ __forceinline__ int64_t fixed_payoff(int64_t x, int64_t inner, int64_t mn, int steps, bool coarse) const {
    if constexpr (PC == PC_TERMINAL && AP == AP_FX32) {
      // S, K < 2^31 on this datapath: 32-bit arithmetic
      const int32_t x32 = (int32_t)x, K32v = (int32_t)fx.K;
      const bool digital = PAY >= 0 ? PAY == 1 : payoff == 1;
      const int32_t v = digital ? (int32_t)1 << fx.fS : x32 - K32v;
      return x32 > K32v ? v : 0;
    } else if constexpr (PC == PC_TERMINAL) {
      if (payoff == 1) return x > fx.K ? ((int64_t)1 << fx.fS) : 0;
      return x > fx.K ? x - fx.K : 0;
    } else if constexpr (PC == PC_ASIAN) {
      const int64_t twice = fx.S0 + 2 * inner + x;
      const int64_t twoNK = 2 * (int64_t)steps * fx.K;
      const int64_t v = twice > twoNK ? twice - twoNK : 0;
      return coarse ? 2 * v : v;
    } else {
      return x - mn;
    }
  }
  __device__ __forceinline__ int64_t half_payoff(HS x, float acc, HS mn, int steps) const {
    float P;
    const float xf = sf(x);
    if constexpr (PC == PC_TERMINAL) {
      if (payoff == 1) {
        P = xf > K32 ? 1.0f : 0.0f;
      } else {
        const float dd = __fsub_rn(xf, K32);
        P = dd > 0.0f ? dd : 0.0f;
      }
    } else if constexpr (PC == PC_ASIAN) {
      const float tot = __fadd_rn(acc, __fmul_rn(0.5f, xf));
      const float avg = __fmul_rn(tot, 1.0f / (float)steps);
      const float dd = __fsub_rn(avg, K32);
      P = dd > 0.0f ? dd : 0.0f;
    } else {
      P = __fsub_rn(xf, sf(mn));
    }
    return __float2ll_rn(__fmul_rn(P, 16777216.0f));
  }

  // Finish the sample: payoffs, sample value, accumulation and optional dump
  // (EAGER false: a LAZY pack that stayed in range, so no saturation).
  // LV: 0 on level 0 (no coarse path), 1 on levels >= 1, -1 not known at compile time.
  template <bool EAGER = true, int PAY = -1, int LV = -1, class Acc>
  __device__ __forceinline__ void finish(Acc &acc, int l, bool valid, mlmc_sample_rec *dump) {
    X pf = X(0), pc = X(0);
    int64_t qf = 0, qc = 0, afS = 0, acS = 0;
    uint32_t lsat = 0;
    const bool coarse = LV >= 0 ? LV == 1 : level > 0;
    if constexpr (HAS_EXACT) {
      pf = exact_payoff(S, accF, minF, nsteps);
      if (coarse) pc = exact_payoff(Sc, accC, minC, nsteps >> 1);
    }
    if constexpr (FIXED) {
      qf = fixed_payoff<PAY>(aS[l], aaccF[l], aminF[l], nsteps, false);
      if (coarse) qc = fixed_payoff<PAY>(aSc[l], aaccC[l], aminC[l], nsteps >> 1, true);
      afS = aS[l];
      acS = aSc[l];
      if constexpr (FAST) lsat = (EAGER && satb[l]) ? 1u : 0u;
      else lsat = sat[l];
    }
    if constexpr (HALF) {
      if constexpr (HAS_APPROX) {
        qf = half_payoff(lane_S(l), haccF[l], hminF[l], nsteps);
        if (coarse) qc = half_payoff(lane_Sc(l), haccC[l], hminC[l], nsteps >> 1);
      }
    }
    double ydump;
    if constexpr (EST == EST_APPROX && AP == AP_FX32 && PC == PC_TERMINAL) {
      // a sample outside the item's range adds zero to the group sums, so the
      // range test does not branch the group's straight-line code (|Y| < 2^31
      // here and the host bounds a group's sum of squares below 2^64)
      const int32_t yi = valid ? (int32_t)(qf - qc) : 0;
      acc.add_group(yi);
      acc.nsat += valid ? lsat : 0u;
      if (!valid) return;
      ydump = (double)yi * (double)unit_scale;
    } else if constexpr (EST == EST_APPROX) {
      if (!valid) return;
      const int64_t yi = qf - qc;
      acc.add_int(yi);
      acc.nsat += lsat;
      ydump = (double)yi * (double)unit_scale;
    } else {
      if (!valid) return;
      if constexpr (EST == EST_EXACT) {
        const X y = pf - pc;
        acc.add_real(y);
        ydump = (double)y;
      } else {
        const float yx = (float)(pf - pc);
        const float ya = __fmul_rn(__ll2float_rn(qf - qc), unit_scale);
        const float y = __fsub_rn(yx, ya);
        acc.add_real(y);
        ydump = (double)y;
      }
      acc.nsat += lsat;
    }
    if (dump) {
      mlmc_sample_rec r;
      r.pf = (double)pf; r.pc = (double)pc;
      r.sf = HAS_EXACT ? (double)S : 0.0;
      r.sc = (HAS_EXACT && level > 0) ? (double)Sc : 0.0;
      if constexpr (FIXED) {
        r.af = ldexp((double)afS, -fx.fS);
        r.ac = level > 0 ? ldexp((double)acS, -fx.fS) : 0.0;
      } else if constexpr (HALF) {
        r.af = HAS_APPROX ? (double)sf(lane_S(l)) : 0.0;
        r.ac = (HAS_APPROX && level > 0) ? (double)sf(lane_Sc(l)) : 0.0;
      } else {
        r.af = 0.0; r.ac = 0.0;
      }
      r.qf = qf; r.qc = qc; r.y = ydump; r.sat = lsat; r.pad = 0;
      *dump = r;
    }
  }
};

// Samples of an FP32 real-valued estimator summed in a float pair before each
// FP64 flush (see ThreadAcc::add_real).
constexpr int REAL_FLUSH_SAMPLES = 8;

// Per-thread accumulator
template <int EST, int XP>
struct ThreadAcc {
  // integer estimators
  int64_t isum;
  uint64_t q_lo, q_hi;
  // real-valued estimators: FP64 sums (FP64 exact path: every sample; FP32
  // paths and corrections: the float pairs below, flushed)
  double ds, dq;
  // float pairs (s + c) of sum Y and sum Y^2 since the last flush
  float fs, fc, fs2, fc2;
  uint32_t nsat;
  __device__ __forceinline__ void init() {
    isum = 0; q_lo = 0; q_hi = 0; gsum = 0; gq = 0; ds = 0.0; dq = 0.0; nsat = 0;
    fs = 0.0f; fc = 0.0f; fs2 = 0.0f; fc2 = 0.0f;
  }
  __device__ __forceinline__ void add_int(int64_t y) {
    isum += y;
    add_square(q_lo, q_hi, y);
  }
  // Two wide multiply-adds per sample (FMA pipe): the group's sum of y and of
  // y^2 in 64 bits; flush_group() adds them into the totals (and
  // discard_group() drops a group that must be redone).
  int64_t gsum;
  uint64_t gq;
  __device__ __forceinline__ void add_group(int32_t y) {
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(gsum) : "r"(y), "r"(1));
    asm("mad.wide.s32 %0, %1, %1, %0;" : "+l"(gq) : "r"(y));
  }
  __device__ __forceinline__ void flush_group() {
    isum += gsum;
    add_u128(q_lo, q_hi, gq, 0);
    gsum = 0;
    gq = 0;
  }
  __device__ __forceinline__ void discard_group() {
    gsum = 0;
    gq = 0;
  }
  // Integer sums at the start of a group, to undo the group's samples (the
  // path-dependent payoffs add each sample to the totals directly).
  struct Mark {
    int64_t isum;
    uint64_t q_lo, q_hi;
  };
  __device__ __forceinline__ Mark mark() const { return Mark{isum, q_lo, q_hi}; }
  __device__ __forceinline__ void rewind(const Mark &m) {
    isum = m.isum; q_lo = m.q_lo; q_hi = m.q_hi;
  }
  // s + y = t + e exactly (Knuth's TwoSum, six FP32 operations); e goes to c.
  static __device__ __forceinline__ void two_sum_into(float &s, float &c, float y) {
    const float t = __fadd_rn(s, y);
    const float z = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(y, z));
    s = t;
    c = __fadd_rn(c, e);
  }
  // A real sample.  FP64 samples are added in FP64.  An FP32 sample y enters
  // the float pair (fs, fc) by TwoSum, so fs + fc misses sum y only by the
  // roundings of the additions into fc; y^2 = p + pe exactly (p = fl(y y),
  // pe = fma(y, y, -p)) enters (fs2, fc2) the same way.  With at most K =
  // REAL_FLUSH_SAMPLES samples between flushes (|fc| <= k u sum |y| after k of
  // them, |fc2| <= (k+1) u sum y^2, u = 2^-24) those roundings total at most
  // u^2 K(K+1)/2 sum |y| and 2 u^2 (K(K+1)/2 + K) sum y^2: below 1.3e-13 of
  // sum |y| and 3.2e-13 of sum y^2.  A flush adds each float, exactly widened,
  // into the FP64 sums, so the thread's sums are within about 3.5e-13 of the
  // exact sums of its samples, at one FP64 operation per sample.
  template <class T>
  __device__ __forceinline__ void add_real(T y) {
    if constexpr (XP == XP_F64 && EST == EST_EXACT) {
      ds += (double)y;
      dq = fma((double)y, (double)y, dq);
    } else {
      const float yf = (float)y;
      two_sum_into(fs, fc, yf);
      const float p = __fmul_rn(yf, yf);
      const float pe = __fmaf_rn(yf, yf, -p);
      two_sum_into(fs2, fc2, p);
      fc2 = __fadd_rn(fc2, pe);
    }
  }
  __device__ __forceinline__ void flush_real() {
    if constexpr (!(XP == XP_F64 && EST == EST_EXACT) && EST != EST_APPROX) {
      ds += (double)fs;
      ds += (double)fc;
      dq += (double)fs2;
      dq += (double)fc2;
      fs = 0.0f; fc = 0.0f; fs2 = 0.0f; fc2 = 0.0f;
    }
  }
};

template <class T>
__device__ __forceinline__ T shfl_xor(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

// Reduce the CTA's thread accumulators into one Partial (thread 0 writes it).
// Approximate-only estimators have integer sums only, the others real sums
// only, so each shuffles just its own.
template <int EST, int XP>
__device__ __forceinline__ void block_reduce_write(ThreadAcc<EST, XP> &a, Partial *out) {
  constexpr bool INT = EST == EST_APPROX;
  int64_t isum = INT ? a.isum : 0;
  uint64_t lo = INT ? a.q_lo : 0, hi = INT ? a.q_hi : 0;
  double ds = INT ? 0.0 : a.ds, dq = INT ? 0.0 : a.dq;
  uint32_t ns = a.nsat;
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    if constexpr (INT) {
      isum += shfl_xor((long long)isum, m);
      const uint64_t olo = (uint64_t)shfl_xor((unsigned long long)lo, m);
      const uint64_t ohi = (uint64_t)shfl_xor((unsigned long long)hi, m);
      add_u128(lo, hi, olo, ohi);
    } else {
      ds += shfl_xor(ds, m);
      dq += shfl_xor(dq, m);
    }
    ns += shfl_xor(ns, m);
  }
  __shared__ Partial wp[LAUNCH_THREADS / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    Partial p;
    p.isum = isum; p.isum2_lo = lo; p.isum2_hi = hi; p.dsum = ds; p.dsum2 = dq; p.nsat = ns;
    wp[warp] = p;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Partial t = wp[0];
    const int nw = blockDim.x >> 5;
    for (int w = 1; w < nw; ++w) {
      t.isum += wp[w].isum;
      add_u128(t.isum2_lo, t.isum2_hi, wp[w].isum2_lo, wp[w].isum2_hi);
      t.dsum += wp[w].dsum;
      t.dsum2 += wp[w].dsum2;
      t.nsat += wp[w].nsat;
    }
    *out = t;
  }
}

template <int P> using PayTag = std::integral_constant<int, P>;

// The compiler may not reuse a value computed before this point: the clamped
// re-run of a LAZY group recomputes its draws instead of keeping the first
// run's live in registers through the group.
__device__ __forceinline__ void opaque(uint64_t &x) { asm volatile("" : "+l"(x)); }

// The item fields the group code reads, copied into registers once per chunk
// (read through the item reference they would be loaded again for every
// group: the kernel's stores to global memory might alias them).
struct GroupCtx {
  uint32_t ctr2, ctr3;
  int d, level, enumerate, lanes;
  uint64_t first, last;
};

// The samples of group g of a chunk, for a level class LC known at compile
// time (0: level 0, 1: level 1, 2: levels >= 2).  A group is one Philox call's
// worth of packs (4 on level 0, 2 on level 1) or, from level 2, one pack over
// 2^l / 4 calls; a pack holds KP samples.  E: the clamped datapath (LAZY
// kernels; always true elsewhere); FULL: every sample of the group is in the
// item's range at compile time (then no per-sample range test splits the
// group's straight-line code); full: the same known at run time; PAY: the
// terminal payoff when fixed at compile time (0 European, 1 digital, -1 not).
template <int LC, bool E, bool FULL, int PAY, bool DUMP, class Sim, class Acc>
__device__ __forceinline__ void run_group(Sim &sim, Acc &acc, const LaunchArgs &args, const GroupCtx &it, uint64_t g,
                                          bool full, uint64_t first, uint64_t last, mlmc_sample_rec *dump) {
  constexpr int KP = Sim::KPV;
  if constexpr (LC == 2) {
    uint64_t P = g;
    uint32_t lsh = 0;   // lane-split packed draws: this sample's field to the top of the word
    if constexpr (KP == 1 && Sim::ESTV == EST_APPROX) {
      if (it.lanes > 1) {
        P = g / 3u;
        lsh = (uint32_t)it.d * (uint32_t)(g - P * 3u);
      }
    }
    const uint32_t calls = 1u << (it.level - 2);
    uint64_t qbase = P * calls;
    if constexpr (E && Sim::LAZY) opaque(qbase);
    sim.begin();
    for (uint32_t c = 0; c < calls; ++c) {
      const uint64_t q = qbase + c;
      const uint4 w = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), it.ctr2, it.ctr3), args.rk);
      const int i0 = (int)(c << 2);
      sim.template step<true, 0, E>(w.x << lsh, i0);
      sim.template step<true, 1, E>(w.y << lsh, i0 + 1);
      sim.template step<true, 0, E>(w.z << lsh, i0 + 2);
      sim.template step<true, 1, E>(w.w << lsh, i0 + 3);
    }
#pragma unroll
    for (int l = 0; l < KP; ++l) {
      const uint64_t s = KP == 1 ? g : P * KP + l;
      const bool valid = FULL || full || (s >= first && s < last);
      sim.template finish<E, PAY, 1>(acc, l, valid, DUMP && valid ? dump + (s - first) : nullptr);
    }
  } else {
    uint64_t gw = g;
    if constexpr (E && Sim::LAZY) opaque(gw);
    uint4 w;
    if constexpr (Sim::ENUMERATE)
      w = it.enumerate ? enum_words(gw, LC, it.d)
                       : philox4x32_10(make_uint4((uint32_t)gw, (uint32_t)(gw >> 32), it.ctr2, it.ctr3), args.rk);
    else
      w = philox4x32_10(make_uint4((uint32_t)gw, (uint32_t)(gw >> 32), it.ctr2, it.ctr3), args.rk);
    constexpr int PPG = LC == 1 ? 2 : 4;  // packs per group
    const uint64_t s0 = (uint64_t)(PPG * KP) * g;
    // samples s0 + k are valid for k in [klo, khi)
    int klo = 0, khi = PPG * KP;
    if (!FULL && !full) {
      klo = s0 >= first ? 0 : (int)min(first - s0, (uint64_t)(PPG * KP));
      khi = last <= s0 ? 0 : (int)min(last - s0, (uint64_t)(PPG * KP));
    }
    if constexpr (LC == 1) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        sim.begin();
        sim.template step<true, 0, E>(u == 0 ? w.x : w.z, 0);
        sim.template step<true, 1, E>(u == 0 ? w.y : w.w, 1);
#pragma unroll
        for (int l = 0; l < KP; ++l) {
          const int k = u * KP + l;
          const bool valid = FULL || (k >= klo && k < khi);
          sim.template finish<E, PAY, 1>(acc, l, valid, DUMP && valid ? dump + (s0 + k - first) : nullptr);
        }
      }
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        sim.begin();
        sim.template step<false, -1, E>(word_of(w, u), 0);
#pragma unroll
        for (int l = 0; l < KP; ++l) {
          const int k = u * KP + l;
          const bool valid = FULL || (k >= klo && k < khi);
          sim.template finish<E, PAY, 0>(acc, l, valid, DUMP && valid ? dump + (s0 + k - first) : nullptr);
        }
      }
    }
  }
}

// One level-0 group of an item whose table holds each index's sample value
// (ItemDesc::tab_y0): per sample one table read and the two group sums.
// Samples k outside [klo, khi) add zero (FULL: the whole group is in range).
template <bool FULL, class Sim, class Acc>
__device__ __forceinline__ void y0_group(const Sim &sim, Acc &acc, const uint4 &w, int klo, int khi) {
  constexpr int KP = Sim::KPV;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
#pragma unroll
    for (int l = 0; l < KP; ++l) {
      const int k = u * KP + l;
      const int32_t y = sim.fx32_entry(word_of(w, u), l).x;
      acc.add_group(FULL || (k >= klo && k < khi) ? y : 0);
    }
  }
  acc.flush_group();
}

// The groups of a chunk of such an item: the same samples and values as
// run_group's path (no saturation: see tab_y0_of).
template <class Sim, class Acc>
__device__ __forceinline__ void group_loop_y0(const Sim &sim, Acc &acc, const LaunchArgs &args, const GroupCtx &it,
                                              uint64_t gbeg, uint32_t ng, uint32_t rf0, uint32_t rf1) {
  constexpr int KP = Sim::KPV;
  const uint64_t first = it.first, last = it.last;
  for (uint32_t r = threadIdx.x; r < ng; r += blockDim.x) {
    const uint64_t g = gbeg + r;
    uint4 w;
    if constexpr (Sim::ENUMERATE)
      w = it.enumerate ? enum_words(g, 0, it.d)
                       : philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), it.ctr2, it.ctr3), args.rk);
    else
      w = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), it.ctr2, it.ctr3), args.rk);
    if (r >= rf0 && r < rf1) {
      y0_group<true>(sim, acc, w, 0, 0);
    } else {
      const uint64_t s0 = (uint64_t)(4 * KP) * g;
      const int klo = s0 >= first ? 0 : (int)min(first - s0, (uint64_t)(4 * KP));
      const int khi = last <= s0 ? 0 : (int)min(last - s0, (uint64_t)(4 * KP));
      y0_group<false>(sim, acc, w, klo, khi);
    }
  }
}

// A thread's groups of one chunk, groups gbeg + r for r = threadIdx.x,
// threadIdx.x + blockDim.x, ... < ng, of level class LC; groups with r in
// [rf0, rf1) lie entirely in the item's range.  LAZY items run each such group
// first with S unclamped and its samples added tentatively; a group whose S
// went above lim_S is dropped and run again on the clamped datapath (rare).
// PAYF: the terminal payoff of the lazy run (terminal payoff classes).
template <int LC, int PAYF, bool DUMP, int EST, int XP, int AP, int PC, class Sim>
__device__ __forceinline__ void group_loop(Sim &sim, ThreadAcc<EST, XP> &acc, const LaunchArgs &args,
                                           const GroupCtx &it, uint64_t gbeg, uint32_t ng, uint32_t rf0, uint32_t rf1,
                                           bool lazy, mlmc_sample_rec *dump) {
  const uint64_t first = it.first, last = it.last;
  // Real-valued estimators flush their float pairs every `flush_groups`
  // groups (at most REAL_FLUSH_SAMPLES samples).
  constexpr bool REAL = EST != EST_APPROX && !(XP == XP_F64 && EST == EST_EXACT);
  constexpr uint32_t FLUSH_GROUPS =
      REAL ? (uint32_t)REAL_FLUSH_SAMPLES / (uint32_t)(Sim::KPV * (LC == 2 ? 1 : (LC == 1 ? 2 : 4))) : 0u;
  uint32_t since_flush = 0;
  for (uint32_t r = threadIdx.x; r < ng; r += blockDim.x) {
    const uint64_t g = gbeg + r;
    const bool full = r >= rf0 && r < rf1;
    if constexpr (Sim::LAZY && !DUMP) {
      bool eager = true;
      if (lazy && full) {
        sim.hi = 0;
        if constexpr (PC == PC_TERMINAL) {
          // the group's sums stay in their own accumulator until the group is kept
          run_group<LC, false, true, PAYF, DUMP>(sim, acc, args, it, g, true, first, last, dump);
          eager = sim.over();
          if (eager) acc.discard_group();
        } else {
          // path-dependent payoffs: one sample per step carries more state, and a
          // FULL instantiation costs registers more than the range test costs
          const auto saved = acc.mark();
          run_group<LC, false, false, -1, DUMP>(sim, acc, args, it, g, true, first, last, dump);
          eager = sim.over();
          if (eager) acc.rewind(saved);
        }
      }
      if (eager) run_group<LC, true, false, -1, DUMP>(sim, acc, args, it, g, full, first, last, dump);
    } else {
      // other datapaths: one instantiation (a FULL one beside it raised the
      // packed binary16 kernels from ~115 to ~165 registers and cost 9%)
      run_group<LC, true, false, -1, DUMP>(sim, acc, args, it, g, full, first, last, dump);
    }
    if constexpr (EST == EST_APPROX && AP == AP_FX32 && PC == PC_TERMINAL) acc.flush_group();
    if constexpr (REAL) {
      if (++since_flush == FLUSH_GROUPS) {
        acc.flush_real();
        since_flush = 0;
      }
    }
  }
}

// Simulate one chunk of an item (its table already in shared memory) and
// write the CTA's Partial for it.  The level class and (on the lazy terminal
// path) the payoff are fixed once per chunk, so the group loop carries no
// branch on them.  DYN (device-scheduled kernel) only keeps the
// instantiations of the static and device-scheduled kernels apart, so that
// each is compiled inline into its own kernel.
template <int EST, int XP, int AP, int SCHEME, int PC, int KP, int MSEL, bool DUMP, bool DYN, bool PRE = false,
          bool MERGED = false>
__device__ __forceinline__ void chunk_body(const LaunchArgs &args, const ItemDesc &it, int item, uint32_t gc,
                                           const unsigned char *smem_tab) {
  using Sim = LevelSim<EST, XP, AP, SCHEME, PC, KP, MSEL, PRE, MERGED>;
  Sim sim;
  sim.load(it, smem_tab);
  ThreadAcc<EST, XP> acc;
  acc.init();

  const uint32_t chunk = gc - it.chunk_begin;
  const uint64_t per_chunk = (uint64_t)it.groups_per_thread * blockDim.x;
  const uint64_t gbeg = it.g0 + (uint64_t)chunk * per_chunk;
  const uint64_t gend = min(it.g1, gbeg + per_chunk);
  const uint32_t ng = gend > gbeg ? (uint32_t)(gend - gbeg) : 0u;
  // the chunk's groups [rf0, rf1) (relative to gbeg) lie entirely in the item's range
  const uint64_t gf0 = max(it.gf0, gbeg), gf1 = min(it.gf1, gend);
  const uint32_t rf0 = gf0 < gf1 ? (uint32_t)(gf0 - gbeg) : 0u;
  const uint32_t rf1 = gf0 < gf1 ? (uint32_t)(gf1 - gbeg) : 0u;
  // per-sample records only in the DUMP instantiation (parity runs)
  mlmc_sample_rec *dump = DUMP ? (mlmc_sample_rec *)it.dump : nullptr;
  const bool lazy = Sim::LAZY && !DUMP && it.ff.lazy;
  const int lc = it.level >= 2 ? 2 : it.level;
  GroupCtx gx;
  gx.ctr2 = it.ctr2; gx.ctr3 = it.ctr3; gx.d = it.d; gx.level = it.level; gx.enumerate = it.enumerate;
  gx.lanes = it.lanes; gx.first = it.first; gx.last = it.first + it.N;
  auto loop = [&](auto lctag, auto paytag) {
    group_loop<decltype(lctag)::value, decltype(paytag)::value, DUMP, EST, XP, AP, PC>(sim, acc, args, gx, gbeg, ng,
                                                                                      rf0, rf1, lazy, dump);
  };
  using L0 = std::integral_constant<int, 0>;
  using L1 = std::integral_constant<int, 1>;
  using L2 = std::integral_constant<int, 2>;
  if constexpr (Sim::LAZY && !DUMP && PC == PC_TERMINAL) {
    const bool dig = it.payoff == 1;
    if (lc == 0) {
      if (it.tab_y0) group_loop_y0(sim, acc, args, gx, gbeg, ng, rf0, rf1);
      else if (dig) loop(L0{}, PayTag<1>{});
      else loop(L0{}, PayTag<0>{});
    }
    else if (lc == 1) { if (dig) loop(L1{}, PayTag<1>{}); else loop(L1{}, PayTag<0>{}); }
    else { if (dig) loop(L2{}, PayTag<1>{}); else loop(L2{}, PayTag<0>{}); }
  } else {
    if (lc == 0) loop(L0{}, PayTag<-1>{});
    else if (lc == 1) loop(L1{}, PayTag<-1>{});
    else loop(L2{}, PayTag<-1>{});
  }
  acc.flush_real();
  block_reduce_write<EST, XP>(acc, args.partials + gc);
  if (args.counters && threadIdx.x < 32) {
    // the CTA that completes the item's last chunk sums all its partials, in
    // chunk order (the partials of other CTAs are read through L2); only its
    // first warp takes part, the other warps are done
    uint32_t last = 0;
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(args.counters + item, 1u) + 1u == it.n_chunks;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      const DevSums r = warp_sum_partials<true>(args.partials + it.chunk_begin, it.n_chunks);
      if (threadIdx.x == 0) {
        args.out[it.out_index] = r;
        args.counters[item] = 0u;   // ready for the next launch
      }
    }
  }
}

// Find the item of chunk gc (the last with chunk_begin <= gc) and stage its
// approximate-Normal table in shared memory (unless *staged, when given, says
// that it is there already).  Every thread has finished the previous chunk
// before the table is overwritten (block_reduce_write ends with a barrier).
template <int AP, int SCHEME, bool PRE = false, bool PHI_BY_KIND = false>
__device__ __forceinline__ int stage_chunk(const ItemDesc *items, int n_items, uint32_t gc, const void **staged) {
  extern __shared__ __align__(16) unsigned char smem_tab[];
  __shared__ int s_item;
  if (threadIdx.x < 32) {
    // last item with chunk_begin <= gc (chunk_begin is non-decreasing and
    // items[0].chunk_begin <= gc): warp 0 samples 32 evenly spaced items per
    // round, one load each, and narrows to the stride after the last sample
    // at or before gc; one round for up to 32 items, two for up to 1024
    const int lane = threadIdx.x;
    int lo = 0, span = n_items;
    while (true) {
      const int stride = span > 32 ? (span + 31) / 32 : 1;
      const int k = lo + lane * stride;
      const bool le = lane * stride < span && items[k].chunk_begin <= gc;
      const int last = __popc(__ballot_sync(0xffffffffu, le)) - 1;
      lo += last * stride;
      if (stride == 1) break;
      span = min(stride, span - last * stride);
    }
    if (lane == 0) s_item = lo;
  }
  __syncthreads();
  const int item = s_item;
  const ItemDesc &it = items[item];
  if constexpr (AP == AP_FX32) {
    // (Z~_j, sum1 of a fine step from Z~_j) for every index j: Method 1 and 2
    // values from the item's table, Method 3 values from its class lines (the
    // arithmetic of LevelSim::fixed_z); sum1 by the datapath's own step code.
    // The table depends on the item's constants as well, so a persistent CTA
    // (staged != nullptr) keeps it while its chunks stay in the same item.
    if (staged && *staged == (const void *)&it) return item;
    if (staged) *staged = (const void *)&it;
    // the item's constants in registers first: the table stores below go
    // through a pointer the compiler cannot tell apart from the item, so
    // fields read inside the loop would be loaded again after every store
    const FastFixed ff = it.ff;
    const int d = it.d, method = it.method, tab_y0 = it.tab_y0, payoff = it.payoff;
    const int fZh = it.fx.fZ2 / 2, fS = it.fx.fS;
    const int32_t S0q = (int32_t)it.fx.S0, Kq = (int32_t)it.fx.K;
    const void *ztab = it.ztab;
    const int n = 1 << d;
    int2 *dst = (int2 *)smem_tab;
    const M3Coef *m3 = (const M3Coef *)ztab;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      int32_t z;
      if (method != 3) {
        z = ((const int32_t *)ztab)[k];
      } else {
        const ApproxIndex ai = approx_index((uint32_t)k << (32 - d), d);
        const int c = m3_class(ai.idx);
        const int64_t t = m3->A[c] + m3->B[c] * (int64_t)ai.idx;
        const int sh = M3_FRAC - fZh;
        const int32_t v = (int32_t)((t + ((int64_t)1 << (sh - 1))) >> sh);
        z = ai.neg ? -v : v;
      }
      const int32_t sum1 = ff_sum1<SCHEME == 1, true>(ff, z, ff.con1r, ff.mfine);
      if (tab_y0) {
        // level 0: the sample is a function of j alone -- S after the one fine
        // step from S0 (mul2 = rd(S0 sum1), S = rd(S0 + mul2), clamped to lim_S
        // as on the clamped datapath) and its terminal payoff
        // (the host sets tab_y0 on lazy items only, whose S_0 <= limT keeps
        // that S within lim_S: the clamp changes nothing there).  The same
        // arithmetic as LevelSim::ff_apply's 32-bit step and fixed_payoff's
        // 32-bit terminal payoff; the level-0 parity tests hold the two equal.
        const int64_t p2 = (int64_t)S0q * sum1 + ff.radd2;
        const int32_t mul2 = (int32_t)__funnelshift_r((uint32_t)p2, (uint32_t)((uint64_t)p2 >> 32), ff.rs2);
        const int32_t s1 = (int32_t)((uint32_t)S0q + (uint32_t)mul2 * (uint32_t)ff.mulS);
        const int32_t lim = (int32_t)ff.limS;
        const int32_t c = min(max(s1, -lim), lim);
        const int32_t y = c > Kq ? (payoff == 1 ? (int32_t)1 << fS : c - Kq) : 0;
        dst[k] = make_int2(y, c != s1 ? 1 : 0);
      } else {
        dst[k] = make_int2(z, PRE ? sum1 * (1 << (32 - ff.rs2)) : sum1);
      }
    }
    if (it.perm) {   // after the table: the method-2 interval ranks
      uint16_t *pd = (uint16_t *)(smem_tab + (size_t)n * TabBytes<AP>::value);
      for (int k = threadIdx.x; k < n; k += blockDim.x) pd[k] = it.perm[k];
    }
    // merged launch: only the correction chunks (kind 2) run the FP32 exact path
    if (PHI_BY_KIND && it.kind == 2) stage_phi_inv();
    __syncthreads();
  } else if constexpr (AP != AP_NONE) {
    if (!staged || it.ztab != *staged) {
      if (staged) *staged = it.ztab;
      if (it.method != 3) {
        const int n = 1 << it.d;
        if constexpr (AP == AP_FIXED || AP == AP_FX64) {
          const int32_t *src = (const int32_t *)it.ztab;
          for (int k = threadIdx.x; k < n; k += blockDim.x) ((int32_t *)smem_tab)[k] = src[k];
        } else {
          const uint16_t *src = (const uint16_t *)it.ztab;
          for (int k = threadIdx.x; k < n; k += blockDim.x) ((uint16_t *)smem_tab)[k] = src[k];
        }
        if (it.perm) {   // after the table: the method-2 interval ranks
          uint16_t *dst = (uint16_t *)(smem_tab + (size_t)n * TabBytes<AP>::value);
          for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = it.perm[k];
        }
      } else {
        const uint32_t *src = (const uint32_t *)it.ztab;
        for (int k = threadIdx.x; k < (int)(sizeof(M3Coef) / 4); k += blockDim.x)
          ((uint32_t *)smem_tab)[k] = src[k];
      }
      __syncthreads();
    }
  }
  return item;
}

// One chunk (gc) of one launch: its item and table (stage_chunk), then the
// chunk's sample groups and the CTA's Partial for the chunk.
template <int EST, int XP, int AP, int SCHEME, int PC, int KP, bool ALLOW_DUMP, bool DYN>
__device__ __forceinline__ void run_chunk(const LaunchArgs &args, const ItemDesc *items, int n_items, uint32_t gc,
                                          const void **staged) {
  extern __shared__ __align__(16) unsigned char smem_tab[];
  const int item = stage_chunk<AP, SCHEME>(items, n_items, gc, staged);
  const ItemDesc &it = items[item];
  if (ALLOW_DUMP && it.dump) {
    if constexpr (ALLOW_DUMP) chunk_body<EST, XP, AP, SCHEME, PC, KP, 2, true, DYN>(args, it, item, gc, smem_tab);
  } else if constexpr (AP == AP_NONE || AP == AP_FX32) {
    // no method choice: exact paths, and the FX32 table that holds every method's values
    chunk_body<EST, XP, AP, SCHEME, PC, KP, 0, false, DYN>(args, it, item, gc, smem_tab);
  } else {
    if (it.method == 3) chunk_body<EST, XP, AP, SCHEME, PC, KP, 1, false, DYN>(args, it, item, gc, smem_tab);
    else chunk_body<EST, XP, AP, SCHEME, PC, KP, 0, false, DYN>(args, it, item, gc, smem_tab);
  }
}

// Static launch: CTA b runs chunk chunk0 + b of the launch.
template <int EST, int XP, int AP, int SCHEME, int PC, int KP>
__global__ void __launch_bounds__(LAUNCH_THREADS, MinCtas<EST, AP, SCHEME, PC>::value)
level_kernel(const __grid_constant__ LaunchArgs args) {
  if constexpr (NeedsPhi<EST, XP>::value) stage_phi_inv();
  run_chunk<EST, XP, AP, SCHEME, PC, KP, false, false>(args, args.items, args.n_items, args.chunk0 + blockIdx.x,
                                                      nullptr);
}

// The same for launches with per-sample records (parity runs): a kernel of
// its own, so that the record-writing code does not weigh on the register
// allocation of the launches without records.
template <int EST, int XP, int AP, int SCHEME, int PC, int KP>
__global__ void __launch_bounds__(LAUNCH_THREADS, MinCtas<EST, AP, SCHEME, PC>::value)
level_kernel_dump(const __grid_constant__ LaunchArgs args) {
  if constexpr (NeedsPhi<EST, XP>::value) stage_phi_inv();
  run_chunk<EST, XP, AP, SCHEME, PC, KP, true, false>(args, args.items, args.n_items, args.chunk0 + blockIdx.x,
                                                     nullptr);
}

// Device-scheduled launch (fixed grid, captured once in a CUDA graph): the item
// and chunk counts come from args.dyn, written on the device before the
// launch; CTA b runs chunks b, b + gridDim.x, ...
template <int EST, int XP, int AP, int SCHEME, int PC, int KP>
__global__ void __launch_bounds__(LAUNCH_THREADS, MinCtas<EST, AP, SCHEME, PC, true>::value)
level_kernel_dyn(const __grid_constant__ LaunchArgs args) {
  const DynLaunch d = *args.dyn;
  const void *staged = nullptr;
  if constexpr (NeedsPhi<EST, XP>::value) stage_phi_inv();
  for (uint32_t rel = blockIdx.x; rel < d.n_chunks; rel += gridDim.x)
    run_chunk<EST, XP, AP, SCHEME, PC, KP, false, true>(args, args.items + d.item_off, (int)d.n_items,
                                                        d.chunk0 + rel, &staged);
}

// A merged launch of the nested estimator's three 32-bit fixed-point kernel
// families for one (scheme, payoff class): approximate with packed draws
// (kind 0), approximate one sample per thread (kind 1) and correction (kind 2).
// Its chunks run the same chunk bodies as the separate launches, in one grid
// ordered by decreasing CTA cost, so the longest chains start first and the
// short chunks of every family fill in behind them.
// PRE: every item's sum1 fits the pre-scaled product (family 24; see LevelSim).
template <int AP, int SCHEME, int PC, bool PRE>
__global__ void __launch_bounds__(LAUNCH_THREADS, 6) nested_kernel(const __grid_constant__ LaunchArgs args) {
  extern __shared__ __align__(16) unsigned char smem_tab[];
  const uint32_t gc = args.chunk0 + blockIdx.x;
  const int item = stage_chunk<AP, SCHEME, PRE, true>(args.items, args.n_items, gc, nullptr);
  const ItemDesc &it = args.items[item];
  if (it.kind == 0)
    chunk_body<EST_APPROX, XP_F32, AP, SCHEME, PC, 3, 0, false, false, PRE, true>(args, it, item, gc, smem_tab);
  else if (it.kind == 1)
    chunk_body<EST_APPROX, XP_F32, AP, SCHEME, PC, 1, 0, false, false, PRE, true>(args, it, item, gc, smem_tab);
  else
    chunk_body<EST_CORR, XP_F32, AP, SCHEME, PC, 1, 0, false, false, PRE, true>(args, it, item, gc, smem_tab);
}

}  // namespace mlmc

namespace mlmc {

template <int EST, int XP, int AP, int SCHEME, int PC, int KP>
cudaError_t launch_one(dim3 grid, dim3 block, size_t smem, cudaStream_t st, const LaunchArgs &a, int *occ) {
  auto k = (a.dyn || occ) ? level_kernel_dyn<EST, XP, AP, SCHEME, PC, KP>
            : a.dump       ? level_kernel_dump<EST, XP, AP, SCHEME, PC, KP>
                           : level_kernel<EST, XP, AP, SCHEME, PC, KP>;
  // above 48 KB of dynamic plus static shared memory (the static part holds
  // up to about 8.6 KB: the inverse-Normal cubics) the kernel must opt in
  if (smem > 32 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, (int)block.x, smem);
  k<<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

// All (scheme, payoff class) instantiations of one (estimator, precision) family.
template <int EST, int XP, int AP, int KP = 1>
cudaError_t launch_family(int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          const LaunchArgs &a, int *occ) {
  switch (scheme * 3 + pc) {
    case 0: return launch_one<EST, XP, AP, 0, PC_TERMINAL, KP>(grid, block, smem, st, a, occ);
    case 1: return launch_one<EST, XP, AP, 0, PC_ASIAN, KP>(grid, block, smem, st, a, occ);
    case 2: return launch_one<EST, XP, AP, 0, PC_LOOKBACK, KP>(grid, block, smem, st, a, occ);
    case 3: return launch_one<EST, XP, AP, 1, PC_TERMINAL, KP>(grid, block, smem, st, a, occ);
    case 4: return launch_one<EST, XP, AP, 1, PC_ASIAN, KP>(grid, block, smem, st, a, occ);
    case 5: return launch_one<EST, XP, AP, 1, PC_LOOKBACK, KP>(grid, block, smem, st, a, occ);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mlmc
