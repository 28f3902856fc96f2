/*
 * Plain, slow FP64 CPU oracle for one level of (nested) MLMC on Geometric
 * Brownian Motion, following Haas & Giles, "A nested MLMC framework for
 * efficient simulations on FPGAs" (arXiv 2502.07123).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference arm of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * Every sample is simulated one at a time with plain loops:
 *   - uniforms: Philox4x32-10 (Salmon et al., SC'11), one call per draw;
 *   - exact Normal Z = Phi^{-1}(U), U = 2^-32 (J + 1/2)        (Sec. 3.1);
 *   - approximate Normal Z~ from a table indexed by the top d bits of J
 *     (Sec. 3.1 Method 1, Sec. 3.3 Method 3; the table values are built by
 *     oracle/tables.py and passed in);
 *   - Euler-Maruyama fine path (eq. GBM_sde) and the coarse path with drift
 *     and volatility frozen at even indices (Sec. 2.1);
 *   - the approximate path in emulated fixed point, decomposed as in
 *     Algorithm 1 (Sec. 4.1), or in IEEE binary16 / bfloat16;
 *   - payoff, level difference, nested correction (eq. chap:nested_exp);
 *   - sums of Y and Y^2 (Neumaier-compensated FP64 for real-valued Y, exact
 *     128-bit integers for integer-valued Y).
 *
 * Must be compiled with -ffp-contract=off so that no a*b+c is fused.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Public enums and records (mirrored, not shared, by the Python wrapper).  */
/* ------------------------------------------------------------------------ */
enum { OR_EURO = 0, OR_DIGITAL = 1, OR_ASIAN = 2, OR_LOOKBACK = 3 };
enum { OR_EULER = 0, OR_MILSTEIN = 1 };
enum {
  OR_FP64_EXACT = 0, OR_FP32_EXACT = 1, OR_FP16_APPROX = 2, OR_BF16_APPROX = 3,
  OR_FIXED_APPROX = 4, OR_CORR_FIXED = 5, OR_CORR_FP16 = 6, OR_CORR_BF16 = 7,
  /* half-precision increments with S in FP32 */
  OR_FP16S_APPROX = 8, OR_BF16S_APPROX = 9, OR_CORR_FP16S = 10, OR_CORR_BF16S = 11
};
/* fixed-point variable order (Algorithm 1): Z~, con1, con2, mul1, sum1, mul2, S */
enum { V_Z = 0, V_CON1 = 1, V_CON2 = 2, V_MUL1 = 3, V_SUM1 = 4, V_MUL2 = 5, V_S = 6 };

typedef struct {
  double S0, K, r, sigma, T;
  int32_t payoff, scheme;
} or_params;

typedef struct { int32_t e[7]; int32_t f[7]; } or_format;

typedef struct {
  double pf, pc;   /* exact-path payoffs, undiscounted (pc = 0 on level 0)     */
  double sf, sc;   /* exact-path terminal values                               */
  double af, ac;   /* approximate-path terminal values as real numbers         */
  int64_t qf, qc;  /* approximate-path payoffs as integers in units 2^-unit    */
  double y;        /* the sample value that enters the sums                    */
  uint32_t sat;    /* 1 if any fixed-point variable saturated on this sample   */
  uint32_t pad;
} or_sample;

typedef struct {
  double sum, sum2;            /* undiscounted sums of Y and Y^2 (real-valued) */
  int64_t isum;                /* exact sum of integer Y (units 2^-unit)       */
  uint64_t isum2_lo, isum2_hi; /* exact sum of integer Y^2 (units 2^-2unit)    */
  uint64_t n, saturations;
  int32_t unit, exact_int;
} or_sums;

/* error codes */
enum { OR_OK = 0, OR_EINVAL = 1, OR_EOVERFLOW = 5 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications    */
/* with the published multipliers and Weyl key increments.                  */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The uniform integer J driving fine step i of sample s on a level.
 * Counter layout (a reading: the paper only says "a D-bit integer J"):
 *   word index w = s * 2^level + i, call q = w / 4, output word w mod 4,
 *   counter = (q_lo, q_hi, level | stream << 8, request), key = (seed_lo, seed_hi). */
uint32_t or_draw(uint64_t seed, uint32_t request, uint32_t level, uint32_t stream,
                 uint64_t sample, uint32_t step) {
  uint64_t w = (sample << level) + (uint64_t)step;
  uint64_t q = w >> 2;
  uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), level | (stream << 8), request};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  or_philox4x32_10(ctr, key, out);
  return out[w & 3u];
}

/* Packed draws of approximate-only estimators (a reading, see below): with
 * k = floor(32 / d) >= 2 fields per 32-bit word, sample s belongs to pack
 * P = s div k and lane L = s mod k; its fine step i reads word
 * w = P 2^level + i (call w div 4, output word w mod 4, same counter layout as
 * or_draw) and uses field L, i.e. bits [32 - d (L+1), 32 - d L).  The result is
 * returned shifted to the top of a 32-bit value, so that the usual "top d bits"
 * rule of the approximate Normal applies unchanged. */
uint32_t or_draw_packed(uint64_t seed, uint32_t request, uint32_t level, uint32_t stream,
                        uint64_t sample, uint32_t step, int d) {
  const uint64_t k = (uint64_t)(32 / d);
  const uint64_t pack = sample / k, lane = sample % k;
  uint64_t w = (pack << level) + (uint64_t)step;
  uint64_t q = w >> 2;
  uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), level | (stream << 8), request};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  or_philox4x32_10(ctr, key, out);
  uint32_t J = out[w & 3u];
  return J << (uint32_t)(d * (int)lane);
}

/* ------------------------------------------------------------------------ */
/* Exact inverse Normal CDF in FP64 (Sec. 3: "computing Z is trivial").     */
/* Newton's method on Phi(z) = u, started from the Abramowitz & Stegun      */
/* 26.2.23 rational approximation.  The residual is formed without          */
/* cancellation: near the centre from erf and the exact difference u - 1/2, */
/* in the lower tail from erfc.  Valid for 0 < u <= 1/2.                    */
/* ------------------------------------------------------------------------ */
static double std_normal_pdf(double z) {
  return exp(-0.5 * z * z) / 2.5066282746310002; /* sqrt(2 pi) */
}

static double phi_residual(double z, double u) {
  if (u > 0.25) {
    /* Phi(z) - u = erf(z/sqrt2)/2 - (u - 1/2); u - 1/2 is exact here */
    return 0.5 * erf(z / M_SQRT2) - (u - 0.5);
  }
  return 0.5 * erfc(-z / M_SQRT2) - u;
}

double or_norminv_lower(double u) {
  double t = sqrt(-2.0 * log(u));
  double z = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                       (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
  for (int it = 0; it < 60; ++it) {
    double dz = phi_residual(z, u) / std_normal_pdf(z);
    z -= dz;
    if (fabs(dz) <= 1e-17 * fabs(z)) break;
  }
  return z;
}

/* Z = Phi^{-1}(2^-32 (J + 1/2)), using Phi^{-1}(1-u) = -Phi^{-1}(u) for the
 * upper half so that no 1 - u is ever formed. */
double or_exact_normal(uint32_t J) {
  if (J < 0x80000000u) return or_norminv_lower(ldexp((double)J + 0.5, -32));
  return -or_norminv_lower(ldexp((double)(~J) + 0.5, -32));
}

/* Table index and sign of the approximate Normal (Sec. 3.1): j = top d bits
 * of J.  Reading of "the leading bit of j gives the sign": Z~ is the mean of
 * Phi^{-1} over the 2^-d interval that contains U, so for the upper half the
 * index is mirrored (j -> 2^d - 1 - j) and the sign flipped. */
static void approx_index(uint32_t J, int d, uint32_t *idx, int *negate) {
  uint32_t j = J >> (32 - d);
  uint32_t half = 1u << (d - 1);
  if (j < half) { *idx = j; *negate = 0; }
  else { *idx = (1u << d) - 1u - j; *negate = 1; }
}

/* ------------------------------------------------------------------------ */
/* Rounding to IEEE binary16 / bfloat16 (round to nearest, ties to even),   */
/* applied to an exactly computed double.                                   */
/* ------------------------------------------------------------------------ */
static double round_to_format(double x, int p, int emin, int emax) {
  if (x == 0.0 || isnan(x) || isinf(x)) return x;
  int ex;
  frexp(fabs(x), &ex);            /* |x| = m 2^ex, m in [0.5, 1) */
  int e = ex - 1;                 /* |x| in [2^e, 2^(e+1)) */
  if (e < emin) e = emin;         /* subnormal quantum */
  double quantum_exp = (double)(e - p + 1);
  double scaled = ldexp(x, -(int)quantum_exp);
  double rounded = nearbyint(scaled); /* default mode: ties to even */
  double y = ldexp(rounded, (int)quantum_exp);
  double maxfinite = ldexp(2.0 - ldexp(1.0, 1 - p), emax);
  if (fabs(y) > maxfinite) return copysign(INFINITY, x);
  return y;
}
double or_round_fp16(double x) { return round_to_format(x, 11, -14, 15); }
double or_round_bf16(double x) { return round_to_format(x, 8, -126, 127); }

/* Two-sum exactness check: a + b is exact in double. */
static int sum_is_exact(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double err = (a - (s - bb)) + (b - bb);
  return err == 0.0;
}

/* ------------------------------------------------------------------------ */
/* Fixed point (Sec. 4.1): x~ = n 2^-f with |n| <= 2^(e+f) - 1.             */
/* Round to nearest, ties toward +infinity (a reading: the paper fixes      */
/* round-to-nearest only); saturation on overflow (a reading: the paper is  */
/* silent).  Products and sums are formed exactly in 128 bits and rounded   */
/* once to the result's format.                                             */
/* ------------------------------------------------------------------------ */
typedef __int128 i128;

/* exact value v = n 2^-from, re-expressed as round(v 2^to) */
static i128 requantize(i128 n, int from, int to) {
  if (to >= from) return n * ((i128)1 << (to - from));  /* exact */
  int k = from - to;
  i128 half = (i128)1 << (k - 1);
  i128 t = n + half;
  /* floor((v + 2^(k-1)) / 2^k): gcc's >> on a signed value is an arithmetic
   * shift, i.e. division rounding toward -infinity */
  return t >> k;
}

static int64_t saturate(i128 n, int e, int f, uint32_t *sat) {
  i128 lim = ((i128)1 << (e + f)) - 1;
  if (n > lim) { *sat = 1; return (int64_t)lim; }
  if (n < -lim) { *sat = 1; return (int64_t)(-lim); }
  return (int64_t)n;
}

/* rd of a real constant to f fractional bits: floor(x 2^f + 1/2) */
static int const_to_fixed(double x, int e, int f, int64_t *out) {
  double s = ldexp(x, f);
  if (!(fabs(s) < 4503599627370496.0)) return OR_EOVERFLOW;
  double n = floor(s + 0.5);
  double lim = ldexp(1.0, e + f) - 1.0;
  if (fabs(n) > lim) return OR_EOVERFLOW;
  *out = (int64_t)n;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Payoffs (undiscounted); exact path in FP64.                              */
/* ------------------------------------------------------------------------ */
typedef struct {
  double first, last, sum_inner, minv; /* path functionals on its own grid */
  int64_t steps;
} path_acc;

static void acc_start(path_acc *a, double s0) {
  a->first = s0; a->last = s0; a->sum_inner = 0.0; a->minv = s0; a->steps = 0;
}
static void acc_push(path_acc *a, double s) {
  /* s is the value after a new step; the previous "last" becomes inner */
  if (a->steps > 0) a->sum_inner += a->last;
  a->last = s;
  if (s < a->minv) a->minv = s;
  a->steps += 1;
}
static double payoff_fp64(const or_params *p, const path_acc *a) {
  double x = a->last;
  switch (p->payoff) {
    case OR_EURO: return x > p->K ? x - p->K : 0.0;
    case OR_DIGITAL: return x > p->K ? 1.0 : 0.0;
    case OR_ASIAN: {
      /* trapezoidal time average on the path's own grid */
      double avg = (0.5 * a->first + a->sum_inner + 0.5 * a->last) / (double)a->steps;
      return avg > p->K ? avg - p->K : 0.0;
    }
    default: return x - a->minv; /* floating-strike lookback call */
  }
}

/* ------------------------------------------------------------------------ */
/* Level configuration shared by all samples of one call.                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  const or_params *p;
  int level, n, variant, d, pack, enumerate;
  uint64_t seed; uint32_t request, stream;
  double h;
  /* approximate-path tables and constants */
  const double *ztab;        /* Z~ value for each table index (already in the target representation) */
  int64_t *zq;               /* fixed-point table (Z format) */
  or_format fmt;
  int64_t con1, con1c, con2, con3, S0q, Kq;
  /* half constants */
  double hc1, hc1c, hc2, hc3, hS0;
  float K32;
  int unit;
  const uint32_t *perm;      /* Method 2: interval rank pi(j) of every d-bit j, or 0 */
} level_cfg;

/* J of the exact path at fine step i of sample s.  With Method 2 (Sec. 3.2) the
 * correction estimator's exact path takes the uniform in the interval pi(j) the
 * approximate value is ranked at, keeping J's low 32 - d bits:
 * U = 2^-d pi(j) + 2^-32 ((J mod 2^(32-d)) + 1/2). */
static uint32_t exact_J(const level_cfg *c, uint64_t s, int i) {
  uint32_t J = or_draw(c->seed, c->request, (uint32_t)c->level, c->stream, s, (uint32_t)i);
  if (c->perm) {
    const int sh = 32 - c->d;
    const uint32_t low = sh >= 32 ? J : (J & ((1u << sh) - 1u));
    J = (c->perm[J >> sh] << sh) | low;
  }
  return J;
}

static int is_corr(int v) {
  return v == OR_CORR_FIXED || v == OR_CORR_FP16 || v == OR_CORR_BF16 || v == OR_CORR_FP16S || v == OR_CORR_BF16S;
}
static int has_exact(int v) { return v == OR_FP64_EXACT || v == OR_FP32_EXACT || is_corr(v); }
static int has_approx(int v) { return v != OR_FP64_EXACT && v != OR_FP32_EXACT; }
static int approx_kind(int v) { /* 0 fixed, 1 fp16, 2 bf16 */
  if (v == OR_FIXED_APPROX || v == OR_CORR_FIXED) return 0;
  if (v == OR_FP16_APPROX || v == OR_CORR_FP16 || v == OR_FP16S_APPROX || v == OR_CORR_FP16S) return 1;
  return 2;
}
/* half-precision increments with S (and its path functionals) in FP32 */
static int s32_path(int v) { return v >= OR_FP16S_APPROX; }

/* ---- exact path (FP64), literal paper form of the coarse path ---------- */
static void exact_sample(const level_cfg *c, uint64_t s, or_sample *out) {
  const or_params *p = c->p;
  double h = c->h, sqh = sqrt(h);
  double S = p->S0;
  path_acc af, ac;
  acc_start(&af, p->S0);
  acc_start(&ac, p->S0);
  double Sc = p->S0, Sc_frozen = p->S0;
  double Zprev = 0.0;
  for (int i = 0; i < c->n; ++i) {
    double Z = or_exact_normal(exact_J(c, s, i));
    /* fine: S_{i+1} = S_i + a(S_i) h + b(S_i) sqrt(h) Z_i, a = r S, b = sigma S */
    double Snew = S + p->r * S * h + p->sigma * S * sqh * Z;
    if (p->scheme == OR_MILSTEIN)  /* + 1/2 b b' h (Z^2 - 1), b b' = sigma^2 S */
      Snew += 0.5 * p->sigma * p->sigma * S * h * (Z * Z - 1.0);
    S = Snew;
    acc_push(&af, S);
    if (c->level > 0) {
      if (p->scheme == OR_EULER) {
        /* coarse: drift and volatility frozen at S^c_{2 floor(i/2)} (Sec. 2.1) */
        if ((i & 1) == 0) Sc_frozen = Sc;
        Sc = Sc + p->r * Sc_frozen * h + p->sigma * Sc_frozen * sqh * Z;
        if (i & 1) acc_push(&ac, Sc);  /* only even indices lie on the coarse grid */
      } else if (i & 1) {
        /* Milstein coarse step (2h, increment dW = sqrt(h)(Z_{2k} + Z_{2k+1})) */
        double dW = sqh * (Zprev + Z);
        Sc = Sc + p->r * Sc * 2.0 * h + p->sigma * Sc * dW +
             0.5 * p->sigma * p->sigma * Sc * (dW * dW - 2.0 * h);
        acc_push(&ac, Sc);
      }
    }
    Zprev = Z;
  }
  out->sf = S;
  out->pf = payoff_fp64(p, &af);
  if (c->level > 0) { out->sc = Sc; out->pc = payoff_fp64(p, &ac); }
  else { out->sc = 0.0; out->pc = 0.0; }
}

/* ---- approximate path in fixed point (Algorithm 1) --------------------- */
typedef struct { int64_t first, last, inner, minv; int64_t steps; } fx_acc;
static void fx_start(fx_acc *a, int64_t s0) { a->first = s0; a->last = s0; a->inner = 0; a->minv = s0; a->steps = 0; }
static void fx_push(fx_acc *a, int64_t s) {
  if (a->steps > 0) a->inner += a->last;
  a->last = s;
  if (s < a->minv) a->minv = s;
  a->steps += 1;
}

/* One Algorithm-1 step: mul1 = con2 z; sum1 = con1 + mul1 [+ mul3]; mul2 = S sum1; S = S + mul2.
 * z is in Z's format (the coarse z is the exact sum of two fine z's); zz_minus is
 * the Milstein term multiplier (1 on the fine path, 2 on the coarse path). */
static int64_t fx_step(const level_cfg *c, int64_t S, int64_t z, int64_t con1, int milstein_m, uint32_t *sat) {
  const or_format *F = &c->fmt;
  int fZ = F->f[V_Z];
  /* mul1 = rd(con2 * z) */
  i128 prod1 = (i128)c->con2 * (i128)z;  /* units 2^-(f_con2 + f_Z) */
  int64_t mul1 = saturate(requantize(prod1, F->f[V_CON2] + fZ, F->f[V_MUL1]), F->e[V_MUL1], F->f[V_MUL1], sat);
  /* sum1 = rd(con1 + mul1 [+ mul3]), all terms aligned exactly first */
  int fmax = F->f[V_CON1] > F->f[V_MUL1] ? F->f[V_CON1] : F->f[V_MUL1];
  i128 acc = requantize(con1, F->f[V_CON1], fmax) + requantize(mul1, F->f[V_MUL1], fmax);
  if (milstein_m) {
    /* Milstein extension (not in Algorithm 1): mul3 = rd(con3 (z^2 - m)), in mul1's format,
     * con3 = sigma^2 h / 2 in con1's format */
    i128 zz = (i128)z * (i128)z - ((i128)milstein_m << (2 * fZ)); /* units 2^-2fZ, exact */
    i128 prod3 = (i128)c->con3 * zz;                             /* units 2^-(f_con1 + 2 fZ) */
    int64_t mul3 = saturate(requantize(prod3, F->f[V_CON1] + 2 * fZ, F->f[V_MUL1]), F->e[V_MUL1], F->f[V_MUL1], sat);
    acc += requantize(mul3, F->f[V_MUL1], fmax);
  }
  int64_t sum1 = saturate(requantize(acc, fmax, F->f[V_SUM1]), F->e[V_SUM1], F->f[V_SUM1], sat);
  /* mul2 = rd(S * sum1) */
  i128 prod2 = (i128)S * (i128)sum1;
  int64_t mul2 = saturate(requantize(prod2, F->f[V_S] + F->f[V_SUM1], F->f[V_MUL2]), F->e[V_MUL2], F->f[V_MUL2], sat);
  /* S = rd(S + mul2) */
  int fmax2 = F->f[V_S] > F->f[V_MUL2] ? F->f[V_S] : F->f[V_MUL2];
  i128 s2 = requantize(S, F->f[V_S], fmax2) + requantize(mul2, F->f[V_MUL2], fmax2);
  return saturate(requantize(s2, fmax2, F->f[V_S]), F->e[V_S], F->f[V_S], sat);
}

static int64_t fx_payoff(const level_cfg *c, const fx_acc *a, int coarse) {
  int64_t x = a->last, K = c->Kq;
  int fS = c->fmt.f[V_S];
  switch (c->p->payoff) {
    case OR_EURO: return x > K ? x - K : 0;
    case OR_DIGITAL: return x > K ? ((int64_t)1 << fS) : 0;
    case OR_ASIAN: {
      /* 2 n A = S_0 + 2 sum_inner + S_n (units 2^-fS); payoff = (2nA - 2nK)/(2n) */
      int64_t twice_sum = a->first + 2 * a->inner + a->last;
      int64_t twoN_K = 2 * a->steps * K;
      int64_t v = twice_sum > twoN_K ? twice_sum - twoN_K : 0;
      /* fine: units 2^-(fS + level + 1); coarse has half the steps: scale by 2 */
      return coarse ? 2 * v : v;
    }
    default: return x - a->minv;
  }
}

static uint32_t approx_draw(const level_cfg *c, uint64_t s, int i) {
  /* enumeration of the table cells (levels 0-1): j_i = (s >> (d i)) mod 2^d, in the top d bits */
  if (c->enumerate) return (uint32_t)((s >> (c->d * i)) & ((1ULL << c->d) - 1ULL)) << (32 - c->d);
  if (c->pack) return or_draw_packed(c->seed, c->request, c->level, c->stream, s, i, c->d);
  return or_draw(c->seed, c->request, c->level, c->stream, s, i);
}

static void fixed_sample(const level_cfg *c, uint64_t s, or_sample *out) {
  int milstein = c->p->scheme == OR_MILSTEIN;
  uint32_t sat = 0;
  int64_t S = c->S0q, Sc = c->S0q, zprev = 0;
  fx_acc af, ac;
  fx_start(&af, c->S0q);
  fx_start(&ac, c->S0q);
  for (int i = 0; i < c->n; ++i) {
    uint32_t J = approx_draw(c, s, i);
    uint32_t idx; int neg;
    approx_index(J, c->d, &idx, &neg);
    int64_t z = neg ? -c->zq[idx] : c->zq[idx];
    S = fx_step(c, S, z, c->con1, milstein ? 1 : 0, &sat);
    fx_push(&af, S);
    if (c->level > 0 && (i & 1)) {
      int64_t zc = zprev + z;  /* exact: one more integer bit than Z */
      Sc = fx_step(c, Sc, zc, c->con1c, milstein ? 2 : 0, &sat);
      fx_push(&ac, Sc);
    }
    zprev = z;
  }
  int fS = c->fmt.f[V_S];
  out->af = ldexp((double)S, -fS);
  out->qf = fx_payoff(c, &af, 0);
  if (c->level > 0) { out->ac = ldexp((double)Sc, -fS); out->qc = fx_payoff(c, &ac, 1); }
  else { out->ac = 0.0; out->qc = 0; }
  out->sat = sat;
}

/* ---- approximate path in binary16 / bfloat16 ---------------------------- */
static double rh(const level_cfg *c, double x) {
  return approx_kind(c->variant) == 1 ? or_round_fp16(x) : or_round_bf16(x);
}
static double rh_sum(const level_cfg *c, double a, double b, int *bad) {
  if (!sum_is_exact(a, b)) *bad = 1;
  return rh(c, a + b);
}

static double half_step(const level_cfg *c, double S, double z, double c1, int milstein_m, int *bad) {
  double mul1 = rh(c, c->hc2 * z);           /* products of two half values are exact in double */
  double sum1 = rh_sum(c, c1, mul1, bad);
  if (milstein_m) {
    double sq = rh(c, z * z);
    double sqm = rh_sum(c, sq, -(double)milstein_m, bad);
    double mul3 = rh(c, c->hc3 * sqm);
    sum1 = rh_sum(c, sum1, mul3, bad);
  }
  double mul2 = rh(c, S * sum1);
  return rh_sum(c, S, mul2, bad);
}

/* The same increment sum1 in half precision; S in FP32: mul2 = fl32(S sum1),
 * S = fl32(S + mul2), one rounding each (sum1 is exact in FP32). */
static float half_step_s32(const level_cfg *c, float S, double z, double c1, int milstein_m, int *bad) {
  double mul1 = rh(c, c->hc2 * z);
  double sum1 = rh_sum(c, c1, mul1, bad);
  if (milstein_m) {
    double sq = rh(c, z * z);
    double sqm = rh_sum(c, sq, -(double)milstein_m, bad);
    double mul3 = rh(c, c->hc3 * sqm);
    sum1 = rh_sum(c, sum1, mul3, bad);
  }
  const float s1 = (float)sum1;
  const float mul2 = S * s1;
  return S + mul2;
}

/* FP32 payoff of a half path (each float operation rounds once) */
typedef struct { float first, acc, last, minv; int64_t steps; } h_acc;
static void h_start(h_acc *a, float s0) { a->first = s0; a->acc = 0.5f * s0; a->last = s0; a->minv = s0; a->steps = 0; }
static void h_push(h_acc *a, float s) {
  if (a->steps > 0) a->acc = a->acc + a->last;  /* inner points enter with weight 1 */
  a->last = s;
  if (s < a->minv) a->minv = s;
  a->steps += 1;
}
static int64_t h_payoff(const level_cfg *c, const h_acc *a) {
  float x = a->last, K = c->K32, P;
  switch (c->p->payoff) {
    case OR_EURO: { float d = x - K; P = d > 0.0f ? d : 0.0f; break; }
    case OR_DIGITAL: P = x > K ? 1.0f : 0.0f; break;
    case OR_ASIAN: {
      float tot = a->acc + 0.5f * a->last;
      float avg = tot * (1.0f / (float)a->steps);  /* steps is a power of two: exact scaling */
      float d = avg - K;
      P = d > 0.0f ? d : 0.0f;
      break;
    }
    default: P = x - a->minv; break;
  }
  /* integer payoff in units 2^-24, rounded to nearest even */
  return (int64_t)nearbyint((double)(P * 16777216.0f));
}

static int half_sample(const level_cfg *c, uint64_t s, or_sample *out) {
  int milstein = c->p->scheme == OR_MILSTEIN;
  int s32 = s32_path(c->variant);
  int bad = 0;
  double S = c->hS0, Sc = c->hS0, zprev = 0.0;
  float Sf = (float)c->p->S0, Scf = Sf;   /* FP32 S of the s32 variants */
  h_acc af, ac;
  h_start(&af, s32 ? Sf : (float)c->hS0);
  h_start(&ac, s32 ? Sf : (float)c->hS0);
  for (int i = 0; i < c->n; ++i) {
    uint32_t J = approx_draw(c, s, i);
    uint32_t idx; int neg;
    approx_index(J, c->d, &idx, &neg);
    double z = neg ? -c->ztab[idx] : c->ztab[idx];
    if (s32) {
      Sf = half_step_s32(c, Sf, z, c->hc1, milstein ? 1 : 0, &bad);
      S = Sf;
    } else {
      S = half_step(c, S, z, c->hc1, milstein ? 1 : 0, &bad);
    }
    h_push(&af, (float)S);
    if (c->level > 0 && (i & 1)) {
      double zc = rh_sum(c, zprev, z, &bad);
      if (s32) {
        Scf = half_step_s32(c, Scf, zc, c->hc1c, milstein ? 2 : 0, &bad);
        Sc = Scf;
      } else {
        Sc = half_step(c, Sc, zc, c->hc1c, milstein ? 2 : 0, &bad);
      }
      h_push(&ac, (float)Sc);
    }
    zprev = z;
  }
  out->af = S;
  out->qf = h_payoff(c, &af);
  if (c->level > 0) { out->ac = Sc; out->qc = h_payoff(c, &ac); }
  else { out->ac = 0.0; out->qc = 0; }
  out->sat = 0;
  return bad;
}

/* ------------------------------------------------------------------------ */
/* Level driver: sums over samples [first, first + N).                      */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } neumaier;
static void nm_add(neumaier *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}

static int validate_format(const or_format *F, int milstein) {
  for (int v = 0; v < 7; ++v) {
    if (F->f[v] < 0 || F->f[v] > 40) return OR_EINVAL;
    if (F->e[v] + F->f[v] < 1 || F->e[v] + F->f[v] > 62) return OR_EINVAL;
  }
  (void)milstein;
  return OR_OK;
}

int or_level(const or_params *p, int level, uint64_t first, uint64_t N, int variant,
             uint64_t seed, uint32_t request, uint32_t stream,
             int d, const double *ztab, const or_format *fmt, int pack, int enumerate,
             or_sums *sums, or_sample *dump, const uint32_t *perm) {
  if (level < 0 || level > 20 || variant < 0 || variant > 11) return OR_EINVAL;
  if (enumerate && (has_exact(variant) || level > 1 || (d << level) > 24)) return OR_EINVAL;
  /* packed draws only feed approximate-only estimators (their uniforms need d bits, not 32) */
  if (pack && (has_exact(variant) || d < 2 || 32 / d < 2)) return OR_EINVAL;
  if (p->payoff < 0 || p->payoff > 3 || p->scheme < 0 || p->scheme > 1) return OR_EINVAL;
  level_cfg c;
  memset(&c, 0, sizeof c);
  c.p = p; c.level = level; c.n = 1 << level; c.variant = variant; c.d = d; c.pack = pack;
  c.enumerate = enumerate;
  c.seed = seed; c.request = request; c.stream = stream;
  c.perm = is_corr(variant) ? perm : 0;   /* the correction's exact path */
  c.h = ldexp(p->T, -level);
  c.ztab = ztab;
  int approx = has_approx(variant), exact = has_exact(variant);
  int kind = approx ? approx_kind(variant) : -1;
  int64_t zq_store[1 << 15];
  if (approx) {
    if (d < 2 || d > 16 || ztab == 0) return OR_EINVAL;
  }
  if (kind == 0) {
    if (!fmt || validate_format(fmt, p->scheme == OR_MILSTEIN)) return OR_EINVAL;
    c.fmt = *fmt;
    int fZ = fmt->f[V_Z];
    for (int k = 0; k < (1 << (d - 1)); ++k) {
      double sc = ldexp(ztab[k], fZ);
      if (sc != floor(sc)) return OR_EINVAL;  /* table must already be on Z's grid */
      zq_store[k] = (int64_t)sc;
      if (fabs(sc) > ldexp(1.0, fmt->e[V_Z] + fZ) - 1.0) return OR_EOVERFLOW;
    }
    c.zq = zq_store;
    double rh_ = p->r * c.h;
    double sqh = sqrt(c.h);
    double c2 = p->sigma * sqh;
    double c3 = 0.5 * p->sigma * p->sigma * c.h;
    int st = 0;
    st |= const_to_fixed(rh_, fmt->e[V_CON1], fmt->f[V_CON1], &c.con1);
    st |= const_to_fixed(p->r * (2.0 * c.h), fmt->e[V_CON1] + 1, fmt->f[V_CON1], &c.con1c);
    st |= const_to_fixed(c2, fmt->e[V_CON2], fmt->f[V_CON2], &c.con2);
    st |= const_to_fixed(c3, fmt->e[V_CON1], fmt->f[V_CON1], &c.con3);
    st |= const_to_fixed(p->S0, fmt->e[V_S], fmt->f[V_S], &c.S0q);
    st |= const_to_fixed(p->K, fmt->e[V_S], fmt->f[V_S], &c.Kq);
    if (st) return OR_EOVERFLOW;
    c.unit = fmt->f[V_S] + (p->payoff == OR_ASIAN ? level + 1 : 0);
  } else if (kind > 0) {
    c.hc1 = rh(&c, p->r * c.h);
    c.hc1c = rh(&c, p->r * (2.0 * c.h));
    c.hc2 = rh(&c, p->sigma * sqrt(c.h));
    c.hc3 = rh(&c, 0.5 * p->sigma * p->sigma * c.h);
    c.hS0 = rh(&c, p->S0);
    c.K32 = (float)p->K;
    c.unit = 24;
  }

  neumaier s1 = {0, 0}, s2 = {0, 0};
  i128 is1 = 0;
  unsigned __int128 is2 = 0;
  uint64_t nsat = 0;
  int bad = 0;
  for (uint64_t t = 0; t < N; ++t) {
    uint64_t s = first + t;
    or_sample rec;
    memset(&rec, 0, sizeof rec);
    if (exact) exact_sample(&c, s, &rec);
    if (approx) {
      if (kind == 0) fixed_sample(&c, s, &rec);
      else bad |= half_sample(&c, s, &rec);
    }
    if (!approx) {
      rec.y = rec.pf - rec.pc;
      nm_add(&s1, rec.y);
      nm_add(&s2, rec.y * rec.y);
    } else if (!exact) {
      int64_t yi = rec.qf - rec.qc;
      rec.y = ldexp((double)yi, -c.unit);
      is1 += yi;
      is2 += (unsigned __int128)((i128)yi * (i128)yi);
    } else {
      int64_t yi = rec.qf - rec.qc;
      rec.y = (rec.pf - rec.pc) - ldexp((double)yi, -c.unit);
      nm_add(&s1, rec.y);
      nm_add(&s2, rec.y * rec.y);
    }
    nsat += rec.sat;
    if (dump) dump[t] = rec;
  }
  memset(sums, 0, sizeof *sums);
  sums->n = N;
  sums->saturations = nsat;
  sums->unit = c.unit;
  if (approx && !exact) {
    sums->exact_int = 1;
    sums->isum = (int64_t)is1;
    sums->isum2_lo = (uint64_t)is2;
    sums->isum2_hi = (uint64_t)(is2 >> 64);
    sums->sum = ldexp((double)is1, -c.unit);
    sums->sum2 = ldexp((double)is2, -2 * c.unit);
  } else {
    sums->sum = s1.s + s1.c;
    sums->sum2 = s2.s + s2.c;
  }
  return bad ? OR_EINVAL : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Array helpers for the Python test layer.                                 */
/* ------------------------------------------------------------------------ */
void or_exact_normal_array(const uint32_t *J, uint64_t n, double *z) {
  for (uint64_t i = 0; i < n; ++i) z[i] = or_exact_normal(J[i]);
}
void or_round_fp16_array(const double *x, uint64_t n, double *y) {
  for (uint64_t i = 0; i < n; ++i) y[i] = or_round_fp16(x[i]);
}
void or_round_bf16_array(const double *x, uint64_t n, double *y) {
  for (uint64_t i = 0; i < n; ++i) y[i] = or_round_bf16(x[i]);
}
void or_draw_array(uint64_t seed, uint32_t request, uint32_t level, uint32_t stream,
                   const uint64_t *sample, const uint32_t *step, uint64_t n, uint32_t *J) {
  for (uint64_t i = 0; i < n; ++i) J[i] = or_draw(seed, request, level, stream, sample[i], step[i]);
}
void or_philox_array(const uint32_t *ctr4, const uint32_t key[2], uint64_t n, uint32_t *out4) {
  for (uint64_t i = 0; i < n; ++i) or_philox4x32_10(ctr4 + 4 * i, key, out4 + 4 * i);
}
/* Approximate Normal of each J from a per-index value table (Sec. 3.1 index/sign rule). */
void or_approx_normal_array(const uint32_t *J, uint64_t n, int d, const double *ztab, double *out) {
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t idx; int neg;
    approx_index(J[i], d, &idx, &neg);
    out[i] = neg ? -ztab[idx] : ztab[idx];
  }
}
void or_draw_packed_array(uint64_t seed, uint32_t request, uint32_t level, uint32_t stream,
                          const uint64_t *sample, const uint32_t *step, uint64_t n, int d, uint32_t *J) {
  for (uint64_t i = 0; i < n; ++i) J[i] = or_draw_packed(seed, request, level, stream, sample[i], step[i], d);
}

/* ------------------------------------------------------------------------ */
/* Error-model statistics of one level (Sec. 4.2-4.3).                      */
/*                                                                          */
/* For the level difference DeltaP = P_f - P_c of the European call        */
/* (discounted, Euler-Maruyama, exact FP64 Normals from stream 0 as the     */
/* correction estimator draws them), every intermediate variable of          */
/* Algorithm 1 -- con1 (and the coarse con1 for 2h), con2, Z_k, mul1_k,      */
/* sum1_k, mul2_k, S_k on the fine and the coarse path, and S0 -- is an      */
/* instance whose rounding error enters DeltaP.  Its sensitivity            */
/* xbar = d DeltaP / d x comes from reverse-mode algorithmic                */
/* differentiation: a forward sweep that records the tape, then a backward  */
/* sweep through the four operations of each step in reverse order.  The    */
/* coarse step uses con1c = r 2h, con2 and Zc_k = Z_2k + Z_2k+1, so Z_j and  */
/* con2 are shared by both paths and S0 starts both.                        */
/*                                                                          */
/* Per sample the sums over instances of xbar^2 of each variable type feed  */
/* V_indep (eq. optimistic); per-instance sums feed V_corr (eq.             */
/* pessimistic); the maxima of |x| give the exponents (Sec. 4.1).           */
/* Instance index within a type (n = 2^l fine steps, m = n/2 coarse):      */
/*   mul1, sum1, mul2: fine k -> k, coarse k -> n + k;                      */
/*   S: S_{k+1} fine -> k, coarse S^c_{k+1} -> n + k, S0 -> n + m;          */
/*   Z: Z_j -> j;  con1: fine 0, coarse 1;  con2: 0.                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  double A[7];        /* sums over samples of sum_instances xbar^2 per type  */
  double maxabs[7];   /* max |x| per type                                    */
  double sum_dp, sum_dp2;
  uint64_t n;
} or_sens;

/* One sample: forward sweep (tape), payoffs, backward sweep.  perturb_type /
 * perturb_inst / delta add delta to one instance right after it is computed
 * (finite-difference checks); xbar_out (7 x n_inst, may be 0) receives the
 * sensitivities of every instance.  Returns DeltaP. */
static double sens_sample(const or_params *p, int level, uint64_t seed, uint32_t request, uint64_t s,
                          int perturb_type, int perturb_inst, double delta, double *tape, double *xbar_out,
                          int n_inst, double *maxabs) {
  const int n = 1 << level, m = level > 0 ? n / 2 : 0;
  const double h = ldexp(p->T, -level);
  const double disc = exp(-p->r * p->T);
  double *Z = tape, *S = Z + n, *mul1 = S + n + 1, *sum1 = mul1 + n, *mul2 = sum1 + n;
  double *Zc = mul2 + n, *Sc = Zc + m, *mul1c = Sc + m + 1, *sum1c = mul1c + m, *mul2c = sum1c + m;
#define PERT(type, inst, x) ((perturb_type == (type) && perturb_inst == (inst)) ? (x) + delta : (x))
  double con1 = PERT(V_CON1, 0, p->r * h);
  double con1c = PERT(V_CON1, 1, p->r * (2.0 * h));
  double con2 = PERT(V_CON2, 0, p->sigma * sqrt(h));
  double S0 = PERT(V_S, n + m, p->S0);
  /* forward sweep, fine path (Algorithm 1) */
  S[0] = S0;
  for (int k = 0; k < n; ++k) {
    Z[k] = PERT(V_Z, k, or_exact_normal(or_draw(seed, request, (uint32_t)level, 0u, s, (uint32_t)k)));
    mul1[k] = PERT(V_MUL1, k, con2 * Z[k]);
    sum1[k] = PERT(V_SUM1, k, con1 + mul1[k]);
    mul2[k] = PERT(V_MUL2, k, S[k] * sum1[k]);
    S[k + 1] = PERT(V_S, k, S[k] + mul2[k]);
  }
  /* coarse path: one step of 2h per pair of fine increments */
  if (level > 0) {
    Sc[0] = S0;
    for (int k = 0; k < m; ++k) {
      Zc[k] = Z[2 * k] + Z[2 * k + 1];
      mul1c[k] = PERT(V_MUL1, n + k, con2 * Zc[k]);
      sum1c[k] = PERT(V_SUM1, n + k, con1c + mul1c[k]);
      mul2c[k] = PERT(V_MUL2, n + k, Sc[k] * sum1c[k]);
      Sc[k + 1] = PERT(V_S, n + k, Sc[k] + mul2c[k]);
    }
  }
#undef PERT
  const double Pf = disc * (S[n] > p->K ? S[n] - p->K : 0.0);
  const double Pc = level > 0 ? disc * (Sc[m] > p->K ? Sc[m] - p->K : 0.0) : 0.0;
  if (maxabs) {
    double v[7] = {0, 0, 0, 0, 0, 0, 0};
    v[V_CON1] = fmax(fabs(con1), level > 0 ? fabs(con1c) : 0.0);
    v[V_CON2] = fabs(con2);
    v[V_S] = fabs(S0);
    for (int k = 0; k < n; ++k) {
      v[V_Z] = fmax(v[V_Z], fabs(Z[k]));
      v[V_MUL1] = fmax(v[V_MUL1], fabs(mul1[k]));
      v[V_SUM1] = fmax(v[V_SUM1], fabs(sum1[k]));
      v[V_MUL2] = fmax(v[V_MUL2], fabs(mul2[k]));
      v[V_S] = fmax(v[V_S], fabs(S[k + 1]));
    }
    for (int k = 0; k < m; ++k) {
      v[V_MUL1] = fmax(v[V_MUL1], fabs(mul1c[k]));
      v[V_SUM1] = fmax(v[V_SUM1], fabs(sum1c[k]));
      v[V_MUL2] = fmax(v[V_MUL2], fabs(mul2c[k]));
      v[V_S] = fmax(v[V_S], fabs(Sc[k + 1]));
    }
    for (int t = 0; t < 7; ++t) maxabs[t] = fmax(maxabs[t], v[t]);
  }
  if (xbar_out) {
    double *xb[7];
    for (int t = 0; t < 7; ++t) {
      xb[t] = xbar_out + (size_t)t * n_inst;
      for (int i = 0; i < n_inst; ++i) xb[t][i] = 0.0;
    }
    /* backward sweep, fine path: seed dDeltaP/dS_n = disc 1[S_n > K] */
    double Sbar = S[n] > p->K ? disc : 0.0;
    double con1bar = 0.0, con2bar = 0.0;
    for (int k = n - 1; k >= 0; --k) {
      xb[V_S][k] = Sbar;                       /* S_{k+1} = S_k + mul2_k     */
      const double mul2bar = Sbar;
      xb[V_MUL2][k] = mul2bar;                 /* mul2_k = S_k * sum1_k      */
      const double sum1bar = mul2bar * S[k];
      Sbar = Sbar + mul2bar * sum1[k];
      xb[V_SUM1][k] = sum1bar;                 /* sum1_k = con1 + mul1_k     */
      const double mul1bar = sum1bar;
      con1bar += sum1bar;
      xb[V_MUL1][k] = mul1bar;                 /* mul1_k = con2 * Z_k        */
      con2bar += mul1bar * Z[k];
      xb[V_Z][k] += mul1bar * con2;
    }
    double S0bar = Sbar;
    xb[V_CON1][0] = con1bar;
    if (level > 0) {
      /* backward sweep, coarse path: seed -disc 1[S^c_m > K] */
      double Scbar = Sc[m] > p->K ? -disc : 0.0;
      double con1cbar = 0.0;
      for (int k = m - 1; k >= 0; --k) {
        xb[V_S][n + k] = Scbar;
        const double mul2bar = Scbar;
        xb[V_MUL2][n + k] = mul2bar;
        const double sum1bar = mul2bar * Sc[k];
        Scbar = Scbar + mul2bar * sum1c[k];
        xb[V_SUM1][n + k] = sum1bar;
        const double mul1bar = sum1bar;
        con1cbar += sum1bar;
        xb[V_MUL1][n + k] = mul1bar;
        con2bar += mul1bar * Zc[k];
        xb[V_Z][2 * k] += mul1bar * con2;      /* Zc_k = Z_2k + Z_2k+1        */
        xb[V_Z][2 * k + 1] += mul1bar * con2;
      }
      S0bar += Scbar;
      xb[V_CON1][1] = con1cbar;
    }
    xb[V_CON2][0] = con2bar;
    xb[V_S][n + m] = S0bar;
  }
  return Pf - Pc;
}

/* Number of instances per type at a level (the stride of per-instance arrays). */
int or_sens_instances(int level) { return (1 << level) + (level > 0 ? (1 << level) / 2 : 0) + 1; }

/* Statistics over samples [first, first + N): per-type sums of xbar^2, maxima,
 * sums of DeltaP and DeltaP^2, and (if inst != 0) per-instance sums of xbar^2
 * (7 x or_sens_instances(level), type-major).  European call, Euler only. */
int or_sensitivities(const or_params *p, int level, uint64_t first, uint64_t N, uint64_t seed, uint32_t request,
                     or_sens *out, double *inst) {
  if (level < 0 || level > 12 || p->payoff != OR_EURO || p->scheme != OR_EULER) return OR_EINVAL;
  const int n = 1 << level, m = level > 0 ? n / 2 : 0;
  const int ni = or_sens_instances(level);
  static double tape[5 * 4096 + 1 + 5 * 2048 + 1];
  static double xbar[7 * (4096 + 2048 + 1)];
  memset(out, 0, sizeof *out);
  if (inst) for (int i = 0; i < 7 * ni; ++i) inst[i] = 0.0;
  neumaier A[7], sdp = {0, 0}, sdp2 = {0, 0};
  memset(A, 0, sizeof A);
  (void)m;
  for (uint64_t s = first; s < first + N; ++s) {
    const double dp = sens_sample(p, level, seed, request, s, -1, -1, 0.0, tape, xbar, ni, out->maxabs);
    nm_add(&sdp, dp);
    nm_add(&sdp2, dp * dp);
    for (int t = 0; t < 7; ++t) {
      double a = 0.0;
      for (int i = 0; i < ni; ++i) {
        const double x = xbar[(size_t)t * ni + i];
        a += x * x;
        if (inst) inst[(size_t)t * ni + i] += x * x;
      }
      nm_add(&A[t], a);
    }
  }
  for (int t = 0; t < 7; ++t) out->A[t] = A[t].s + A[t].c;
  out->sum_dp = sdp.s + sdp.c;
  out->sum_dp2 = sdp2.s + sdp2.c;
  out->n = N;
  return OR_OK;
}

/* DeltaP of one sample with delta added to one instance, and the adjoint
 * sensitivities of all instances of the unperturbed sample (xbar: 7 x n_inst). */
double or_sens_probe(const or_params *p, int level, uint64_t seed, uint32_t request, uint64_t s, int type,
                     int inst, double delta, double *xbar) {
  static double tape[5 * 4096 + 1 + 5 * 2048 + 1];
  if (xbar) sens_sample(p, level, seed, request, s, -1, -1, 0.0, tape, xbar, or_sens_instances(level), 0);
  return sens_sample(p, level, seed, request, s, type, inst, delta, tape, 0, 0, 0);
}
