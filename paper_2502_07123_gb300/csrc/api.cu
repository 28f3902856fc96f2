// Host side of the C ABI declared in include/mlmc.h: device context and table
// cache, work-item planning (chunking, per-level constants and fixed-point
// formats), plan launch on forked streams, the deterministic finalize kernel,
// and the adaptive MLMC driver (Sec. 2.1-2.2 sample allocation).
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

// The Python binding mirrors these layouts.
static_assert(sizeof(mlmc_params) == 80, "mlmc_params layout");
static_assert(sizeof(mlmc_sums) == 72, "mlmc_sums layout");
static_assert(sizeof(mlmc_work) == 40, "mlmc_work layout");
static_assert(sizeof(mlmc_sample) == 80, "mlmc_sample layout");
static_assert(sizeof(mlmc_format) == 14, "mlmc_format layout");

// ---------------------------------------------------------------------------
// plan object (opaque in the C ABI)
// ---------------------------------------------------------------------------
struct LaunchRec {
  int family;               // kernel family, see launch_by_family
  int scheme, pc;
  int threads;              // CTA size
  uint32_t chunk0, n_chunks;
  int item_off, n_items;
  size_t smem;
};

struct mlmc_plan {
  int n_work = 0;
  int threads = 128;
  std::vector<ItemDesc> items;       // launch sub-arrays first, zero-chunk items last
  std::vector<LaunchRec> launches;
  std::vector<double> disc;          // per work item
  std::vector<int> unit, exact_int;
  std::vector<uint64_t> N;
  uint32_t total_chunks = 0;
  uint64_t path_steps = 0;
  RoundKeys rk{};
  ItemDesc *d_items = nullptr;
  Partial *d_partials = nullptr;
  DevSums *d_out = nullptr;
  uint32_t *d_counters = nullptr;    // per item, zero between launches
  std::vector<uint32_t> empty_out;   // out_index of items without samples (sums reset per launch)
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> join;
  std::vector<cudaEvent_t> kstart, kstop;   // around each level kernel, on its stream
  cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
  cudaStream_t last_stream = nullptr;
  bool launched = false;
  bool borrowed = false;   // device buffers, streams and events belong to the context arena
};

namespace mlmc_host {

// ---------------------------------------------------------------------------
// device context and table cache
// ---------------------------------------------------------------------------
// Reusable device buffers, streams and events of the synchronous calls
// (mlmc_level, mlmc_run, mlmc_estimate), grown on demand.
struct Arena {
  ItemDesc *items = nullptr;
  size_t cap_items = 0;
  Partial *partials = nullptr;
  size_t cap_chunks = 0;
  DevSums *out = nullptr;
  size_t cap_out = 0;
  uint32_t *counters = nullptr;
  size_t cap_counters = 0;
  ItemDesc *h_items = nullptr;       // pinned staging of the work list
  size_t cap_h_items = 0;
  DevSums *h_out = nullptr;          // pinned staging of the results
  size_t cap_h_out = 0;
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> join, kstart, kstop;
  cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
};

struct Ctx {
  bool inited = false;
  Arena arena;
  int device = -1;
  int num_sms = 0;
  cudaStream_t st = nullptr;
  std::map<int, std::vector<double>> m1_host;               // d -> Method-1 table (FP64)
  std::map<int, double *> m1_dev;                           // d -> device FP64 table
  std::map<std::tuple<int, int, int, int, int>, void *> tables;  // (method, d, rep, fZ, signed) -> table
  std::map<int, uint16_t *> m2_perm;                         // d -> device interval ranks (Method 2)
};
Ctx g;

// Work items already built, by everything their constants depend on (params,
// the level's format, level, variant, stream); the sample range is set per call.
struct CachedItem {
  BuiltItem b;
  double disc;
  int unit, exact_int;
};
std::unordered_map<std::string, CachedItem> g_item_cache;

double g_cost[4] = {8.0, 1.0, 0.5, 1.5};
const double g_cost_default[4] = {8.0, 1.0, 0.5, 1.5};

// Launch shape per (kernel family, scheme, payoff class, level class): CTA
// threads and fine path-steps per thread.  Defaults 128 / 256 until
// mlmc_autotune installs measured choices.
constexpr int TUNE_THREADS = 128, TUNE_SPT = 256;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune;

int level_class(int level) { return level <= 1 ? level : (level <= 4 ? 2 : (level <= 7 ? 3 : 4)); }

void tuning_for(int family, int scheme, int pc, int level, int *threads, int *spt) {
  auto f = g_tune.find(std::make_tuple(family, scheme, pc, level_class(level)));
  *threads = f == g_tune.end() ? TUNE_THREADS : f->second.first;
  *spt = f == g_tune.end() ? TUNE_SPT : f->second.second;
}

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return MLMC_ECUDA;         \
  } while (0)

mlmc_status ensure_ctx() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return MLMC_ECUDA;
  if (g.inited && g.device == dev) return MLMC_OK;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return MLMC_ECUDA;
  if (g.inited && g.device != dev) {
    // a different device became current: start a fresh cache for it
    g.m1_host.clear();
    g.m1_dev.clear();
    g.tables.clear();
    g.m2_perm.clear();
    g_item_cache.clear();
  }
  CK(cudaDeviceGetAttribute(&g.num_sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking));
  g.device = dev;
  g.inited = true;
  return MLMC_OK;
}

mlmc_status m1_table(int d, double **dev, const std::vector<double> **host) {
  auto it = g.m1_dev.find(d);
  if (it == g.m1_dev.end()) {
    const int n = 1 << (d - 1);
    double *p = nullptr;
    CK(cudaMalloc(&p, sizeof(double) * n));
    CK(launch_m1_table(d, p, g.st));
    std::vector<double> h(n);
    CK(cudaMemcpyAsync(h.data(), p, sizeof(double) * n, cudaMemcpyDeviceToHost, g.st));
    CK(cudaStreamSynchronize(g.st));
    g.m1_dev[d] = p;
    g.m1_host[d] = std::move(h);
    it = g.m1_dev.find(d);
  }
  *dev = it->second;
  *host = &g.m1_host[d];
  return MLMC_OK;
}

// Method 3 (Sec. 3.3): least-squares line a + b k through (k, Z_k) on each
// dyadic index class {0,1}, {2,3}, {4..7}, ..., {2^(d-2) .. 2^(d-1)-1}.
void m3_fit(const std::vector<double> &Z, int d, M3Coef &c) {
  std::memset(&c, 0, sizeof c);
  for (int cls = 0; cls < d - 1; ++cls) {
    const int lo = cls == 0 ? 0 : (1 << cls);
    const int hi = cls == 0 ? 1 : (1 << (cls + 1)) - 1;
    const int n = hi - lo + 1;
    double kbar = 0.0, zbar = 0.0;
    for (int k = lo; k <= hi; ++k) { kbar += k; zbar += Z[k]; }
    kbar /= n;
    zbar /= n;
    double sxx = 0.0, sxy = 0.0;
    for (int k = lo; k <= hi; ++k) {
      sxx += (k - kbar) * (k - kbar);
      sxy += (k - kbar) * (Z[k] - zbar);
    }
    const double b = sxy / sxx;
    const double a = zbar - b * kbar;
    c.a[cls] = (float)a;
    c.b[cls] = (float)b;
    c.A[cls] = (int64_t)std::floor(std::ldexp(a, M3_FRAC) + 0.5);
    c.B[cls] = (int64_t)std::floor(std::ldexp(b, M3_FRAC) + 0.5);
  }
}

// Device table of one representation.  full_signed (method 1 only): all 2^d
// entries indexed directly by j, as the level kernels use it; otherwise the
// 2^(d-1) entries of the lower half (parity checks).
uint16_t half_bits(double x) { return __half_as_ushort(__double2half(x)); }
uint16_t bf16_bits(double x) { return __bfloat16_as_ushort(__double2bfloat16(x)); }

// Method 2 (Sec. 3.2) with two fields: the d-bit index j splits into a high
// and a low field of b = d/2 bits; each gives +-x_k from a small table of
// 2^(b-1) values (Method-1 sign rule per field) and Z~_j is their sum.  The
// small table starts as the b-bit Method-1 table / sqrt(2); then the 2^d sums
// are ranked ascending (ties by j), pi(j) = rank, and x is refitted by least
// squares (normal equations, Cholesky in long double) to the d-bit Method-1
// values Z_{pi(j)}, until pi stops changing (at most 1000 fits).
struct M2Table {
  std::vector<double> x;         // small table
  std::vector<double> values;    // Z~_j, j < 2^d, FP64 sums in field order
  std::vector<uint32_t> pi;      // interval rank of every j
  int iterations = 0;
};
std::map<int, M2Table> g_m2;

struct M2Field { int idx; double sgn; };
inline void m2_fields(int j, int b, M2Field &hi, M2Field &lo) {
  const int full = 1 << b, half = 1 << (b - 1);
  const int f1 = j >> b, f2 = j & (full - 1);
  hi = f1 < half ? M2Field{f1, 1.0} : M2Field{full - 1 - f1, -1.0};
  lo = f2 < half ? M2Field{f2, 1.0} : M2Field{full - 1 - f2, -1.0};
}

bool chol_solve(std::vector<long double> M, std::vector<long double> r, int k, std::vector<double> &y) {
  for (int c = 0; c < k; ++c) {
    long double dg = M[c * k + c];
    for (int q = 0; q < c; ++q) dg -= M[c * k + q] * M[c * k + q];
    if (!(dg > 0.0L)) return false;
    dg = std::sqrt(dg);
    M[c * k + c] = dg;
    for (int rr = c + 1; rr < k; ++rr) {
      long double v = M[rr * k + c];
      for (int q = 0; q < c; ++q) v -= M[rr * k + q] * M[c * k + q];
      M[rr * k + c] = v / dg;
    }
  }
  for (int c = 0; c < k; ++c) {          // L z = r
    long double v = r[c];
    for (int q = 0; q < c; ++q) v -= M[c * k + q] * r[q];
    r[c] = v / M[c * k + c];
  }
  for (int c = k - 1; c >= 0; --c) {     // L^T y = z
    long double v = r[c];
    for (int q = c + 1; q < k; ++q) v -= M[q * k + c] * r[q];
    r[c] = v / M[c * k + c];
  }
  y.resize(k);
  for (int c = 0; c < k; ++c) y[c] = (double)r[c];
  return true;
}

mlmc_status m2_build(int d, const M2Table **out) {
  auto it = g_m2.find(d);
  if (it != g_m2.end()) { *out = &it->second; return MLMC_OK; }
  if (d % 2 || d < 4) return MLMC_EINVAL;
  const int b = d / 2, k = 1 << (b - 1), N = 1 << d;
  double *dv;
  const std::vector<double> *zb = nullptr, *zd = nullptr;
  mlmc_status s;
  if ((s = m1_table(b, &dv, &zb)) != MLMC_OK) return s;
  if ((s = m1_table(d, &dv, &zd)) != MLMC_OK) return s;
  std::vector<double> T(N);
  for (int j = 0; j < N; ++j) T[j] = j < N / 2 ? (*zd)[j] : -(*zd)[N - 1 - j];
  std::vector<M2Field> fh(N), fl(N);
  for (int j = 0; j < N; ++j) m2_fields(j, b, fh[j], fl[j]);
  // normal matrix A^T A (A has one +-1 per field in every row)
  std::vector<long double> M((size_t)k * k, 0.0L);
  for (int j = 0; j < N; ++j) {
    const M2Field f[2] = {fh[j], fl[j]};
    for (int a = 0; a < 2; ++a)
      for (int c = 0; c < 2; ++c) M[(size_t)f[a].idx * k + f[c].idx] += (long double)(f[a].sgn * f[c].sgn);
  }
  M2Table t;
  t.x.resize(k);
  for (int q = 0; q < k; ++q) t.x[q] = (*zb)[q] / std::sqrt(2.0);
  auto sums = [&](const std::vector<double> &x, std::vector<double> &v) {
    v.resize(N);
    for (int j = 0; j < N; ++j) v[j] = fh[j].sgn * x[fh[j].idx] + fl[j].sgn * x[fl[j].idx];
  };
  auto rank = [&](const std::vector<double> &v, std::vector<uint32_t> &pi) {
    std::vector<int> order(N);
    for (int j = 0; j < N; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return v[a] < v[c]; });
    pi.resize(N);
    for (int r = 0; r < N; ++r) pi[order[r]] = (uint32_t)r;
  };
  sums(t.x, t.values);
  rank(t.values, t.pi);
  for (t.iterations = 0; t.iterations < 1000;) {
    std::vector<long double> rhs(k, 0.0L);
    for (int j = 0; j < N; ++j) {
      const long double y = T[t.pi[j]];
      rhs[fh[j].idx] += fh[j].sgn * y;
      rhs[fl[j].idx] += fl[j].sgn * y;
    }
    if (!chol_solve(M, rhs, k, t.x)) return MLMC_EINVAL;
    ++t.iterations;
    sums(t.x, t.values);
    std::vector<uint32_t> pn;
    rank(t.values, pn);
    if (pn == t.pi) break;
    t.pi.swap(pn);
  }
  auto ins = g_m2.emplace(d, std::move(t));
  *out = &ins.first->second;
  return MLMC_OK;
}

// Method-2 value of index j in a representation: each small-table value rounded
// once, the two fields added exactly (fixed point) or with one rounding.
double m2_value(const M2Table &t, int d, int j, int rep, int fZ) {
  const int b = d / 2;
  M2Field h, l;
  m2_fields(j, b, h, l);
  const double a = t.x[h.idx], c = t.x[l.idx];
  switch (rep) {
    case REP_FIXED: {
      const int64_t qa = (int64_t)std::floor(std::ldexp(a, fZ) + 0.5), qc = (int64_t)std::floor(std::ldexp(c, fZ) + 0.5);
      return std::ldexp((double)((int64_t)h.sgn * qa + (int64_t)l.sgn * qc), -fZ);
    }
    case REP_FP16: {
      const double ha = (double)__half2float(__double2half(a)), hc = (double)__half2float(__double2half(c));
      return (double)__half2float(__double2half(h.sgn * ha + l.sgn * hc));
    }
    case REP_BF16: {
      const double ba = (double)__bfloat162float(__double2bfloat16(a));
      const double bc = (double)__bfloat162float(__double2bfloat16(c));
      return (double)__bfloat162float(__double2bfloat16(h.sgn * ba + l.sgn * bc));
    }
    case REP_FP32: {
      const double fa = (double)(float)a, fc = (double)(float)c;
      return (double)(float)(h.sgn * fa + l.sgn * fc);
    }
    default: return t.values[j];
  }
}

// Device copy of the Method-2 interval ranks of index width d.
mlmc_status m2_perm_device(int d, const uint16_t **out) {
  auto it = g.m2_perm.find(d);
  if (it != g.m2_perm.end()) { *out = it->second; return MLMC_OK; }
  const M2Table *t;
  mlmc_status s = m2_build(d, &t);
  if (s != MLMC_OK) return s;
  std::vector<uint16_t> h(1 << d);
  for (int j = 0; j < (1 << d); ++j) h[j] = (uint16_t)t->pi[j];
  uint16_t *p = nullptr;
  CK(cudaMalloc(&p, sizeof(uint16_t) * h.size()));
  CK(cudaMemcpy(p, h.data(), sizeof(uint16_t) * h.size(), cudaMemcpyHostToDevice));
  g.m2_perm[d] = p;
  *out = p;
  return MLMC_OK;
}

mlmc_status get_table(int method, int d, int rep, int fZ, const void **out, bool full_signed = false) {
  if (rep != REP_FIXED) fZ = 0;
  if (method == 3) full_signed = false;
  auto key = std::make_tuple(method, d, rep, fZ, full_signed ? 1 : 0);
  auto it = g.tables.find(key);
  if (it != g.tables.end()) { *out = it->second; return MLMC_OK; }
  double *z64 = nullptr;
  const std::vector<double> *zh = nullptr;
  mlmc_status s = m1_table(d, &z64, &zh);
  if (s != MLMC_OK) return s;
  void *p = nullptr;
  const int n = 1 << (d - 1);
  if (method == 2) {
    // the signed table over all 2^d indices, built on the host
    if (!full_signed) return MLMC_EINVAL;
    const M2Table *t;
    if ((s = m2_build(d, &t)) != MLMC_OK) return s;
    if (rep == REP_FIXED) {
      std::vector<int32_t> h(2 * n);
      for (int j = 0; j < 2 * n; ++j) h[j] = (int32_t)std::llround(std::ldexp(m2_value(*t, d, j, rep, fZ), fZ));
      CK(cudaMalloc(&p, sizeof(int32_t) * h.size()));
      CK(cudaMemcpy(p, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice));
    } else if (rep == REP_FP16 || rep == REP_BF16) {
      std::vector<uint16_t> h(2 * n);
      for (int j = 0; j < 2 * n; ++j) {
        const double v = m2_value(*t, d, j, rep, fZ);
        h[j] = rep == REP_FP16 ? half_bits(v) : bf16_bits(v);
      }
      CK(cudaMalloc(&p, sizeof(uint16_t) * h.size()));
      CK(cudaMemcpy(p, h.data(), sizeof(uint16_t) * h.size(), cudaMemcpyHostToDevice));
    } else {
      return MLMC_EINVAL;
    }
  } else if (method == 1 && full_signed) {
    const size_t es = (rep == REP_FP16 || rep == REP_BF16) ? 2 : 4;
    CK(cudaMalloc(&p, es * 2 * n));
    CK(launch_m1_signed(z64, d, rep, fZ, p, g.st));
    CK(cudaStreamSynchronize(g.st));
  } else if (method == 1) {
    if (rep == REP_FP64) {
      p = z64;
    } else {
      const size_t es = (rep == REP_FP16 || rep == REP_BF16) ? 2 : 4;
      CK(cudaMalloc(&p, es * n));
      CK(launch_m1_convert(z64, n, rep, fZ, p, g.st));
      CK(cudaStreamSynchronize(g.st));
    }
  } else {
    M3Coef c;
    m3_fit(*zh, d, c);
    CK(cudaMalloc(&p, sizeof(M3Coef)));
    CK(cudaMemcpy(p, &c, sizeof(M3Coef), cudaMemcpyHostToDevice));
  }
  g.tables[key] = p;
  *out = p;
  return MLMC_OK;
}

// ---------------------------------------------------------------------------
// parameters, formats and constants
// ---------------------------------------------------------------------------
enum { F_Z = 0, F_CON1 = 1, F_CON2 = 2, F_MUL1 = 3, F_SUM1 = 4, F_MUL2 = 5, F_S = 6 };

bool params_ok(const mlmc_params *p) {
  if (!p) return false;
  if (!(std::isfinite(p->S0) && std::isfinite(p->K) && std::isfinite(p->r) && std::isfinite(p->sigma) &&
        std::isfinite(p->T)))
    return false;
  if (!(p->S0 > 0.0) || p->K < 0.0 || p->sigma < 0.0 || !(p->T > 0.0)) return false;
  if (p->payoff < 0 || p->payoff > 3 || p->scheme < 0 || p->scheme > 1) return false;
  if (p->icdf_method < 1 || p->icdf_method > 3) return false;
  if (p->icdf_bits < 2 || p->icdf_bits > 14) return false;
  if (p->icdf_method == 2 && (p->icdf_bits % 2 || p->icdf_bits < 4)) return false;   // two fields of >= 2 bits
  if (p->formats && p->n_formats < 0) return false;
  if (p->rng_pack != 0 && p->rng_pack != 1) return false;
  if (p->reserved != 0) return false;
  return true;
}

// Lanes per pack of an approximate-only estimator (packed draws need 3 fields of d bits).
int pack_lanes(const mlmc_params *p, int variant) {
  const bool approx_only = variant == MLMC_FIXED_APPROX || variant == MLMC_FP16_APPROX || variant == MLMC_BF16_APPROX;
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
  e[F_S] = bitlen_rounded(std::max(S0 * std::exp(std::fabs(r) * T + 6.0 * sig * std::sqrt(T)), K), f[F_S]);
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
  // 0 exact f32, 1 exact f64, 2 approx fixed, 3 approx f16, 4 approx bf16, 5 corr fixed, 6 corr f16, 7 corr bf16
  switch (variant) {
    case MLMC_FP32_EXACT: return 0;
    case MLMC_FP64_EXACT: return 1;
    case MLMC_FIXED_APPROX: return 2;
    case MLMC_FP16_APPROX: return 3;
    case MLMC_BF16_APPROX: return 4;
    case MLMC_NESTED_CORR_FIXED: return 5;
    case MLMC_NESTED_CORR_FP16: return 6;
    default: return 7;
  }
}
int cost_kind_of(int variant) {
  if (variant == MLMC_FP64_EXACT) return 0;
  if (variant == MLMC_FP32_EXACT) return 1;
  if (variant == MLMC_FIXED_APPROX || variant == MLMC_FP16_APPROX || variant == MLMC_BF16_APPROX) return 2;
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
bool fast_fixed(const int e[7], const int f[7], int64_t con1, int64_t con1c, int64_t con2, int64_t con3,
                int64_t zmax, bool milstein, FastFixed &ff, bool &s64) {
  typedef __int128 I;
  const int fZ = f[F_Z];
  if (f[F_CON1] < f[F_MUL1] || f[F_CON1] < f[F_SUM1] || f[F_S] < f[F_MUL2]) return false;
  const int rs1 = f[F_CON2] + fZ - f[F_MUL1];
  const int rs3 = f[F_CON1] + 2 * fZ - f[F_MUL1];
  const int rs_sum1 = f[F_CON1] - f[F_SUM1];
  const int rs2 = f[F_S] + f[F_SUM1] - f[F_MUL2];
  if (rs1 < 0 || rs3 < 0 || rs2 < 0 || rs1 > 62 || rs3 > 62 || rs2 > 62 || rs_sum1 > 30) return false;
  const int shF1 = f[F_CON1] - f[F_MUL1];
  const int shS = f[F_S] - f[F_MUL2];
  if (shF1 > 30 || shS > 30) return false;
  auto lim = [&](int v) { return ((I)1 << (e[v] + f[v])) - 1; };
  const I zc = 2 * (I)zmax;  // coarse increments are sums of two table values
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
  const I c1max = std::max((I)(con1 < 0 ? -con1 : con1), (I)(con1c < 0 ? -con1c : con1c));
  const I acc_abs = c1max + rsum + (mul1_abs + mul3_abs) * ((I)1 << shF1);
  if (acc_abs >= ((I)1 << 31) - 1) return false;
  const I sum1_abs = floor_shift(acc_abs, rs_sum1) + 1;
  if (sum1_abs > lim(F_SUM1)) return false;
  const I limS = lim(F_S);
  if (limS * sum1_abs + r2 >= ((I)1 << 62)) return false;
  const I mul2_abs = floor_shift(limS * sum1_abs + r2, rs2) + 1;
  if (mul2_abs > lim(F_MUL2) || mul2_abs >= ((I)1 << 31)) return false;
  const I snew = limS + mul2_abs * ((I)1 << shS);
  if (snew >= ((I)1 << 62)) return false;
  s64 = !(snew < ((I)1 << 31) - 1);
  ff.con2 = (int32_t)con2;
  ff.con3 = (int32_t)con3;
  ff.con1r = (int32_t)(con1 + (int64_t)rsum);
  ff.con1cr = (int32_t)(con1c + (int64_t)rsum);
  ff.mulF1 = 1 << shF1;
  ff.rs1 = rs1; ff.rs3 = rs3; ff.rs_sum1 = rs_sum1; ff.rs2 = rs2;
  ff.mulS = 1 << shS;
  ff.radd1 = (int64_t)r1; ff.radd3 = (int64_t)r3; ff.radd2 = (int64_t)r2;
  ff.mfine = (int64_t)1 << (2 * fZ);
  ff.mcoarse = (int64_t)2 << (2 * fZ);
  ff.limS = (int64_t)limS;
  return true;
}

// Largest |table value| in Z's fixed-point format, as the kernels evaluate it.
int64_t table_zmax_fixed(const std::vector<double> &Z, int d, int method, int fZ) {
  int64_t zmax = 0;
  if (method == 2) {
    const M2Table *t;
    if (m2_build(d, &t) != MLMC_OK) return INT64_MAX;
    for (int j = 0; j < (1 << d); ++j)
      zmax = std::max<int64_t>(zmax, std::llabs(std::llround(std::ldexp(m2_value(*t, d, j, REP_FIXED, fZ), fZ))));
    return zmax;
  }
  if (method == 1) {
    for (double v : Z) zmax = std::max<int64_t>(zmax, std::llabs((int64_t)std::floor(std::ldexp(v, fZ) + 0.5)));
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



// Split an item's sample groups into chunks of `threads` x groups_per_thread.
mlmc_status chunk_built(BuiltItem &b, int threads, int spt) {
  ItemDesc &it = b.it;
  uint32_t gpt = 1;
  const uint64_t spg = steps_per_group(it.level);
  const uint64_t nch = chunk_count(it.g1 - it.g0, spg, b.kp, threads, spt, g.num_sms, &gpt);
  if (nch > 0x7fffffffULL) return MLMC_EINVAL;
  it.groups_per_thread = gpt;
  it.n_chunks = (uint32_t)nch;
  b.chunk_cost = (double)gpt * (double)threads * (double)spg * b.kp * b.cost_step;
  return MLMC_OK;
}

// Packed draws of an item with fewer packs than one wave of resident threads
// run one sample per thread: latency rather than throughput bounds such items.
bool lane_split(uint64_t N) {
  const uint64_t wave = 6ULL * 128ULL * (uint64_t)std::max(1, g.num_sms);
  return N > 0 && (N + 2) / 3 < wave;
}

mlmc_status build_item(const mlmc_work &w, int out_index, void *dump, BuiltItem &b, double &disc, int &unit,
                       int &exact_int) {
  const mlmc_params *p = w.params;
  if (!params_ok(p)) return MLMC_EINVAL;
  if (w.level < 0 || w.level > 20 || w.variant < 0 || w.variant > 7) return MLMC_EINVAL;
  if (w.stream < -1 || w.stream > 255) return MLMC_EINVAL;
  const int lev = w.level;
  // word index s 2^l + i and the group index must stay below 2^62
  if (w.N > (1ULL << 58) || w.first_sample > (1ULL << (60 - lev)) - w.N) return MLMC_EINVAL;
  ItemDesc &it = b.it;
  std::memset(&it, 0, sizeof it);
  const int v = w.variant;
  const bool approx = !(v == MLMC_FP32_EXACT || v == MLMC_FP64_EXACT);
  const int stream = w.stream >= 0 ? w.stream
                     : (v == MLMC_FIXED_APPROX || v == MLMC_FP16_APPROX || v == MLMC_BF16_APPROX ? 1 : 0);
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
    const bool approx_only = v == MLMC_FIXED_APPROX || v == MLMC_FP16_APPROX || v == MLMC_BF16_APPROX;
    const int bits = p->icdf_bits << lev;
    if (!approx_only || lev > 1 || bits > 24 || w.first_sample != 0 || w.N != (1ULL << bits)) return MLMC_EINVAL;
    KP = 1;
    it.enumerate = 1;
  }
  if (KP == 0) return MLMC_EINVAL;
  if (KP == 3 && lev >= 2 && lane_split(w.N)) {
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
    const bool bf = (v == MLMC_BF16_APPROX || v == MLMC_NESTED_CORR_BF16);
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
      double *z64;
      const std::vector<double> *zh;
      if ((s = m1_table(p->icdf_bits, &z64, &zh)) != MLMC_OK) return s;
      const int64_t zmax = table_zmax_fixed(*zh, p->icdf_bits, p->icdf_method, fZ);
      if ((double)zmax > std::ldexp(1.0, e[F_Z] + fZ) - 1.0) return MLMC_EOVERFLOW;
      unit = f[F_S] + (p->payoff == MLMC_ASIAN ? lev + 1 : 0);
      bool s64 = false;
      fast = fast_fixed(e, f, con1, con1c, con2, con3, zmax, p->scheme == MLMC_MILSTEIN, it.ff, s64);
      fast64 = s64;
      if (fast && !s64) {
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
    mlmc_status s = get_table(p->icdf_method, p->icdf_bits, rep, fZ, &tab, true);
    if (s != MLMC_OK) return s;
    it.ztab = tab;
    b.smem = p->icdf_method != 3 ? (size_t)(1 << p->icdf_bits) * (fixed ? 4 : 2) : sizeof(M3Coef);
    exact_int = (v == MLMC_FIXED_APPROX || v == MLMC_FP16_APPROX || v == MLMC_BF16_APPROX) ? 1 : 0;
    if (p->icdf_method == 2 && !exact_int) {
      // Method 2 coupling: the correction's exact path reads the interval ranks
      const uint16_t *perm = nullptr;
      if ((s = m2_perm_device(p->icdf_bits, &perm)) != MLMC_OK) return s;
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
      default: return MLMC_EINVAL;
    }
  }
  b.scheme = p->scheme;
  b.pc = p->payoff == MLMC_ASIAN ? PC_ASIAN : (p->payoff == MLMC_LOOKBACK ? PC_LOOKBACK : PC_TERMINAL);
  return MLMC_OK;
}

// build_item through the cache (flags 0): the constants, tables and family
// come from the first build of the same (params, format, level, variant,
// stream); the sample range and its groups are set for this call.
mlmc_status build_item_cached(const mlmc_work &w, int out_index, void *dump, BuiltItem &b, double &disc, int &unit,
                              int &exact_int) {
  const mlmc_params *p = w.params;
  if (w.flags != 0 || !params_ok(p) || w.level < 0 || w.level > 20)
    return build_item(w, out_index, dump, b, disc, unit, exact_int);
  std::string key;
  key.reserve(96);
  auto put = [&](const void *x, size_t n) { key.append((const char *)x, n); };
  put(&p->S0, sizeof(double) * 5);
  put(&p->payoff, sizeof(int32_t) * 4);
  put(&p->request_id, sizeof(uint32_t));
  put(&p->rng_pack, sizeof(int32_t));
  const int has_fmt = p->formats ? (w.level < p->n_formats ? 1 : 2) : 0;
  put(&has_fmt, sizeof has_fmt);
  if (has_fmt == 1) put(&p->formats[w.level], sizeof(mlmc_format));
  put(&w.level, sizeof(int32_t) * 2);     // level, variant
  put(&w.stream, sizeof(int32_t));
  const int split = lane_split(w.N) ? 1 : 0;   // the packed-draw layout depends on N
  put(&split, sizeof split);
  auto f = g_item_cache.find(key);
  if (f == g_item_cache.end()) {
    mlmc_status s = build_item(w, out_index, dump, b, disc, unit, exact_int);
    if (s != MLMC_OK) return s;
    if (g_item_cache.size() > 8192) g_item_cache.clear();
    g_item_cache.emplace(key, CachedItem{b, disc, unit, exact_int});
    return MLMC_OK;
  }
  const int lev = w.level;
  if (w.N > (1ULL << 58) || w.first_sample > (1ULL << (60 - lev)) - w.N) return MLMC_EINVAL;
  b = f->second.b;
  disc = f->second.disc;
  unit = f->second.unit;
  exact_int = f->second.exact_int;
  ItemDesc &it = b.it;
  it.first = w.first_sample;
  it.N = w.N;
  it.out_index = (uint32_t)out_index;
  it.dump = dump;
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

// Deterministic sum of each item's chunk partials (fixed lane assignment and
// tree order, so repeated launches give bit-identical results).
__global__ void finalize_kernel(const ItemDesc *items, int n_items, const Partial *partials, DevSums *out) {
  const int i = blockIdx.x;
  if (i >= n_items) return;
  const ItemDesc &it = items[i];
  const DevSums r = warp_sum_partials(partials + it.chunk_begin, it.n_chunks);
  if (threadIdx.x == 0) out[it.out_index] = r;
}

void free_plan_device(mlmc_plan *pl) {
  if (pl->borrowed) {
    pl->d_items = nullptr; pl->d_partials = nullptr; pl->d_out = nullptr; pl->d_counters = nullptr;
    pl->aux.clear(); pl->join.clear(); pl->kstart.clear(); pl->kstop.clear();
    pl->fork = pl->t0 = pl->t1 = nullptr;
    return;
  }
  if (pl->d_items) cudaFree(pl->d_items);
  if (pl->d_partials) cudaFree(pl->d_partials);
  if (pl->d_out) cudaFree(pl->d_out);
  if (pl->d_counters) cudaFree(pl->d_counters);
  for (auto s : pl->aux) cudaStreamDestroy(s);
  for (auto e : pl->join) cudaEventDestroy(e);
  for (auto e : pl->kstart) cudaEventDestroy(e);
  for (auto e : pl->kstop) cudaEventDestroy(e);
  pl->kstart.clear(); pl->kstop.clear();
  if (pl->fork) cudaEventDestroy(pl->fork);
  if (pl->t0) cudaEventDestroy(pl->t0);
  if (pl->t1) cudaEventDestroy(pl->t1);
  pl->d_items = nullptr; pl->d_partials = nullptr; pl->d_out = nullptr; pl->d_counters = nullptr;
  pl->aux.clear(); pl->join.clear();
  pl->fork = pl->t0 = pl->t1 = nullptr;
}

template <class T>
bool grow(T *&p, size_t &cap, size_t need) {
  if (need <= cap) return true;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  const size_t n = std::max(need, cap * 2);
  if (cudaMalloc(&p, sizeof(T) * n) != cudaSuccess) return false;
  cap = n;
  return true;
}

bool arena_events(Arena &A, size_t launches) {
  if (!A.t0) {
    if (cudaEventCreate(&A.t0) != cudaSuccess || cudaEventCreate(&A.t1) != cudaSuccess ||
        cudaEventCreateWithFlags(&A.fork, cudaEventDisableTiming) != cudaSuccess)
      return false;
  }
  while (A.aux.size() < launches) {
    cudaStream_t st;
    cudaEvent_t j, a, b;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
      return false;
    A.aux.push_back(st); A.join.push_back(j); A.kstart.push_back(a); A.kstop.push_back(b);
  }
  return true;
}

mlmc_status plan_create_impl(mlmc_plan **out, const mlmc_work *work, int n_work, uint64_t seed,
                             const mlmc_tuning *tuning, void *const *dumps, Arena *arena = nullptr,
                             bool defer_copy = false) {
  if (!out || !work || n_work <= 0) return MLMC_EINVAL;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  int o_threads = 0, o_spt = 0;  // 0: the tuning table's choice per item
  if (tuning) {
    o_threads = tuning->threads;
    o_spt = tuning->steps_per_thread;
    if (o_threads && (o_threads < 32 || o_threads > 128 || o_threads % 32)) return MLMC_EINVAL;
    if (o_spt < 0) return MLMC_EINVAL;
  }
  mlmc_plan *pl = new (std::nothrow) mlmc_plan;
  if (!pl) return MLMC_ENOMEM;
  pl->n_work = n_work;
  pl->disc.resize(n_work);
  pl->unit.resize(n_work);
  pl->exact_int.resize(n_work);
  pl->N.resize(n_work);
  std::vector<BuiltItem> built(n_work);
  std::vector<int> item_threads(n_work);
  for (int i = 0; i < n_work; ++i) {
    s = build_item_cached(work[i], i, dumps ? dumps[i] : nullptr, built[i], pl->disc[i], pl->unit[i],
                          pl->exact_int[i]);
    if (s != MLMC_OK) { delete pl; return s; }
    int th, sp;
    tuning_for(built[i].family, built[i].scheme, built[i].pc, work[i].level, &th, &sp);
    if (o_threads) th = o_threads;
    if (o_spt) sp = o_spt;
    item_threads[i] = th;
    s = chunk_built(built[i], th, sp);
    if (s != MLMC_OK) { delete pl; return s; }
    pl->N[i] = work[i].N;
    pl->path_steps += work[i].N << work[i].level;
  }
  // group by kernel configuration; within a launch, most expensive chunks first
  std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
  std::vector<int> empty;
  for (int i = 0; i < n_work; ++i) {
    if (built[i].it.n_chunks == 0) { empty.push_back(i); continue; }
    groups[std::make_tuple(built[i].family, built[i].scheme, built[i].pc, item_threads[i])].push_back(i);
  }
  // launches are ordered by their most expensive CTA, so that the longest
  // chains (deep levels, exact paths) start first and the rest fill in
  std::vector<std::pair<double, std::vector<int>>> order;
  for (auto &kv : groups) {
    auto &v = kv.second;
    std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return built[a].chunk_cost > built[b].chunk_cost; });
    order.push_back({built[v[0]].chunk_cost, v});
  }
  std::stable_sort(order.begin(), order.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
  uint32_t chunk = 0;
  for (auto &o : order) {
    LaunchRec L;
    const BuiltItem &b0 = built[o.second[0]];
    L.family = b0.family; L.scheme = b0.scheme; L.pc = b0.pc;
    L.threads = item_threads[o.second[0]];
    L.chunk0 = chunk;
    L.item_off = (int)pl->items.size();
    L.n_items = (int)o.second.size();
    L.smem = 0;
    for (int i : o.second) {
      ItemDesc it = built[i].it;
      it.chunk_begin = chunk;
      chunk += it.n_chunks;
      L.smem = std::max(L.smem, built[i].smem);
      pl->items.push_back(it);
    }
    L.n_chunks = chunk - L.chunk0;
    pl->launches.push_back(L);
  }
  for (int i : empty) {
    ItemDesc it = built[i].it;
    it.chunk_begin = chunk;
    pl->items.push_back(it);
    pl->empty_out.push_back(it.out_index);
  }
  pl->total_chunks = chunk;
  make_round_keys(seed, pl->rk);
  const size_t ni = pl->items.size();
  if (arena) {
    Arena &A = *arena;
    const size_t nl = pl->launches.size();
    const size_t old_counters = A.cap_counters;
    if (!grow(A.items, A.cap_items, ni) || !grow(A.partials, A.cap_chunks, std::max<size_t>(1, chunk)) ||
        !grow(A.out, A.cap_out, (size_t)n_work) || !grow(A.counters, A.cap_counters, ni) ||
        !arena_events(A, nl)) {
      delete pl;
      return MLMC_ENOMEM;
    }
    if (A.cap_counters != old_counters && cudaMemset(A.counters, 0, sizeof(uint32_t) * A.cap_counters) != cudaSuccess) {
      delete pl;
      return MLMC_ECUDA;
    }
    pl->borrowed = true;
    pl->d_items = A.items; pl->d_partials = A.partials; pl->d_out = A.out; pl->d_counters = A.counters;
    pl->fork = A.fork; pl->t0 = A.t0; pl->t1 = A.t1;
    if (nl > 1) {
      pl->aux.assign(A.aux.begin(), A.aux.begin() + nl);
      pl->join.assign(A.join.begin(), A.join.begin() + nl);
    }
    pl->kstart.assign(A.kstart.begin(), A.kstart.begin() + nl);
    pl->kstop.assign(A.kstop.begin(), A.kstop.begin() + nl);
    if (!defer_copy &&
        cudaMemcpyAsync(pl->d_items, pl->items.data(), sizeof(ItemDesc) * ni, cudaMemcpyHostToDevice, g.st) !=
            cudaSuccess) {
      delete pl;
      return MLMC_ECUDA;
    }
    *out = pl;
    return MLMC_OK;
  }
  if (cudaMalloc(&pl->d_items, sizeof(ItemDesc) * ni) != cudaSuccess ||
      cudaMalloc(&pl->d_partials, sizeof(Partial) * std::max<uint32_t>(1, chunk)) != cudaSuccess ||
      cudaMalloc(&pl->d_out, sizeof(DevSums) * n_work) != cudaSuccess ||
      cudaMalloc(&pl->d_counters, sizeof(uint32_t) * ni) != cudaSuccess) {
    free_plan_device(pl);
    delete pl;
    return MLMC_ENOMEM;
  }
  if (cudaMemset(pl->d_counters, 0, sizeof(uint32_t) * ni) != cudaSuccess) {
    free_plan_device(pl);
    delete pl;
    return MLMC_ECUDA;
  }
  if (cudaMemcpy(pl->d_items, pl->items.data(), sizeof(ItemDesc) * ni, cudaMemcpyHostToDevice) != cudaSuccess) {
    free_plan_device(pl);
    delete pl;
    return MLMC_ECUDA;
  }
  bool ok = cudaEventCreate(&pl->t0) == cudaSuccess && cudaEventCreate(&pl->t1) == cudaSuccess &&
            cudaEventCreateWithFlags(&pl->fork, cudaEventDisableTiming) == cudaSuccess;
  if (ok && pl->launches.size() > 1) {
    for (size_t i = 0; i < pl->launches.size() && ok; ++i) {
      cudaStream_t st;
      cudaEvent_t ev;
      ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
      if (ok) { pl->aux.push_back(st); pl->join.push_back(ev); }
    }
  }
  for (size_t i = 0; i < pl->launches.size() && ok; ++i) {
    cudaEvent_t a, b;
    ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
    if (ok) { pl->kstart.push_back(a); pl->kstop.push_back(b); }
  }
  if (!ok) { free_plan_device(pl); delete pl; return MLMC_ECUDA; }
  *out = pl;
  return MLMC_OK;
}

mlmc_status plan_launch_impl(mlmc_plan *pl, cudaStream_t st) {
  CK(cudaEventRecord(pl->t0, st));
  const bool fork = pl->launches.size() > 1;
  if (fork) CK(cudaEventRecord(pl->fork, st));
  for (size_t i = 0; i < pl->launches.size(); ++i) {
    const LaunchRec &L = pl->launches[i];
    cudaStream_t ls = st;
    if (fork) {
      ls = pl->aux[i];
      CK(cudaStreamWaitEvent(ls, pl->fork, 0));
    }
    LaunchArgs a;
    a.items = pl->d_items + L.item_off;
    a.n_items = L.n_items;
    a.chunk0 = L.chunk0;
    a.dyn = nullptr;
    a.partials = pl->d_partials;
    a.rk = pl->rk;
    a.counters = pl->d_counters + L.item_off;
    a.out = pl->d_out;
    // per-kernel events only for plans a caller owns (mlmc_plan_kernel_time)
    if (!pl->borrowed) CK(cudaEventRecord(pl->kstart[i], ls));
    CK(launch_by_family(L.family, L.scheme, L.pc, dim3(L.n_chunks), dim3(L.threads), L.smem, ls, a, nullptr));
    if (!pl->borrowed) CK(cudaEventRecord(pl->kstop[i], ls));
    if (fork) {
      CK(cudaEventRecord(pl->join[i], ls));
      CK(cudaStreamWaitEvent(st, pl->join[i], 0));
    }
  }
  // items without samples: zero sums (no CTA writes them)
  for (uint32_t o : pl->empty_out) CK(cudaMemsetAsync(pl->d_out + o, 0, sizeof(DevSums), st));
  CK(cudaEventRecord(pl->t1, st));
  pl->last_stream = st;
  pl->launched = true;
  return MLMC_OK;
}

double u128_to_double(uint64_t lo, uint64_t hi) {
  const unsigned __int128 v = ((unsigned __int128)hi << 64) | lo;
  return (double)v;
}

// Per-item results from the undiscounted device sums h (host copy).
void convert_results(const mlmc_plan *pl, const DevSums *h, float ms, mlmc_sums *out) {
  for (int i = 0; i < pl->n_work; ++i) {
    mlmc_sums &o = out[i];
    std::memset(&o, 0, sizeof o);
    const double disc = pl->disc[i];
    o.n = pl->N[i];
    o.seconds = ms * 1e-3;
    o.saturations = h[i].nsat;
    o.unit = pl->unit[i];
    o.exact_int = pl->exact_int[i];
    if (o.exact_int) {
      o.isum = h[i].isum;
      o.isum2_lo = h[i].isum2_lo;
      o.isum2_hi = h[i].isum2_hi;
      o.sum = disc * std::ldexp((double)h[i].isum, -o.unit);
      o.sum2 = disc * disc * std::ldexp(u128_to_double(h[i].isum2_lo, h[i].isum2_hi), -2 * o.unit);
    } else {
      o.sum = disc * h[i].dsum;
      o.sum2 = disc * disc * h[i].dsum2;
    }
  }
}

mlmc_status plan_results_impl(mlmc_plan *pl, mlmc_sums *out) {
  if (!pl->launched) return MLMC_ENOTREADY;
  CK(cudaEventSynchronize(pl->t1));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, pl->t0, pl->t1));
  std::vector<DevSums> h(pl->n_work);
  CK(cudaMemcpy(h.data(), pl->d_out, sizeof(DevSums) * pl->n_work, cudaMemcpyDeviceToHost));
  convert_results(pl, h.data(), ms, out);
  return MLMC_OK;
}

template <class T>
bool grow_pinned(T *&p, size_t &cap, size_t need) {
  if (need <= cap) return true;
  if (p) cudaFreeHost(p);
  p = nullptr;
  cap = 0;
  const size_t n = std::max<size_t>(need, 64);
  if (cudaHostAlloc((void **)&p, sizeof(T) * n, cudaHostAllocDefault) != cudaSuccess) return false;
  cap = n;
  return true;
}

// One synchronous pass on stream st: work list to the device through pinned
// staging, the launch, the sums back through pinned staging, one stream sync.
mlmc_status run_sync(const mlmc_work *work, int n_work, uint64_t seed, const mlmc_tuning *tuning,
                     void *const *dumps, mlmc_sums *out, cudaStream_t st) {
  mlmc_plan *pl = nullptr;
  mlmc_status s = plan_create_impl(&pl, work, n_work, seed, tuning, dumps, &g.arena, true);
  if (s != MLMC_OK) return s;
  Arena &A = g.arena;
  const size_t ni = pl->items.size();
  do {
    if (!grow_pinned(A.h_items, A.cap_h_items, ni) || !grow_pinned(A.h_out, A.cap_h_out, (size_t)n_work)) {
      s = MLMC_ENOMEM;
      break;
    }
    std::memcpy(A.h_items, pl->items.data(), sizeof(ItemDesc) * ni);
    if (cudaMemcpyAsync(pl->d_items, A.h_items, sizeof(ItemDesc) * ni, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      s = MLMC_ECUDA;
      break;
    }
    if ((s = plan_launch_impl(pl, st)) != MLMC_OK) break;
    float ms = 0.0f;
    if (cudaMemcpyAsync(A.h_out, pl->d_out, sizeof(DevSums) * n_work, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaEventElapsedTime(&ms, pl->t0, pl->t1) != cudaSuccess) {
      s = MLMC_ECUDA;
      break;
    }
    convert_results(pl, A.h_out, ms, out);
  } while (0);
  free_plan_device(pl);
  delete pl;
  return s;
}

cudaStream_t ctx_stream() { return g.st; }
std::recursive_mutex &api_mutex() {
  static std::recursive_mutex m;
  return m;
}
int ctx_num_sms() { return g.num_sms; }
double cost_of_variant(int variant) { return g_cost[cost_kind_of(variant)]; }
mlmc_status plan_create_transient(mlmc_plan **out, const mlmc_work *work, int n_work, uint64_t seed,
                                  const mlmc_tuning *tuning) {
  return plan_create_impl(out, work, n_work, seed, tuning, nullptr, &g.arena);
}
mlmc_status plan_launch_on(mlmc_plan *pl, cudaStream_t st) {
  if (st != g.st) {
    // a transient plan's work list was copied on the context stream: order after it
    MLMC_CK(cudaEventRecord(g.arena.fork, g.st));
    MLMC_CK(cudaStreamWaitEvent(st, g.arena.fork, 0));
  }
  return plan_launch_impl(pl, st);
}
const mlmc::DevSums *plan_out_device(const mlmc_plan *pl) { return pl->d_out; }
void plan_item_scale(const mlmc_plan *pl, int i, double *disc, int *unit, int *exact_int) {
  *disc = pl->disc[i];
  *unit = pl->unit[i];
  *exact_int = pl->exact_int[i];
}
void plan_release(mlmc_plan *pl) {
  free_plan_device(pl);
  delete pl;
}

// Median device time (ms) of `reps` launches of a plan of `work` (launch
// shapes from the tuning table), after one untimed launch.
mlmc_status time_plan(const mlmc_work *work, int n_work, uint64_t seed, int reps, double *ms) {
  mlmc_plan *pl = nullptr;
  mlmc_status s = plan_create_impl(&pl, work, n_work, seed, nullptr, nullptr);
  if (s != MLMC_OK) return s;
  std::vector<float> v;
  for (int r = 0; r <= reps && s == MLMC_OK; ++r) {
    s = plan_launch_impl(pl, g.st);
    float x = 0.0f;
    if (s == MLMC_OK && (cudaEventSynchronize(pl->t1) != cudaSuccess ||
                         cudaEventElapsedTime(&x, pl->t0, pl->t1) != cudaSuccess))
      s = MLMC_ECUDA;
    if (r > 0) v.push_back(x);
  }
  free_plan_device(pl);
  delete pl;
  if (s != MLMC_OK) return s;
  std::sort(v.begin(), v.end());
  *ms = v[v.size() / 2];
  return MLMC_OK;
}

}  // namespace mlmc_host

using namespace mlmc_host;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

mlmc_status mlmc_level(int level, uint64_t N, const mlmc_params *p, mlmc_variant v, uint64_t seed,
                       uint64_t first_sample, mlmc_sums *out) {
  MLMC_API_LOCK();
  if (!out) return MLMC_EINVAL;
  mlmc_work w;
  std::memset(&w, 0, sizeof w);
  w.params = p; w.level = level; w.variant = (int32_t)v; w.first_sample = first_sample; w.N = N; w.stream = -1;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  return run_sync(&w, 1, seed, nullptr, nullptr, out, g.st);
}

mlmc_status mlmc_level_dump(int level, uint64_t N, const mlmc_params *p, mlmc_variant v, uint64_t seed,
                            uint64_t first_sample, int32_t stream, mlmc_sample *d_samples, mlmc_sums *out) {
  MLMC_API_LOCK();
  if (!out || (N > 0 && !d_samples)) return MLMC_EINVAL;
  mlmc_work w;
  std::memset(&w, 0, sizeof w);
  w.params = p; w.level = level; w.variant = (int32_t)v; w.first_sample = first_sample; w.N = N;
  w.stream = stream;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  void *dumps[1] = {d_samples};
  return run_sync(&w, 1, seed, nullptr, dumps, out, g.st);
}

mlmc_status mlmc_plan_create(mlmc_plan **plan, const mlmc_work *work, int n_work, uint64_t seed,
                             const mlmc_tuning *tuning) {
  MLMC_API_LOCK();
  return plan_create_impl(plan, work, n_work, seed, tuning, nullptr);
}

mlmc_status mlmc_plan_launch(mlmc_plan *plan, void *stream) {
  MLMC_API_LOCK();
  if (!plan) return MLMC_EINVAL;
  return plan_launch_impl(plan, (cudaStream_t)stream);
}

mlmc_status mlmc_plan_results(mlmc_plan *plan, mlmc_sums *out) {
  MLMC_API_LOCK();
  if (!plan || !out) return MLMC_EINVAL;
  return plan_results_impl(plan, out);
}

mlmc_status mlmc_plan_info(const mlmc_plan *plan, int *kernels, uint64_t *ctas, uint64_t *path_steps,
                           uint64_t *h2d_bytes, uint64_t *d2h_bytes) {
  if (!plan) return MLMC_EINVAL;
  if (kernels) *kernels = (int)plan->launches.size();
  if (ctas) *ctas = plan->total_chunks;
  if (path_steps) *path_steps = plan->path_steps;
  if (h2d_bytes) *h2d_bytes = sizeof(ItemDesc) * plan->items.size();
  if (d2h_bytes) *d2h_bytes = sizeof(DevSums) * (uint64_t)plan->n_work;
  return MLMC_OK;
}

mlmc_status mlmc_plan_launch_info(const mlmc_plan *plan, int k, int *family, int *items, uint64_t *ctas,
                                  uint64_t *path_steps) {
  if (!plan || k < 0 || k >= (int)plan->launches.size()) return MLMC_EINVAL;
  const LaunchRec &L = plan->launches[k];
  if (family) *family = L.family;
  if (items) *items = L.n_items;
  if (ctas) *ctas = L.n_chunks;
  if (path_steps) {
    uint64_t ps = 0;
    for (int i = 0; i < L.n_items; ++i) {
      const ItemDesc &it = plan->items[L.item_off + i];
      ps += it.N << it.level;
    }
    *path_steps = ps;
  }
  return MLMC_OK;
}

mlmc_status mlmc_plan_kernel_time(const mlmc_plan *plan, int k, int *family, double *ms) {
  if (!plan || k < 0 || k >= (int)plan->launches.size()) return MLMC_EINVAL;
  if (!plan->launched) return MLMC_ENOTREADY;
  if (family) *family = plan->launches[k].family;
  if (ms) {
    CK(cudaEventSynchronize(plan->kstop[k]));
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, plan->kstart[k], plan->kstop[k]));
    *ms = t;
  }
  return MLMC_OK;
}

void mlmc_plan_destroy(mlmc_plan *plan) {
  MLMC_API_LOCK();
  if (!plan) return;
  if (plan->launched) cudaEventSynchronize(plan->t1);
  free_plan_device(plan);
  delete plan;
}

mlmc_status mlmc_autotune(const mlmc_work *work, int n_work, uint64_t seed, int reps, mlmc_tuning *chosen) {
  MLMC_API_LOCK();
  if (!work || n_work <= 0 || reps < 1 || reps > 1000) return MLMC_EINVAL;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  // kernel classes among the items, with their model work
  typedef std::tuple<int, int, int, int> Key;
  std::map<Key, std::vector<int>> cls;
  std::map<Key, double> work_of;
  std::vector<BuiltItem> built(n_work);
  for (int i = 0; i < n_work; ++i) {
    double disc;
    int unit, ei;
    if ((s = build_item(work[i], i, nullptr, built[i], disc, unit, ei)) != MLMC_OK) return s;
    const Key k = std::make_tuple(built[i].family, built[i].scheme, built[i].pc, level_class(work[i].level));
    cls[k].push_back(i);
    work_of[k] += std::ldexp((double)work[i].N, work[i].level) * built[i].cost_step;
  }
  std::vector<Key> order;
  for (auto &kv : cls) order.push_back(kv.first);
  std::stable_sort(order.begin(), order.end(), [&](const Key &a, const Key &b) { return work_of[a] > work_of[b]; });
  static const int cand_threads[] = {128, 96, 64};
  static const int cand_spt[] = {256, 64, 128, 512, 1024, 2048};
  // one pass of coordinate descent: each class in turn takes the shape that
  // makes the whole work list fastest, the other classes keeping theirs
  for (const Key &k : order) {
    const std::vector<int> &ix = cls[k];
    int cur_t, cur_s;
    tuning_for(std::get<0>(k), std::get<1>(k), std::get<2>(k), work[ix[0]].level, &cur_t, &cur_s);
    int best_t = cur_t, best_s = cur_s;
    double best_ms = 0.0;
    if ((s = time_plan(work, n_work, seed, reps, &best_ms)) != MLMC_OK) return s;
    std::vector<std::vector<uint32_t>> seen;   // chunkings already timed
    for (int pass = 0; pass < 2; ++pass)
      for (int th : cand_threads)
        for (int sp : cand_spt) {
          if (pass == 0 && !(th == cur_t && sp == cur_s)) continue;   // the current shape first
          std::vector<uint32_t> sig{(uint32_t)th};
          for (int i : ix) {
            BuiltItem b = built[i];
            if ((s = chunk_built(b, th, sp)) != MLMC_OK) return s;
            sig.push_back(b.it.groups_per_thread);
          }
          if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
          seen.push_back(sig);
          if (pass == 0) continue;
          g_tune[k] = std::make_pair(th, sp);
          double ms = 0.0;
          if ((s = time_plan(work, n_work, seed, reps, &ms)) != MLMC_OK) return s;
          // a candidate must make the work list 2% faster than the best so far
          if (ms < 0.98 * best_ms) {
            best_ms = ms;
            best_t = th;
            best_s = sp;
          }
        }
    g_tune[k] = std::make_pair(best_t, best_s);
    if (chosen)
      for (int i : ix) {
        chosen[i].threads = best_t;
        chosen[i].steps_per_thread = best_s;
      }
  }
  return MLMC_OK;
}

void mlmc_tuning_reset(void) {
  MLMC_API_LOCK();
  g_tune.clear();
}

mlmc_status mlmc_run(const mlmc_work *work, int n_work, uint64_t seed, const mlmc_tuning *tuning,
                     mlmc_sums *out, void *stream) {
  MLMC_API_LOCK();
  if (!out) return MLMC_EINVAL;
  return run_sync(work, n_work, seed, tuning, nullptr, out, (cudaStream_t)stream);
}

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

mlmc_status mlmc_icdf_table(int method, int d, int rep, int fZ, double *out) {
  MLMC_API_LOCK();
  if (method < 1 || method > 3 || d < 2 || d > 14 || rep < 0 || rep > 4 || !out) return MLMC_EINVAL;
  if (rep == REP_FIXED && (fZ < 0 || fZ > 28)) return MLMC_EINVAL;
  if (method == 3 && rep == REP_FP64) return MLMC_EINVAL;
  if (method == 2 && (d % 2 || d < 4)) return MLMC_EINVAL;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  if (method == 2) {
    // the host-built values the device tables are made of
    const M2Table *t;
    if ((s = m2_build(d, &t)) != MLMC_OK) return s;
    for (int j = 0; j < (1 << (d - 1)); ++j) out[j] = m2_value(*t, d, j, rep, fZ);
    return MLMC_OK;
  }
  const void *tab = nullptr;
  if ((s = get_table(method, d, rep, fZ, &tab)) != MLMC_OK) return s;
  const int n = 1 << (d - 1);
  double *dv = nullptr;
  CK(cudaMalloc(&dv, sizeof(double) * n));
  cudaError_t e = launch_table_values(method, d, rep, fZ, tab, dv, g.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dv, sizeof(double) * n, cudaMemcpyDeviceToHost, g.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g.st);
  cudaFree(dv);
  return e == cudaSuccess ? MLMC_OK : MLMC_ECUDA;
}

mlmc_status mlmc_icdf_method2(int d, double *x, uint32_t *perm, int *iterations) {
  MLMC_API_LOCK();
  if (d % 2 || d < 4 || d > 14) return MLMC_EINVAL;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  const M2Table *t;
  if ((s = m2_build(d, &t)) != MLMC_OK) return s;
  if (x) std::memcpy(x, t->x.data(), sizeof(double) * t->x.size());
  if (perm) std::memcpy(perm, t->pi.data(), sizeof(uint32_t) * t->pi.size());
  if (iterations) *iterations = t->iterations;
  return MLMC_OK;
}

mlmc_status mlmc_philox(const uint32_t *ctr, uint64_t n, uint64_t seed, uint32_t *out) {
  MLMC_API_LOCK();
  if ((!ctr || !out) && n) return MLMC_EINVAL;
  if (n == 0) return MLMC_OK;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  RoundKeys rk;
  make_round_keys(seed, rk);
  uint4 *dc = nullptr, *dout = nullptr;
  if (cudaMalloc(&dc, 16 * n) != cudaSuccess) return MLMC_ENOMEM;
  if (cudaMalloc(&dout, 16 * n) != cudaSuccess) { cudaFree(dc); return MLMC_ENOMEM; }
  cudaError_t e = cudaMemcpyAsync(dc, ctr, 16 * n, cudaMemcpyHostToDevice, g.st);
  if (e == cudaSuccess) e = launch_philox(dc, n, rk, dout, g.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, 16 * n, cudaMemcpyDeviceToHost, g.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g.st);
  cudaFree(dc);
  cudaFree(dout);
  return e == cudaSuccess ? MLMC_OK : MLMC_ECUDA;
}

const char *mlmc_strerror(mlmc_status s) {
  switch (s) {
    case MLMC_OK: return "ok";
    case MLMC_EINVAL: return "invalid argument";
    case MLMC_ENOMEM: return "out of memory";
    case MLMC_ECUDA: return "CUDA runtime error or no CUDA device";
    case MLMC_ETIMEOUT: return "timed out";
    case MLMC_EOVERFLOW: return "constant outside its fixed-point format";
    case MLMC_ENOTREADY: return "results requested before launch";
    default: return "unknown status";
  }
}

const char *mlmc_version(void) { return "mlmc-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// adaptive MLMC (Giles 2008 loop; nested variant of Sec. 2.2)
// ---------------------------------------------------------------------------
namespace {

struct EstPlan {
  int n;          // estimators per level
  int variant[2];
  bool exact_low; // approximate terms of levels 0-1 computed exactly by enumeration
};

// Levels whose approximate level difference is a finite sum over 2^(d 2^l) <= 2^20 cells.
constexpr int EXACT_MAX_BITS = 20;

bool est_plan(int mode, EstPlan &e) {
  switch (mode) {
    case 0: e = {1, {MLMC_FP64_EXACT, 0}, false}; return true;
    case 1: e = {1, {MLMC_FP32_EXACT, 0}, false}; return true;
    case 2: e = {2, {MLMC_FIXED_APPROX, MLMC_NESTED_CORR_FIXED}, false}; return true;
    case 3: e = {2, {MLMC_FP16_APPROX, MLMC_NESTED_CORR_FP16}, false}; return true;
    case 4: e = {2, {MLMC_BF16_APPROX, MLMC_NESTED_CORR_BF16}, false}; return true;
    case 5: e = {2, {MLMC_FIXED_APPROX, MLMC_NESTED_CORR_FIXED}, true}; return true;
    case 6: e = {2, {MLMC_FP16_APPROX, MLMC_NESTED_CORR_FP16}, true}; return true;
    default: return false;
  }
}

// N_k = ceil(lambda sqrt(V_k / C_k)), lambda = sum_j sqrt(V_j C_j) / var_target (Sec. 2.1 / 2.2).
void optimal_counts(const std::vector<double> &V, const std::vector<double> &C, double var_target,
                    std::vector<uint64_t> &Nopt) {
  double lam = 0.0;
  for (size_t k = 0; k < V.size(); ++k) lam += std::sqrt(V[k] * C[k]);
  lam /= var_target;
  Nopt.resize(V.size());
  for (size_t k = 0; k < V.size(); ++k) {
    const double x = V[k] > 0.0 ? lam * std::sqrt(V[k] / C[k]) : 0.0;
    Nopt[k] = (uint64_t)std::ceil(std::min(x, 1e18));
  }
}

}  // namespace

extern "C" mlmc_status mlmc_estimate(double eps, const mlmc_params *p, int mode, uint64_t seed, int max_level,
                                     double *price, double *stderr_out, int *Lout, uint64_t *N_l,
                                     int cap_levels) {
  MLMC_API_LOCK();
  EstPlan ep;
  if (!(eps > 0.0) || !std::isfinite(eps) || !params_ok(p) || !est_plan(mode, ep)) return MLMC_EINVAL;
  if (max_level < 2 || max_level > 20 || cap_levels <= max_level || !price || !stderr_out || !Lout || !N_l)
    return MLMC_EINVAL;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  const int ne = ep.n;
  const double theta = 0.5, alpha = 1.0;
  const double beta = p->scheme == MLMC_MILSTEIN ? 2.0 : 1.0;
  const uint64_t N_init = 10000;
  int L = 2;
  std::vector<std::vector<uint64_t>> N(L + 1, std::vector<uint64_t>(ne, 0)), dN(L + 1, std::vector<uint64_t>(ne, N_init));
  std::vector<std::vector<double>> S1(L + 1, std::vector<double>(ne, 0.0)), S2 = S1;
  std::vector<std::vector<double>> Vext(L + 1, std::vector<double>(ne, 0.0));
  auto is_exact = [&](int l, int k) { return ep.exact_low && k == 0 && l <= 1 && (p->icdf_bits << l) <= EXACT_MAX_BITS; };
  for (int l = 0; l <= 1; ++l)
    if (is_exact(l, 0)) dN[l][0] = 1ULL << (p->icdf_bits << l);  // every combination of table cells once
  std::vector<mlmc_work> work;
  std::vector<mlmc_sums> res;
  std::vector<std::pair<int, int>> idx;
  auto level_var = [&](int l, int k) {
    if (is_exact(l, k)) return 0.0;  // an exact mean has no variance
    if (N[l][k] == 0) return Vext[l][k];
    const double m = S1[l][k] / (double)N[l][k];
    return std::max(S2[l][k] / (double)N[l][k] - m * m, 0.0);
  };
  const double beta_factor = std::pow(2.0, beta);
  auto update_dn = [&]() {
    std::vector<double> V, C;
    double vprev[2] = {0.0, 0.0};
    for (int l = 0; l <= L; ++l)
      for (int k = 0; k < ne; ++k) {
        // variance floor V_l >= V_{l-1} / (2 * 2^beta) from level 2 on, so that a level
        // whose few samples show (almost) no variance still receives samples
        double v = level_var(l, k);
        if (l >= 2) v = std::max(v, 0.5 * vprev[k] / beta_factor);
        vprev[k] = v;
        V.push_back(std::max(v, 1e-300));
        C.push_back(std::ldexp(g_cost[cost_kind_of(ep.variant[k])], l));
      }
    std::vector<uint64_t> Nopt;
    optimal_counts(V, C, (1.0 - theta) * eps * eps, Nopt);
    for (int l = 0; l <= L; ++l)
      for (int k = 0; k < ne; ++k) {
        const uint64_t want = Nopt[(size_t)l * ne + k];
        dN[l][k] = want > N[l][k] ? want - N[l][k] : 0;
      }
  };
  for (int iter = 0; iter < 1000; ++iter) {
    bool any = true;
    while (any) {
      work.clear();
      idx.clear();
      for (int l = 0; l <= L; ++l)
        for (int k = 0; k < ne; ++k)
          if (dN[l][k] > 0) {
            mlmc_work w;
            std::memset(&w, 0, sizeof w);
            w.params = p; w.level = l; w.variant = ep.variant[k]; w.first_sample = N[l][k]; w.N = dN[l][k];
            w.stream = -1;
            w.flags = is_exact(l, k) ? MLMC_WORK_ENUMERATE : 0;
            work.push_back(w);
            idx.push_back({l, k});
          }
      if (work.empty()) break;
      res.resize(work.size());
      s = run_sync(work.data(), (int)work.size(), seed, nullptr, nullptr, res.data(), g.st);
      if (s != MLMC_OK) return s;
      for (size_t j = 0; j < work.size(); ++j) {
        const int l = idx[j].first, k = idx[j].second;
        S1[l][k] += res[j].sum;
        S2[l][k] += res[j].sum2;
        N[l][k] += work[j].N;
      }
      update_dn();
      any = false;
      for (int l = 0; l <= L; ++l)
        for (int k = 0; k < ne; ++k) any |= dN[l][k] > 0;
    }
    // bias test on the last two levels (weak order alpha)
    std::vector<double> means(L + 1, 0.0);
    for (int l = 0; l <= L; ++l) {
      for (int k = 0; k < ne; ++k) means[l] += S1[l][k] / (double)N[l][k];
      means[l] = std::fabs(means[l]);
      // the same floor on the level means: |m_l| >= |m_{l-1}| / (2 * 2^alpha)
      if (l >= 2) means[l] = std::max(means[l], 0.5 * means[l - 1] / std::pow(2.0, alpha));
    }
    double rem = std::fabs(means[L]) / (std::pow(2.0, alpha) - 1.0);
    rem = std::max(rem, std::fabs(means[L - 1]) / std::pow(2.0, alpha) / (std::pow(2.0, alpha) - 1.0));
    if (rem <= std::sqrt(theta) * eps || L >= max_level) break;
    L += 1;
    N.push_back(std::vector<uint64_t>(ne, 0));
    dN.push_back(std::vector<uint64_t>(ne, 0));
    S1.push_back(std::vector<double>(ne, 0.0));
    S2.push_back(std::vector<double>(ne, 0.0));
    std::vector<double> ve(ne);
    for (int k = 0; k < ne; ++k) ve[k] = std::max(level_var(L - 1, k), 1e-300) / std::pow(2.0, beta);
    Vext.push_back(ve);
    update_dn();
  }
  double pr = 0.0, var = 0.0;
  for (int l = 0; l <= L; ++l)
    for (int k = 0; k < ne; ++k) {
      pr += S1[l][k] / (double)N[l][k];
      var += level_var(l, k) / (double)N[l][k];
    }
  *price = pr;
  *stderr_out = std::sqrt(var);
  *Lout = L;
  for (int l = 0; l < cap_levels; ++l)
    for (int k = 0; k < 2; ++k) N_l[2 * l + k] = (l <= L && k < ne) ? N[l][k] : 0;
  return MLMC_OK;
}

// ---------------------------------------------------------------------------
// mlmc_level_noalloc: the single-level estimator without any device allocation
// ---------------------------------------------------------------------------
// Everything the launch needs besides the caller's stream lives in one
// file-scope device array: the per-CTA partial sums (the level kernel's
// scratch), the work-item descriptor, the Method-1 table in FP64 and in the
// representation the kernel reads, the Method-3 coefficients and the result
// record.  Each call rebuilds and overwrites all of it, so nothing has to
// start at zero; two calls that overlap on the GPU would overwrite each
// other's data.
namespace {

constexpr uint32_t NOALLOC_MAX_CTAS = 16384;
constexpr int NOALLOC_MAX_D = 14;

struct NoAllocScratch {
  Partial partials[NOALLOC_MAX_CTAS];
  DevSums out;
  ItemDesc item;
  M3Coef m3;
  double z64[1 << (NOALLOC_MAX_D - 1)];
  uint32_t table[1 << NOALLOC_MAX_D];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// Host-side copies used while building the work item (static: no heap use).
constexpr int NOALLOC_MAX_DEVICES = 64;
NoAllocScratch *g_noalloc_dev[NOALLOC_MAX_DEVICES] = {};
double g_noalloc_zhost[1 << (NOALLOC_MAX_D - 1)];

// Device address of the scratch array on the current device (looked up once per device).
mlmc_status noalloc_scratch(NoAllocScratch **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return MLMC_ECUDA;
  if (!g_noalloc_dev[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return MLMC_ECUDA;
    g_noalloc_dev[dev] = (NoAllocScratch *)ptr;
  }
  *out = g_noalloc_dev[dev];
  return MLMC_OK;
}

// Method-3 least-squares lines from a host FP64 table (same fit as m3_fit).
void noalloc_m3_fit(const double *Z, int d, M3Coef &c) {
  std::memset(&c, 0, sizeof c);
  for (int cls = 0; cls < d - 1; ++cls) {
    const int lo = cls == 0 ? 0 : (1 << cls);
    const int hi = cls == 0 ? 1 : (1 << (cls + 1)) - 1;
    const int n = hi - lo + 1;
    double kbar = 0.0, zbar = 0.0;
    for (int k = lo; k <= hi; ++k) { kbar += k; zbar += Z[k]; }
    kbar /= n;
    zbar /= n;
    double sxx = 0.0, sxy = 0.0;
    for (int k = lo; k <= hi; ++k) {
      sxx += (k - kbar) * (k - kbar);
      sxy += (k - kbar) * (Z[k] - zbar);
    }
    const double b = sxy / sxx;
    const double a = zbar - b * kbar;
    c.a[cls] = (float)a;
    c.b[cls] = (float)b;
    c.A[cls] = (int64_t)std::floor(std::ldexp(a, M3_FRAC) + 0.5);
    c.B[cls] = (int64_t)std::floor(std::ldexp(b, M3_FRAC) + 0.5);
  }
}

// Largest |table value| in Z's fixed-point format (as table_zmax_fixed).
int64_t noalloc_zmax(const double *Z, int d, int method, int fZ, const M3Coef &c) {
  int64_t zmax = 0;
  const int half = 1 << (d - 1);
  if (method == 1) {
    for (int k = 0; k < half; ++k)
      zmax = std::max<int64_t>(zmax, std::llabs((int64_t)std::floor(std::ldexp(Z[k], fZ) + 0.5)));
    return zmax;
  }
  const int sh = M3_FRAC - fZ;
  for (int k = 0; k < half; ++k) {
    const int cls = k < 2 ? 0 : 31 - __builtin_clz((unsigned)k);
    const int64_t t = c.A[cls] + c.B[cls] * (int64_t)k;
    zmax = std::max<int64_t>(zmax, std::llabs((t + ((int64_t)1 << (sh - 1))) >> sh));
  }
  return zmax;
}

}  // namespace

extern "C" mlmc_status mlmc_level_noalloc(int level, uint64_t N, const mlmc_params *p, mlmc_variant v,
                                          uint64_t seed, uint64_t first_sample, mlmc_sums *out, void *stream) {
  MLMC_API_LOCK();
  if (!out || !params_ok(p)) return MLMC_EINVAL;
  if (level < 0 || level > 20 || (int)v < 0 || (int)v > 7) return MLMC_EINVAL;
  if (N > (1ULL << 58) || first_sample > (1ULL << (60 - level)) - N) return MLMC_EINVAL;
  if (p->icdf_method == 2) return MLMC_EINVAL;   // its tables are built on the host, with allocation
  const cudaStream_t st = (cudaStream_t)stream;
  NoAllocScratch *S = nullptr;
  mlmc_status s = noalloc_scratch(&S);
  if (s != MLMC_OK) return s;
  int dev = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));

  // the work item, chunked exactly as mlmc_level chunks it
  ItemDesc it;
  std::memset(&it, 0, sizeof it);
  const int vi = (int)v;
  const bool approx = !(vi == MLMC_FP32_EXACT || vi == MLMC_FP64_EXACT);
  const int strm = (vi == MLMC_FIXED_APPROX || vi == MLMC_FP16_APPROX || vi == MLMC_BF16_APPROX) ? 1 : 0;
  it.first = first_sample;
  it.N = N;
  it.level = level;
  it.nlog = level;
  it.payoff = p->payoff;
  it.scheme = p->scheme;
  it.method = p->icdf_method;
  it.d = p->icdf_bits;
  it.ctr2 = (uint32_t)level | ((uint32_t)strm << 8);
  it.ctr3 = p->request_id;
  it.out_index = 0;
  it.dump = nullptr;
  const int KP = pack_lanes(p, vi);
  if (KP == 0) return MLMC_EINVAL;
  const uint64_t spc = samples_per_group(level, KP);
  it.g0 = first_sample / spc;
  it.g1 = N == 0 ? it.g0 : (first_sample + N + spc - 1) / spc;
  const uint64_t groups = it.g1 - it.g0;
  it.gf0 = (first_sample + spc - 1) / spc;
  it.gf1 = (first_sample + N) / spc;
  if (it.gf1 < it.gf0) it.gf1 = it.gf0;
  const double h = std::ldexp(p->T, -level);
  const double rh = p->r * h, rh2 = p->r * (2.0 * h), sqh = std::sqrt(h);
  const double c2 = p->sigma * sqh, c3 = 0.5 * p->sigma * p->sigma * h;
  it.c1d = rh; it.c2d = c2; it.c1cd = rh2; it.c3d = c3; it.S0d = p->S0; it.Kd = p->K;
  it.c1f = (float)rh; it.c2f = (float)c2; it.c1cf = (float)rh2; it.c3f = (float)c3;
  it.S0f = (float)p->S0; it.Kf = (float)p->K;
  const double disc = std::exp(-p->r * p->T);
  int unit = 0, exact_int = 0, family = family_of(vi);
  size_t smem = 0;
  if (approx) {
    const bool fixed = (vi == MLMC_FIXED_APPROX || vi == MLMC_NESTED_CORR_FIXED);
    const bool bf = (vi == MLMC_BF16_APPROX || vi == MLMC_NESTED_CORR_BF16);
    const int rep = fixed ? REP_FIXED : (bf ? REP_BF16 : REP_FP16);
    const int d = p->icdf_bits;
    // Method-1 table in FP64 on the device, and a host copy for the bounds and the Method-3 fit
    CK(launch_m1_table(d, S->z64, st));
    CK(cudaMemcpyAsync(g_noalloc_zhost, S->z64, sizeof(double) << (d - 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    M3Coef m3;
    noalloc_m3_fit(g_noalloc_zhost, d, m3);
    int fZ = 0;
    bool fast = false, fast64 = false;
    if (fixed) {
      mlmc_format F;
      if (p->formats && level < p->n_formats) F = p->formats[level];
      else if (p->formats) return MLMC_EINVAL;
      else default_format(p, level, &F);
      if (!format_ok_gpu(F, p->scheme == MLMC_MILSTEIN, d)) return MLMC_EINVAL;
      int e[7], f[7];
      for (int i = 0; i < 7; ++i) { e[i] = F.e[i]; f[i] = F.f[i]; }
      fZ = f[F_Z];
      FixedConsts &fx = it.fx;
      int64_t con1, con1c, con2, con3, S0q, Kq;
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
      const int64_t zmax = noalloc_zmax(g_noalloc_zhost, d, p->icdf_method, fZ, m3);
      if ((double)zmax > std::ldexp(1.0, e[F_Z] + fZ) - 1.0) return MLMC_EOVERFLOW;
      unit = f[F_S] + (p->payoff == MLMC_ASIAN ? level + 1 : 0);
      fast = fast_fixed(e, f, con1, con1c, con2, con3, zmax, p->scheme == MLMC_MILSTEIN, it.ff, fast64);
      if (fast && !fast64) {
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
    if (p->icdf_method == 1) {
      CK(launch_m1_signed(S->z64, d, rep, fZ, S->table, st));
      it.ztab = S->table;
      smem = (size_t)(1 << d) * (fixed ? 4 : 2);
    } else {
      CK(cudaMemcpyAsync(&S->m3, &m3, sizeof(M3Coef), cudaMemcpyHostToDevice, st));
      it.ztab = &S->m3;
      smem = sizeof(M3Coef);
    }
    exact_int = (vi == MLMC_FIXED_APPROX || vi == MLMC_FP16_APPROX || vi == MLMC_BF16_APPROX) ? 1 : 0;
    if (fast) {
      if (family == 2) family = fast64 ? 9 : 8;
      else if (family == 5) family = fast64 ? 11 : 10;
    }
    if (KP == 3) {
      switch (family) {
        case 2: family = 12; break;
        case 3: family = 13; break;
        case 4: family = 14; break;
        case 8: family = 15; break;
        case 9: family = 16; break;
        default: return MLMC_EINVAL;
      }
    }
  }
  it.unit = unit;
  it.unit_scale = std::ldexp(1.0f, -unit);
  const int pc = p->payoff == MLMC_ASIAN ? PC_ASIAN : (p->payoff == MLMC_LOOKBACK ? PC_LOOKBACK : PC_TERMINAL);
  int threads, spt;
  tuning_for(family, p->scheme, pc, level, &threads, &spt);
  uint32_t gpt = 1;
  const uint64_t nch = chunk_count(groups, steps_per_group(level), KP, threads, spt, nsm, &gpt);
  if (nch > NOALLOC_MAX_CTAS) return MLMC_EINVAL;  // beyond the scratch array's CTA capacity
  it.groups_per_thread = gpt;
  it.n_chunks = (uint32_t)nch;
  it.chunk_begin = 0;
  CK(cudaMemcpyAsync(&S->item, &it, sizeof(ItemDesc), cudaMemcpyHostToDevice, st));
  LaunchArgs a;
  a.items = &S->item;
  a.n_items = 1;
  a.chunk0 = 0;
  a.dyn = nullptr;
  a.counters = nullptr;
  a.out = nullptr;
  a.partials = S->partials;
  make_round_keys(seed, a.rk);
  if (it.n_chunks > 0) CK(launch_by_family(family, p->scheme, pc, dim3(it.n_chunks), dim3(threads), smem, st, a, nullptr));
  finalize_kernel<<<1, 32, 0, st>>>(&S->item, 1, S->partials, &S->out);
  CK(cudaGetLastError());
  DevSums res;
  CK(cudaMemcpyAsync(&res, &S->out, sizeof(DevSums), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::memset(out, 0, sizeof *out);
  out->n = N;
  out->seconds = 0.0;
  out->saturations = res.nsat;
  out->unit = unit;
  out->exact_int = exact_int;
  if (exact_int) {
    out->isum = res.isum;
    out->isum2_lo = res.isum2_lo;
    out->isum2_hi = res.isum2_hi;
    out->sum = disc * std::ldexp((double)res.isum, -unit);
    out->sum2 = disc * disc * std::ldexp(u128_to_double(res.isum2_lo, res.isum2_hi), -2 * unit);
  } else {
    out->sum = disc * res.dsum;
    out->sum2 = disc * disc * res.dsum2;
  }
  return MLMC_OK;
}
