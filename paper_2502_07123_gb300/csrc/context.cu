// Device context of the C ABI (device, SM count, internal stream, reusable
// buffers), the process-wide lock, and the approximate-Normal tables: Method 1
// (Sec. 3.1) in FP64 and in each representation, the Method-3 line fit
// (Sec. 3.3), and the Method-2 small table with its interval ranks (Sec. 3.2);
// the table, generator and version entry points.
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

Ctx g;


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
    item_cache_clear();
  }
  MLMC_CK(cudaDeviceGetAttribute(&g.num_sms, cudaDevAttrMultiProcessorCount, dev));
  MLMC_CK(cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking));
  g.device = dev;
  g.inited = true;
  return MLMC_OK;
}

mlmc_status m1_table(int d, double **dev, const std::vector<double> **host) {
  auto it = g.m1_dev.find(d);
  if (it == g.m1_dev.end()) {
    const int n = 1 << (d - 1);
    double *p = nullptr;
    MLMC_CK(cudaMalloc(&p, sizeof(double) * n));
    MLMC_CK(launch_m1_table(d, p, g.st));
    std::vector<double> h(n);
    MLMC_CK(cudaMemcpyAsync(h.data(), p, sizeof(double) * n, cudaMemcpyDeviceToHost, g.st));
    MLMC_CK(cudaStreamSynchronize(g.st));
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
void m3_fit_fp64(const double *Z, int d, double *a, double *b) {
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
    b[cls] = sxy / sxx;
    a[cls] = zbar - b[cls] * kbar;
  }
}

void m3_fit(const double *Z, int d, M3Coef &c) {
  std::memset(&c, 0, sizeof c);
  double a[16], b[16];
  m3_fit_fp64(Z, d, a, b);
  for (int cls = 0; cls < d - 1; ++cls) {
    c.a[cls] = (float)a[cls];
    c.b[cls] = (float)b[cls];
    c.A[cls] = (int64_t)std::floor(std::ldexp(a[cls], M3_FRAC) + 0.5);
    c.B[cls] = (int64_t)std::floor(std::ldexp(b[cls], M3_FRAC) + 0.5);
  }
}

uint16_t half_bits(double x) { return __half_as_ushort(__double2half(x)); }
uint16_t bf16_bits(double x) { return __bfloat16_as_ushort(__double2bfloat16(x)); }

// Method 2 (Sec. 3.2) with n fields: the d-bit index j splits into n fields
// of b = d/n bits (top bits first); each gives +-x_k from a small table of
// 2^(b-1) values (Method-1 sign rule per field) and Z~_j is their sum, formed
// as sum_k c_k x_k over the nonzero net counts c_k of +x_k minus -x_k in
// ascending k (fields holding the same values in another order, or a
// cancelling pair, then give the identical FP64 sum).  The small table starts
// as the b-bit Method-1 table / sqrt(n); then the 2^d sums are ranked
// ascending (ties by j), pi(j) = rank, and x is refitted by least squares
// (normal equations, Cholesky in long double) to the d-bit Method-1 values
// Z_{pi(j)}, until pi equals the previous or any earlier permutation (for
// n > 2 the iteration can alternate between two for ever), at most 1000 fits.
std::map<std::pair<int, int>, M2Table> g_m2;

bool m2_shape_ok(int d, int n) { return n >= 2 && d <= 14 && d % n == 0 && d / n >= 2; }

// Net count c_k of every index j (row-major, 2^d rows of 2^(b-1)).
std::vector<int8_t> m2_counts(int d, int n) {
  const int b = d / n, full = 1 << b, half = 1 << (b - 1), N = 1 << d;
  std::vector<int8_t> c((size_t)N * half, 0);
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < n; ++i) {
      const int f = (j >> (b * (n - 1 - i))) & (full - 1);
      if (f < half) ++c[(size_t)j * half + f];
      else --c[(size_t)j * half + (full - 1 - f)];
    }
  return c;
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

mlmc_status m2_build(int d, int n, const M2Table **out) {
  auto it = g_m2.find(std::make_pair(d, n));
  if (it != g_m2.end()) { *out = &it->second; return MLMC_OK; }
  if (!m2_shape_ok(d, n)) return MLMC_EINVAL;
  const int b = d / n, k = 1 << (b - 1), N = 1 << d;
  double *dv;
  const std::vector<double> *zb = nullptr, *zd = nullptr;
  mlmc_status s;
  if ((s = m1_table(b, &dv, &zb)) != MLMC_OK) return s;
  if ((s = m1_table(d, &dv, &zd)) != MLMC_OK) return s;
  std::vector<double> T(N);
  for (int j = 0; j < N; ++j) T[j] = j < N / 2 ? (*zd)[j] : -(*zd)[N - 1 - j];
  M2Table t;
  t.n = n;
  t.c = m2_counts(d, n);
  const int8_t *C = t.c.data();
  // normal matrix A^T A (row j of A holds the net counts)
  std::vector<long double> M((size_t)k * k, 0.0L);
  for (int j = 0; j < N; ++j)
    for (int a = 0; a < k; ++a) {
      const int ca = C[(size_t)j * k + a];
      if (!ca) continue;
      for (int q = 0; q < k; ++q) M[(size_t)a * k + q] += (long double)(ca * C[(size_t)j * k + q]);
    }
  t.x.resize(k);
  for (int q = 0; q < k; ++q) t.x[q] = (*zb)[q] / std::sqrt((double)n);
  auto sums = [&](const std::vector<double> &x, std::vector<double> &v) {
    v.resize(N);
    for (int j = 0; j < N; ++j) {
      double acc = 0.0;
      for (int q = 0; q < k; ++q) {
        const int cq = C[(size_t)j * k + q];
        if (cq) acc = acc + (double)cq * x[q];
      }
      v[j] = acc;
    }
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
  std::vector<std::vector<uint32_t>> seen{t.pi};
  for (t.iterations = 0; t.iterations < 1000;) {
    std::vector<long double> rhs(k, 0.0L);
    for (int j = 0; j < N; ++j) {
      const long double y = T[t.pi[j]];
      for (int q = 0; q < k; ++q) {
        const int cq = C[(size_t)j * k + q];
        if (cq) rhs[q] += cq * y;
      }
    }
    if (!chol_solve(M, rhs, k, t.x)) return MLMC_EINVAL;
    ++t.iterations;
    sums(t.x, t.values);
    rank(t.values, t.pi);
    if (std::find(seen.begin(), seen.end(), t.pi) != seen.end()) break;   // converged or cycling
    seen.push_back(t.pi);
  }
  auto ins = g_m2.emplace(std::make_pair(d, n), std::move(t));
  *out = &ins.first->second;
  return MLMC_OK;
}

// Method-2 value of index j in a representation: each small-table value
// rounded once, then sum_k c_k x_k over the nonzero net counts in ascending k,
// exactly in fixed point and otherwise with one rounding per product and per
// addition.
double m2_value(const M2Table &t, int d, int j, int rep, int fZ) {
  const int k = 1 << (d / t.n - 1);
  const int8_t *C = t.c.data() + (size_t)j * k;
  auto rnd = [&](double v) -> double {
    switch (rep) {
      case REP_FP16: return (double)__half2float(__double2half(v));
      case REP_BF16: return (double)__bfloat162float(__double2bfloat16(v));
      case REP_FP32: return (double)(float)v;
      default: return v;
    }
  };
  if (rep == REP_FIXED) {
    int64_t acc = 0;
    for (int q = 0; q < k; ++q)
      if (C[q]) acc += (int64_t)C[q] * (int64_t)std::floor(std::ldexp(t.x[q], fZ) + 0.5);
    return std::ldexp((double)acc, -fZ);
  }
  if (rep != REP_FP16 && rep != REP_BF16 && rep != REP_FP32) return t.values[j];
  double acc = 0.0;
  for (int q = 0; q < k; ++q)
    if (C[q]) acc = rnd(acc + rnd((double)C[q] * rnd(t.x[q])));
  return acc;
}

// Device copy of the Method-2 interval ranks of (d, n).
mlmc_status m2_perm_device(int d, int n, const uint16_t **out) {
  auto it = g.m2_perm.find(std::make_pair(d, n));
  if (it != g.m2_perm.end()) { *out = it->second; return MLMC_OK; }
  const M2Table *t;
  mlmc_status s = m2_build(d, n, &t);
  if (s != MLMC_OK) return s;
  std::vector<uint16_t> h(1 << d);
  for (int j = 0; j < (1 << d); ++j) h[j] = (uint16_t)t->pi[j];
  uint16_t *p = nullptr;
  MLMC_CK(cudaMalloc(&p, sizeof(uint16_t) * h.size()));
  MLMC_CK(cudaMemcpy(p, h.data(), sizeof(uint16_t) * h.size(), cudaMemcpyHostToDevice));
  g.m2_perm[std::make_pair(d, n)] = p;
  *out = p;
  return MLMC_OK;
}

// Device table of one representation.  full_signed (method 1 only): all 2^d
// entries indexed directly by j, as the level kernels use it; otherwise the
// 2^(d-1) entries of the lower half (parity checks).  Method 2 (always the
// full signed table) takes its field count n from fields.
mlmc_status get_table(int method, int d, int rep, int fZ, const void **out, bool full_signed, int fields) {
  if (rep != REP_FIXED) fZ = 0;
  if (method == 3) full_signed = false;
  if (method != 2) fields = 0;
  auto key = std::make_tuple(method, d, rep, fZ, full_signed ? 1 : 0, fields);
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
    if ((s = m2_build(d, fields, &t)) != MLMC_OK) return s;
    if (rep == REP_FIXED) {
      std::vector<int32_t> h(2 * n);
      for (int j = 0; j < 2 * n; ++j) h[j] = (int32_t)std::llround(std::ldexp(m2_value(*t, d, j, rep, fZ), fZ));
      MLMC_CK(cudaMalloc(&p, sizeof(int32_t) * h.size()));
      MLMC_CK(cudaMemcpy(p, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice));
    } else if (rep == REP_FP16 || rep == REP_BF16) {
      std::vector<uint16_t> h(2 * n);
      for (int j = 0; j < 2 * n; ++j) {
        const double v = m2_value(*t, d, j, rep, fZ);
        h[j] = rep == REP_FP16 ? half_bits(v) : bf16_bits(v);
      }
      MLMC_CK(cudaMalloc(&p, sizeof(uint16_t) * h.size()));
      MLMC_CK(cudaMemcpy(p, h.data(), sizeof(uint16_t) * h.size(), cudaMemcpyHostToDevice));
    } else {
      return MLMC_EINVAL;
    }
  } else if (method == 1 && full_signed) {
    const size_t es = (rep == REP_FP16 || rep == REP_BF16) ? 2 : 4;
    MLMC_CK(cudaMalloc(&p, es * 2 * n));
    MLMC_CK(launch_m1_signed(z64, d, rep, fZ, p, g.st));
    MLMC_CK(cudaStreamSynchronize(g.st));
  } else if (method == 1) {
    if (rep == REP_FP64) {
      p = z64;
    } else {
      const size_t es = (rep == REP_FP16 || rep == REP_BF16) ? 2 : 4;
      MLMC_CK(cudaMalloc(&p, es * n));
      MLMC_CK(launch_m1_convert(z64, n, rep, fZ, p, g.st));
      MLMC_CK(cudaStreamSynchronize(g.st));
    }
  } else {
    M3Coef c;
    m3_fit(zh->data(), d, c);
    MLMC_CK(cudaMalloc(&p, sizeof(M3Coef)));
    MLMC_CK(cudaMemcpy(p, &c, sizeof(M3Coef), cudaMemcpyHostToDevice));
  }
  g.tables[key] = p;
  *out = p;
  return MLMC_OK;
}

// Tables of the device context (cached per process, allocated on first use).
struct CtxTables final : TableSource {
  int num_sms() const override { return g.num_sms; }
  mlmc_status zmax_fixed(int method, int d, int fZ, int fields, int64_t *out) override {
    double *z64 = nullptr;
    const std::vector<double> *zh = nullptr;
    mlmc_status s = m1_table(d, &z64, &zh);
    if (s != MLMC_OK) return s;
    *out = table_zmax_fixed(zh->data(), d, method, fZ, fields);
    return MLMC_OK;
  }
  mlmc_status device_table(int method, int d, int rep, int fZ, int fields, const void **out) override {
    return get_table(method, d, rep, fZ, out, true, fields);
  }
  mlmc_status m2_perm(int d, int fields, const uint16_t **out) override { return m2_perm_device(d, fields, out); }
};

TableSource &ctx_tables() {
  static CtxTables t;
  return t;
}

cudaStream_t ctx_stream() { return g.st; }
std::recursive_mutex &api_mutex() {
  static std::recursive_mutex m;
  return m;
}
int ctx_num_sms() { return g.num_sms; }

}  // namespace mlmc_host

using namespace mlmc_host;

extern "C" {

mlmc_status mlmc_icdf_table(int method, int d, int rep, int fZ, double *out) {
  MLMC_API_LOCK();
  if (method < 1 || method > 3 || d < 2 || d > 14 || rep < 0 || rep > 4 || !out) return MLMC_EINVAL;
  if (rep == REP_FIXED && (fZ < 0 || fZ > 28)) return MLMC_EINVAL;
  if (method == 3 && rep == REP_FP64) return MLMC_EINVAL;
  if (method == 2) return mlmc_icdf_method2_table(d, 2, rep, fZ, out);
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  const void *tab = nullptr;
  if ((s = get_table(method, d, rep, fZ, &tab)) != MLMC_OK) return s;
  const int n = 1 << (d - 1);
  double *dv = nullptr;
  MLMC_CK(cudaMalloc(&dv, sizeof(double) * n));
  cudaError_t e = launch_table_values(method, d, rep, fZ, tab, dv, g.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dv, sizeof(double) * n, cudaMemcpyDeviceToHost, g.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g.st);
  cudaFree(dv);
  return e == cudaSuccess ? MLMC_OK : MLMC_ECUDA;
}

mlmc_status mlmc_icdf_mse(int method, int d, int fields, double *out) {
  MLMC_API_LOCK();
  if (!out || method < 1 || method > 3 || d < 2 || d > 14) return MLMC_EINVAL;
  if (method != 2 && fields != 0) return MLMC_EINVAL;
  if (method == 2 && fields == 0) fields = 2;
  if (method == 2 && !m2_shape_ok(d, fields)) return MLMC_EINVAL;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  double *z64 = nullptr;
  const std::vector<double> *zh = nullptr;
  if ((s = m1_table(d, &z64, &zh)) != MLMC_OK) return s;
  const double *Z = zh->data();
  const int half = 1 << (d - 1);
  // Method 1: Z~ is the mean of Phi^{-1} over its interval, so the cross term
  // cancels and E[(Z - Z~)^2] = E[Z^2] - E[Z~^2] = 1 - 2^(1-d) sum_k Z_k^2
  double s2 = 0.0;
  for (int k = 0; k < half; ++k) s2 += Z[k] * Z[k];
  const double mse1 = 1.0 - std::ldexp(s2, 1 - d);
  if (method == 1) {
    *out = mse1;
    return MLMC_OK;
  }
  // any other value v_j on interval j adds its distance from the interval mean
  // (eq. mse_dyadic): MSE = MSE_1 + 2^-d sum_j (Z_j - v_j)^2 over all 2^d intervals
  double extra = 0.0;
  if (method == 3) {
    double a[16], b[16];
    m3_fit_fp64(Z, d, a, b);
    for (int k = 0; k < half; ++k) {
      const int cls = k < 2 ? 0 : 31 - __builtin_clz((unsigned)k);
      const double dv = a[cls] + b[cls] * (double)k - Z[k];
      extra += dv * dv;
    }
    *out = mse1 + std::ldexp(extra, 1 - d);   // both halves, by symmetry
    return MLMC_OK;
  }
  // Method 2: U is drawn in interval pi(j), whose mean is the d-bit Method-1 value Z_pi(j)
  const M2Table *t;
  if ((s = m2_build(d, fields, &t)) != MLMC_OK) return s;
  for (int j = 0; j < 2 * half; ++j) {
    const int q = (int)t->pi[j];
    const double zq = q < half ? Z[q] : -Z[2 * half - 1 - q];
    const double dv = zq - t->values[j];
    extra += dv * dv;
  }
  *out = mse1 + std::ldexp(extra, -d);
  return MLMC_OK;
}

mlmc_status mlmc_icdf_method2_table(int d, int n, int rep, int fZ, double *out) {
  MLMC_API_LOCK();
  if (n == 0) n = 2;
  if (!m2_shape_ok(d, n) || rep < 0 || rep > 4 || !out) return MLMC_EINVAL;
  if (rep == REP_FIXED && (fZ < 0 || fZ > 28)) return MLMC_EINVAL;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  // the host-built values the device tables are made of
  const M2Table *t;
  if ((s = m2_build(d, n, &t)) != MLMC_OK) return s;
  for (int j = 0; j < (1 << (d - 1)); ++j) out[j] = m2_value(*t, d, j, rep, fZ);
  return MLMC_OK;
}

mlmc_status mlmc_icdf_method2(int d, int n, double *x, uint32_t *perm, int *iterations) {
  MLMC_API_LOCK();
  if (n == 0) n = 2;
  if (!m2_shape_ok(d, n)) return MLMC_EINVAL;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  const M2Table *t;
  if ((s = m2_build(d, n, &t)) != MLMC_OK) return s;
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
