// mlmc_level_noalloc: the single-level estimator of mlmc_level without any
// device allocation.
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

using namespace mlmc_host;

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
  MLMC_CK(cudaGetDevice(&dev));
  MLMC_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));

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
    MLMC_CK(launch_m1_table(d, S->z64, st));
    MLMC_CK(cudaMemcpyAsync(g_noalloc_zhost, S->z64, sizeof(double) << (d - 1), cudaMemcpyDeviceToHost, st));
    MLMC_CK(cudaStreamSynchronize(st));
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
      fast = fast_fixed(e, f, con1, con1c, con2, con3, zmax, p->scheme == MLMC_MILSTEIN, (int64_t)1 << level, it.ff,
                        fast64);
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
      MLMC_CK(launch_m1_signed(S->z64, d, rep, fZ, S->table, st));
      it.ztab = S->table;
      smem = (size_t)(1 << d) * (fixed ? 4 : 2);
    } else {
      MLMC_CK(cudaMemcpyAsync(&S->m3, &m3, sizeof(M3Coef), cudaMemcpyHostToDevice, st));
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
  MLMC_CK(cudaMemcpyAsync(&S->item, &it, sizeof(ItemDesc), cudaMemcpyHostToDevice, st));
  LaunchArgs a;
  a.items = &S->item;
  a.n_items = 1;
  a.chunk0 = 0;
  a.dyn = nullptr;
  a.counters = nullptr;
  a.dump = 0;
  a.out = nullptr;
  a.partials = S->partials;
  make_round_keys(seed, a.rk);
  if (it.n_chunks > 0) MLMC_CK(launch_by_family(family, p->scheme, pc, dim3(it.n_chunks), dim3(threads), smem, st, a, nullptr));
  finalize_kernel<<<1, 32, 0, st>>>(&S->item, 1, S->partials, &S->out);
  MLMC_CK(cudaGetLastError());
  DevSums res;
  MLMC_CK(cudaMemcpyAsync(&res, &S->out, sizeof(DevSums), cudaMemcpyDeviceToHost, st));
  MLMC_CK(cudaStreamSynchronize(st));
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
