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
// record.  Each call writes every part it reads (every CTA writes its own
// partial, the finalize kernel the result), so nothing has to start at zero;
// two calls that overlapped on the GPU would overwrite each other's data.
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

// Host copies of the FP64 Method-1 tables (static: no heap use), filled by the
// first call for each d from the table the device builds; they serve the
// fixed-point bound and the Method-3 fit of later calls.  The values depend on
// d only (the same kernel builds them on every device).
double g_noalloc_zhost[NOALLOC_MAX_D + 1][1 << (NOALLOC_MAX_D - 1)];
bool g_noalloc_zhost_ok[NOALLOC_MAX_D + 1] = {};
M3Coef g_noalloc_m3;    // staging of the Method-3 coefficients for their copy

// Device address of the scratch array on the current device, looked up on
// every call (a context reset would leave a stored address stale).
mlmc_status noalloc_scratch(NoAllocScratch **out) {
  void *ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return MLMC_ECUDA;
  *out = (NoAllocScratch *)ptr;
  return MLMC_OK;
}

// The tables of one call, in the scratch array, on the caller's stream.
struct NoAllocTables final : TableSource {
  NoAllocScratch *S;
  cudaStream_t st;
  int nsm;
  int z64_d = 0;    // d of the FP64 table this call has put in S->z64 (0: none yet)
  NoAllocTables(NoAllocScratch *s, cudaStream_t t, int n) : S(s), st(t), nsm(n) {}
  int num_sms() const override { return nsm; }
  // the FP64 table of d in S->z64 (enqueued) and its host copy
  mlmc_status fp64_table(int d, const double **host) {
    if (d < 2 || d > NOALLOC_MAX_D) return MLMC_EINVAL;
    if (z64_d != d) {
      MLMC_CK(launch_m1_table(d, S->z64, st));
      z64_d = d;
    }
    if (!g_noalloc_zhost_ok[d]) {
      MLMC_CK(cudaMemcpyAsync(g_noalloc_zhost[d], S->z64, sizeof(double) << (d - 1), cudaMemcpyDeviceToHost, st));
      MLMC_CK(cudaStreamSynchronize(st));
      g_noalloc_zhost_ok[d] = true;
    }
    *host = g_noalloc_zhost[d];
    return MLMC_OK;
  }
  mlmc_status zmax_fixed(int method, int d, int fZ, int fields, int64_t *out) override {
    if (method == 2) return MLMC_EINVAL;
    const double *z = nullptr;
    mlmc_status s = fp64_table(d, &z);
    if (s != MLMC_OK) return s;
    *out = table_zmax_fixed(z, d, method, fZ, fields);
    return MLMC_OK;
  }
  mlmc_status device_table(int method, int d, int rep, int fZ, int fields, const void **out) override {
    (void)fields;
    if (method == 2) return MLMC_EINVAL;
    const double *z = nullptr;
    mlmc_status s = fp64_table(d, &z);
    if (s != MLMC_OK) return s;
    if (method == 1) {
      MLMC_CK(launch_m1_signed(S->z64, d, rep, rep == REP_FIXED ? fZ : 0, S->table, st));
      *out = S->table;
      return MLMC_OK;
    }
    m3_fit(z, d, g_noalloc_m3);
    MLMC_CK(cudaMemcpyAsync(&S->m3, &g_noalloc_m3, sizeof(M3Coef), cudaMemcpyHostToDevice, st));
    *out = &S->m3;
    return MLMC_OK;
  }
  mlmc_status m2_perm(int, int, const uint16_t **) override { return MLMC_EINVAL; }
};

}  // namespace

extern "C" mlmc_status mlmc_level_noalloc(int level, uint64_t N, const mlmc_params *p, mlmc_variant v,
                                          uint64_t seed, uint64_t first_sample, mlmc_sums *out, void *stream) {
  MLMC_API_LOCK();
  if (!out || !params_ok(p)) return MLMC_EINVAL;
  if (p->icdf_method == 2) return MLMC_EINVAL;   // its tables are built on the host, with allocation
  const cudaStream_t st = (cudaStream_t)stream;
  NoAllocScratch *S = nullptr;
  mlmc_status s = noalloc_scratch(&S);
  if (s != MLMC_OK) return s;
  int dev = 0, nsm = 0;
  MLMC_CK(cudaGetDevice(&dev));
  MLMC_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));

  // the work item, built and chunked by the same code as mlmc_level's
  mlmc_work w;
  std::memset(&w, 0, sizeof w);
  w.params = p;
  w.level = level;
  w.variant = (int32_t)v;
  w.first_sample = first_sample;
  w.N = N;
  w.stream = -1;
  w.flags = 0;
  NoAllocTables src(S, st, nsm);
  BuiltItem b;
  double disc = 1.0;
  int unit = 0, exact_int = 0;
  if ((s = build_item(w, 0, nullptr, b, disc, unit, exact_int, src)) != MLMC_OK) return s;
  int threads, spt;
  tuning_for(b.family, b.scheme, b.pc, level, &threads, &spt);
  if ((s = chunk_built(b, threads, spt, nsm)) != MLMC_OK) return s;
  if (b.it.n_chunks > NOALLOC_MAX_CTAS) return MLMC_EINVAL;  // beyond the scratch array's CTA capacity
  b.it.chunk_begin = 0;
  MLMC_CK(cudaMemcpyAsync(&S->item, &b.it, sizeof(ItemDesc), cudaMemcpyHostToDevice, st));
  LaunchArgs a;
  std::memset(&a, 0, sizeof a);
  a.items = &S->item;
  a.n_items = 1;
  a.chunk0 = 0;
  a.dyn = nullptr;
  a.counters = nullptr;
  a.dump = 0;
  a.out = nullptr;
  a.partials = S->partials;
  make_round_keys(seed, a.rk);
  if (b.it.n_chunks > 0)
    MLMC_CK(launch_by_family(b.family, b.scheme, b.pc, dim3(b.it.n_chunks), dim3(threads), b.smem, st, a, nullptr));
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
