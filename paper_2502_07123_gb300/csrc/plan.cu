// Plans: device work lists chunked into CTAs and launched as one level kernel
// per kernel class on forked streams (no host synchronisation), their results,
// the synchronous entry points (mlmc_level, mlmc_level_dump, mlmc_run), the
// plan entry points and the launch-shape autotuner.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <cmath>
#include <cstdint>
#include <cstddef>
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
  bool dump;                // an item writes per-sample records
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
  bool out_on_host = false;  // d_out is the device address of mapped pinned host memory
};

namespace mlmc_host {

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

// A cached single-launch plan's synchronous pass as one CUDA graph (the
// work-list copy from pinned staging, the timing events and the kernel),
// replayed while the buffers and round keys it was captured with stay the same.
struct ReplayGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void *bufs[6] = {};   // d_items, d_partials, d_out, d_counters, h_items, and t0 (events)
  const void *t1 = nullptr;
  RoundKeys rk{};
  int device = -1;
  bool failed = false;        // a capture failed: this plan keeps the direct path
  ~ReplayGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

// Host part of a plan, as mlmc_run's plan cache keeps it.
struct PlanHost {
  std::vector<ItemDesc> items;
  std::vector<LaunchRec> launches;
  std::vector<double> disc;
  std::vector<int> unit, exact_int;
  std::vector<uint64_t> N;
  uint64_t path_steps;
  uint32_t total_chunks;
  std::vector<uint32_t> empty_out;
  std::shared_ptr<ReplayGraph> replay;
};
std::unordered_map<std::string, PlanHost> g_plan_cache;
void plan_cache_clear() { g_plan_cache.clear(); }
cudaStream_t g_capture_st = nullptr;   // stream the replay graphs are captured on

// The bytes a plan's host part depends on: the device, the explicit shape, the
// shape table's generation and the cost model, and every work item with its
// parameters' contents (the format table by value, not by address).  Empty:
// not cacheable.
std::string plan_key(const mlmc_work *work, int n, const mlmc_tuning *tuning) {
  std::string k;
  k.reserve((size_t)n * 200 + 64);
  auto put = [&](const void *x, size_t b) { k.append((const char *)x, b); };
  const int32_t dev = g.device;
  const int32_t th = tuning ? tuning->threads : 0, sp = tuning ? tuning->steps_per_thread : 0;
  put(&dev, 4); put(&th, 4); put(&sp, 4); put(&n, 4);
  put(&g_tune_gen, sizeof g_tune_gen);
  put(g_cost, sizeof(double) * 4);
  for (int i = 0; i < n; ++i) {
    const mlmc_work &w = work[i];
    const mlmc_params *p = w.params;
    if (!p || (p->formats && (p->n_formats < 0 || p->n_formats > 64))) return std::string();
    put(&w.level, 4); put(&w.variant, 4); put(&w.first_sample, 8); put(&w.N, 8); put(&w.stream, 4); put(&w.flags, 4);
    put(p, offsetof(mlmc_params, formats));
    put(&p->n_formats, sizeof(mlmc_params) - offsetof(mlmc_params, n_formats));
    const int32_t nf = p->formats ? p->n_formats : -1;
    put(&nf, 4);
    if (p->formats) put(p->formats, sizeof(mlmc_format) * (size_t)p->n_formats);
  }
  return k;
}

// launch_chunking: chunk the items of each launch together (see below); false
// keeps every item's chunking independent of the other items (mlmc_level,
// mlmc_estimate, whose results then equal the engine's, which chunks per item).
mlmc_status plan_create_impl(mlmc_plan **out, const mlmc_work *work, int n_work, uint64_t seed,
                             const mlmc_tuning *tuning, void *const *dumps, bool launch_chunking,
                             Arena *arena = nullptr, bool defer_copy = false, PlanHost **entry = nullptr) {
  if (entry) *entry = nullptr;
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
  // The host part of the plan: items, chunking, launches (everything but the
  // round keys and the device buffers).
  auto build = [&]() -> mlmc_status {
    pl->n_work = n_work;
    pl->disc.resize(n_work);
    pl->unit.resize(n_work);
    pl->exact_int.resize(n_work);
    pl->N.resize(n_work);
    std::vector<BuiltItem> built(n_work);
    std::vector<int> item_threads(n_work), item_spt(n_work);
    for (int i = 0; i < n_work; ++i) {
      s = build_item_cached(work[i], i, dumps ? dumps[i] : nullptr, built[i], pl->disc[i], pl->unit[i],
                            pl->exact_int[i]);
      if (s != MLMC_OK) return s;
      int th, sp;
      tuning_for(built[i].family, built[i].scheme, built[i].pc, work[i].level, &th, &sp);
      if (o_threads) th = o_threads;
      if (o_spt) sp = o_spt;
      item_threads[i] = th;
      item_spt[i] = sp;
      s = chunk_built(built[i], th, sp, g.num_sms);
      if (s != MLMC_OK) return s;
      pl->N[i] = work[i].N;
      pl->path_steps += work[i].N << work[i].level;
    }
    // The nested estimator's 32-bit fixed-point families with Euler-Maruyama and
    // a terminal payoff (15 approximate packed, 8 approximate one sample per
    // thread, 10 correction) share one launch of the merged kernel (family 17)
    // when more than one of them is present: the same chunk bodies, one grid;
    // family 24 when every item's sum1 fits the pre-scaled product.
    {
      auto kind_of = [&](int i) { return merged_kind(built[i]); };
      int seen = 0;
      bool pre = true;   // every merged item takes the pre-scaled product (family 24)
      for (int i = 0; i < n_work; ++i)
        if (kind_of(i) >= 0 && built[i].it.n_chunks > 0) {
          seen |= 1 << kind_of(i);
          pre = pre && built[i].it.ff.pre_ok;
        }
      if (seen & (seen - 1))
        for (int i = 0; i < n_work; ++i) {
          const int k = kind_of(i);
          if (k < 0) continue;
          built[i].it.kind = k;
          built[i].family = pre ? 24 : 17;
        }
    }
    // group by kernel configuration; within a launch, most expensive chunks first
    std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
    std::vector<int> empty;
    for (int i = 0; i < n_work; ++i) {
      if (built[i].it.n_chunks == 0) { empty.push_back(i); continue; }
      groups[std::make_tuple(built[i].family, built[i].scheme, built[i].pc, item_threads[i])].push_back(i);
    }
    if (launch_chunking) {
      // An item alone keeps at least four CTAs per SM (chunk_count), which splits
      // the items of a long work list into chunks of a few dozen path-steps per
      // thread.  When the launch as a whole has that many CTAs without the floor,
      // each item is chunked by its path-steps per thread alone.
      for (auto &kv : groups) {
        std::vector<BuiltItem> alt;
        uint64_t total = 0;
        for (int i : kv.second) {
          alt.push_back(built[i]);
          if ((s = chunk_built(alt.back(), item_threads[i], item_spt[i], g.num_sms, false)) != MLMC_OK) {
            return s;
          }
          total += alt.back().it.n_chunks;
        }
        if (total >= 4ULL * (uint64_t)g.num_sms)
          for (size_t j = 0; j < kv.second.size(); ++j) built[kv.second[j]] = alt[j];
      }
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
      L.dump = false;
      for (int i : o.second) {
        ItemDesc it = built[i].it;
        it.chunk_begin = chunk;
        chunk += it.n_chunks;
        L.smem = std::max(L.smem, built[i].smem);
        L.dump = L.dump || it.dump != nullptr;
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
    return MLMC_OK;
  };
  // mlmc_run's plans are kept by the bytes of everything their host part
  // depends on, so that a work list run again skips the build.
  const bool cacheable = arena && launch_chunking && !dumps;
  std::string key = cacheable ? plan_key(work, n_work, tuning) : std::string();
  auto hit = key.empty() ? g_plan_cache.end() : g_plan_cache.find(key);
  if (hit != g_plan_cache.end()) {
    const PlanHost &h = hit->second;
    if (entry) *entry = &hit->second;
    pl->n_work = n_work;
    pl->items = h.items; pl->launches = h.launches; pl->disc = h.disc; pl->unit = h.unit;
    pl->exact_int = h.exact_int; pl->N = h.N; pl->path_steps = h.path_steps; pl->total_chunks = h.total_chunks;
    pl->empty_out = h.empty_out;
  } else {
    if ((s = build()) != MLMC_OK) { delete pl; return s; }
    if (!key.empty()) {
      if (g_plan_cache.size() >= 64) g_plan_cache.clear();
      auto ins = g_plan_cache.emplace(std::move(key), PlanHost{pl->items, pl->launches, pl->disc, pl->unit,
                                                              pl->exact_int, pl->N, pl->path_steps,
                                                              pl->total_chunks, pl->empty_out, nullptr});
      if (entry) *entry = &ins.first->second;
    }
  }
  const uint32_t chunk = pl->total_chunks;
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

// capture: the stream is being captured into a graph, so the timing events
// are recorded as event nodes of their own (external records)
mlmc_status plan_launch_impl(mlmc_plan *pl, cudaStream_t st, bool capture = false, bool timed = true) {
  // items without samples: zero sums (no CTA writes them; host-side results
  // are zeroed by the host before the launch)
  if (!pl->out_on_host)
    for (uint32_t o : pl->empty_out) MLMC_CK(cudaMemsetAsync(pl->d_out + o, 0, sizeof(DevSums), st));
  if (capture) MLMC_CK(cudaEventRecordWithFlags(pl->t0, st, cudaEventRecordExternal));
  else if (timed) MLMC_CK(cudaEventRecord(pl->t0, st));
  const bool fork = pl->launches.size() > 1;
  // per-kernel events only for plans a caller owns (mlmc_plan_kernel_time) with
  // more than one launch: a single launch is timed by the plan's own events,
  // which then bracket that kernel alone
  const bool kev = !pl->borrowed && fork && timed;
  if (fork) MLMC_CK(cudaEventRecord(pl->fork, st));
  for (size_t i = 0; i < pl->launches.size(); ++i) {
    const LaunchRec &L = pl->launches[i];
    cudaStream_t ls = st;
    if (fork) {
      ls = pl->aux[i];
      MLMC_CK(cudaStreamWaitEvent(ls, pl->fork, 0));
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
    a.dump = L.dump ? 1 : 0;
    if (kev) MLMC_CK(cudaEventRecord(pl->kstart[i], ls));
    MLMC_CK(launch_by_family(L.family, L.scheme, L.pc, dim3(L.n_chunks), dim3(L.threads), L.smem, ls, a, nullptr));
    if (kev) MLMC_CK(cudaEventRecord(pl->kstop[i], ls));
    if (fork) {
      MLMC_CK(cudaEventRecord(pl->join[i], ls));
      MLMC_CK(cudaStreamWaitEvent(st, pl->join[i], 0));
    }
  }
  if (capture) MLMC_CK(cudaEventRecordWithFlags(pl->t1, st, cudaEventRecordExternal));
  else if (timed) MLMC_CK(cudaEventRecord(pl->t1, st));
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
  MLMC_CK(cudaEventSynchronize(pl->t1));
  float ms = 0.0f;
  MLMC_CK(cudaEventElapsedTime(&ms, pl->t0, pl->t1));
  std::vector<DevSums> h(pl->n_work);
  MLMC_CK(cudaMemcpy(h.data(), pl->d_out, sizeof(DevSums) * pl->n_work, cudaMemcpyDeviceToHost));
  convert_results(pl, h.data(), ms, out);
  return MLMC_OK;
}

template <class T>
bool grow_pinned(T *&p, size_t &cap, size_t need, T **dev = nullptr) {
  if (need <= cap) return true;
  if (p) cudaFreeHost(p);
  p = nullptr;
  cap = 0;
  if (dev) *dev = nullptr;
  const size_t n = std::max<size_t>(need, 64);
  if (cudaHostAlloc((void **)&p, sizeof(T) * n, dev ? cudaHostAllocMapped : cudaHostAllocDefault) != cudaSuccess)
    return false;
  if (dev && cudaHostGetDevicePointer((void **)dev, p, 0) != cudaSuccess) {
    cudaFreeHost(p);
    p = nullptr;
    return false;
  }
  cap = n;
  return true;
}

// Launch a cached plan's pass (work-list copy, timing events, kernel) as its
// replay graph on st, capturing the graph first when it is missing or was
// captured with other buffers, events, round keys or device.
mlmc_status replay(PlanHost *entry, mlmc_plan *pl, Arena &A, size_t ni, cudaStream_t st) {
  if (!entry->replay) entry->replay = std::make_shared<ReplayGraph>();
  ReplayGraph &R = *entry->replay;
  const void *bufs[6] = {pl->d_items, pl->d_partials, pl->d_out, pl->d_counters, A.h_items, pl->t0};
  bool same = R.exec && R.device == g.device && R.t1 == (const void *)pl->t1 &&
              std::memcmp(R.bufs, bufs, sizeof bufs) == 0 && std::memcmp(&R.rk, &pl->rk, sizeof(RoundKeys)) == 0;
  if (!same) {
    if (R.exec) { cudaGraphExecDestroy(R.exec); R.exec = nullptr; }
    if (R.graph) { cudaGraphDestroy(R.graph); R.graph = nullptr; }
    if (!g_capture_st) MLMC_CK(cudaStreamCreateWithFlags(&g_capture_st, cudaStreamNonBlocking));
    MLMC_CK(cudaStreamBeginCapture(g_capture_st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemcpyAsync(pl->d_items, A.h_items, sizeof(ItemDesc) * ni, cudaMemcpyHostToDevice,
                                    g_capture_st);
    mlmc_status ls = e == cudaSuccess ? plan_launch_impl(pl, g_capture_st, true) : MLMC_ECUDA;
    cudaGraph_t gr = nullptr;
    const cudaError_t end = cudaStreamEndCapture(g_capture_st, &gr);
    if (ls != MLMC_OK || end != cudaSuccess || !gr) {
      if (gr) cudaGraphDestroy(gr);
      R.failed = true;
      (void)cudaGetLastError();
      return MLMC_ENOTREADY;
    }
    R.graph = gr;
    if (cudaGraphInstantiate(&R.exec, R.graph, 0) != cudaSuccess) {
      R.exec = nullptr;
      R.failed = true;
      (void)cudaGetLastError();
      return MLMC_ENOTREADY;
    }
    std::memcpy(R.bufs, bufs, sizeof bufs);
    R.t1 = pl->t1;
    R.rk = pl->rk;
    R.device = g.device;
  }
  MLMC_CK(cudaGraphLaunch(R.exec, st));
  return MLMC_OK;
}

// One synchronous pass on stream st: work list to the device through pinned
// staging, the launch, one stream sync.  The CTA that completes an item writes
// its sums straight into mapped pinned host memory, so no copy back is queued
// (a small device-to-host copy costs about as much as the launch itself).
mlmc_status run_sync(const mlmc_work *work, int n_work, uint64_t seed, const mlmc_tuning *tuning,
                     void *const *dumps, mlmc_sums *out, cudaStream_t st, bool launch_chunking, bool timed) {
  mlmc_plan *pl = nullptr;
  PlanHost *entry = nullptr;
  mlmc_status s = plan_create_impl(&pl, work, n_work, seed, tuning, dumps, launch_chunking, &g.arena, true, &entry);
  if (s != MLMC_OK) return s;
  Arena &A = g.arena;
  const size_t ni = pl->items.size();
  do {
    if (!grow_pinned(A.h_items, A.cap_h_items, ni) ||
        !grow_pinned(A.h_out, A.cap_h_out, (size_t)n_work, &A.d_hout)) {
      s = MLMC_ENOMEM;
      break;
    }
    std::memcpy(A.h_items, pl->items.data(), sizeof(ItemDesc) * ni);
    // results in host memory: items without samples are zeroed here (no CTA
    // writes them), the others by their last CTA
    pl->d_out = A.d_hout;
    pl->out_on_host = true;
    for (uint32_t o : pl->empty_out) std::memset(&A.h_out[o], 0, sizeof(DevSums));
    s = MLMC_ENOTREADY;
    if (timed && entry && pl->launches.size() == 1 && !(entry->replay && entry->replay->failed)) {
      // a cached single-launch plan: its pass as one graph launch (a plan whose
      // capture failed keeps the direct path below)
      s = replay(entry, pl, A, ni, st);
      if (s != MLMC_OK && s != MLMC_ENOTREADY) break;
    }
    if (s == MLMC_ENOTREADY) {
      s = MLMC_OK;
      if (cudaMemcpyAsync(pl->d_items, A.h_items, sizeof(ItemDesc) * ni, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        s = MLMC_ECUDA;
        break;
      }
      if ((s = plan_launch_impl(pl, st, false, timed)) != MLMC_OK) break;
    }
    float ms = 0.0f;
    if (cudaStreamSynchronize(st) != cudaSuccess ||
        (timed && cudaEventElapsedTime(&ms, pl->t0, pl->t1) != cudaSuccess)) {
      s = MLMC_ECUDA;
      break;
    }
    convert_results(pl, A.h_out, ms, out);
  } while (0);
  free_plan_device(pl);
  delete pl;
  return s;
}


// Median device time (ms) of `reps` launches of a plan of `work` (launch
// shapes from the tuning table), after one untimed launch.
mlmc_status time_plan(const mlmc_work *work, int n_work, uint64_t seed, int reps, double *ms) {
  mlmc_plan *pl = nullptr;
  mlmc_status s = plan_create_impl(&pl, work, n_work, seed, nullptr, nullptr, true);
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
  return run_sync(&w, 1, seed, nullptr, nullptr, out, g.st, false);
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
  return run_sync(&w, 1, seed, nullptr, dumps, out, g.st, false);
}

mlmc_status mlmc_plan_create(mlmc_plan **plan, const mlmc_work *work, int n_work, uint64_t seed,
                             const mlmc_tuning *tuning) {
  MLMC_API_LOCK();
  return plan_create_impl(plan, work, n_work, seed, tuning, nullptr, true);
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

mlmc_status mlmc_plan_launch_items(const mlmc_plan *plan, int k, int32_t *work_index, int cap, int *n) {
  if (!plan || k < 0 || k >= (int)plan->launches.size() || !n || cap < 0 || (cap > 0 && !work_index))
    return MLMC_EINVAL;
  const LaunchRec &L = plan->launches[k];
  for (int i = 0; i < L.n_items && i < cap; ++i) work_index[i] = (int32_t)plan->items[L.item_off + i].out_index;
  *n = L.n_items;
  return MLMC_OK;
}

mlmc_status mlmc_plan_kernel_time(const mlmc_plan *plan, int k, int *family, double *ms) {
  if (!plan || k < 0 || k >= (int)plan->launches.size()) return MLMC_EINVAL;
  if (!plan->launched) return MLMC_ENOTREADY;
  if (family) *family = plan->launches[k].family;
  if (ms) {
    // a single launch: the plan's events bracket the kernel alone
    const bool one = plan->launches.size() == 1;
    const cudaEvent_t a = one ? plan->t0 : plan->kstart[k], b = one ? plan->t1 : plan->kstop[k];
    MLMC_CK(cudaEventSynchronize(b));
    float t = 0.0f;
    MLMC_CK(cudaEventElapsedTime(&t, a, b));
    *ms = t;
  }
  return MLMC_OK;
}

mlmc_status mlmc_plan_elapsed(const mlmc_plan *plan, double *ms) {
  if (!plan || !ms) return MLMC_EINVAL;
  if (!plan->launched) return MLMC_ENOTREADY;
  MLMC_CK(cudaEventSynchronize(plan->t1));
  float t = 0.0f;
  MLMC_CK(cudaEventElapsedTime(&t, plan->t0, plan->t1));
  *ms = t;
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
    if ((s = build_item(work[i], i, nullptr, built[i], disc, unit, ei, ctx_tables())) != MLMC_OK) return s;
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
            if ((s = chunk_built(b, th, sp, g.num_sms)) != MLMC_OK) return s;
            sig.push_back(b.it.groups_per_thread);
          }
          if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
          seen.push_back(sig);
          if (pass == 0) continue;
          g_tune[k] = std::make_pair(th, sp);
          ++g_tune_gen;
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
    ++g_tune_gen;
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
  ++g_tune_gen;
}

mlmc_status mlmc_run(const mlmc_work *work, int n_work, uint64_t seed, const mlmc_tuning *tuning,
                     mlmc_sums *out, void *stream) {
  MLMC_API_LOCK();
  if (!out) return MLMC_EINVAL;
  return run_sync(work, n_work, seed, tuning, nullptr, out, (cudaStream_t)stream, true);
}

}  // extern "C"
