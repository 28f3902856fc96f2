// Host-side internals of the C ABI, shared by its translation units:
// context.cu (device context, tables), items.cu (work items), plan.cu (plans
// and synchronous calls), estimate.cu (adaptive driver), noalloc.cu and
// engine.cu (continuous batching).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "item.h"
#include "mlmc.h"

namespace mlmc_host {

// Status-returning wrapper of a CUDA call.
#define MLMC_CK(call)                                 \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return MLMC_ECUDA;         \
  } while (0)

// ---------------------------------------------------------------------------
// device context (context.cu)
// ---------------------------------------------------------------------------
// Reusable device buffers, streams and events of the synchronous calls
// (mlmc_level, mlmc_run, mlmc_estimate), grown on demand.
struct Arena {
  mlmc::ItemDesc *items = nullptr;
  size_t cap_items = 0;
  mlmc::Partial *partials = nullptr;
  size_t cap_chunks = 0;
  mlmc::DevSums *out = nullptr;
  size_t cap_out = 0;
  uint32_t *counters = nullptr;
  size_t cap_counters = 0;
  mlmc::ItemDesc *h_items = nullptr;       // pinned staging of the work list
  size_t cap_h_items = 0;
  mlmc::DevSums *h_out = nullptr;          // pinned, mapped: the results, written by the kernels
  mlmc::DevSums *d_hout = nullptr;         // its device address
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
  std::map<std::tuple<int, int, int, int, int, int>, void *> tables;  // (method, d, rep, fZ, signed, n) -> table
  std::map<std::pair<int, int>, uint16_t *> m2_perm;         // (d, n) -> device interval ranks (Method 2)
};
extern Ctx g;

// The library's context (streams, tables, caches, staging buffers, tuning
// table) is shared by every call: the public entry points hold this lock, so
// calls from several host threads are serialised.
std::recursive_mutex &api_mutex();
#define MLMC_API_LOCK() std::lock_guard<std::recursive_mutex> mlmc_api_lock_(mlmc_host::api_mutex())

// Initialise (once per device) the library's context on the current device.
mlmc_status ensure_ctx();
// The context's internal stream.
cudaStream_t ctx_stream();
// The context's SM count.
int ctx_num_sms();

// ---------------------------------------------------------------------------
// approximate-Normal tables (context.cu)
// ---------------------------------------------------------------------------
// Method-1 table of index width d (Sec. 3.1): device FP64 copy and host copy.
mlmc_status m1_table(int d, double **dev, const std::vector<double> **host);
// Method 3 (Sec. 3.3): least-squares line a + b k per dyadic index class of
// the lower-half Method-1 table Z (2^(d-1) values), in FP64 (a, b: d-1 each).
void m3_fit_fp64(const double *Z, int d, double *a, double *b);
// The same lines in the representations the kernels read.
void m3_fit(const double *Z, int d, mlmc::M3Coef &c);
uint16_t half_bits(double x);
uint16_t bf16_bits(double x);
// Method 2 (Sec. 3.2), n fields of d/n bits.
struct M2Table {
  int n = 2;
  std::vector<int8_t> c;         // net count of every small-table index in every j
  std::vector<double> x;         // small table
  std::vector<double> values;    // Z~_j, j < 2^d, FP64 sums (ascending index)
  std::vector<uint32_t> pi;      // interval rank of every j
  int iterations = 0;
};
// n divides d, at least 2 bits per field, d <= 14.
bool m2_shape_ok(int d, int n);
mlmc_status m2_build(int d, int n, const M2Table **out);
double m2_value(const M2Table &t, int d, int j, int rep, int fZ);
mlmc_status m2_perm_device(int d, int n, const uint16_t **out);
// Device table of one (method, d, representation, f_Z[, Method-2 fields]),
// cached per process.
mlmc_status get_table(int method, int d, int rep, int fZ, const void **out, bool full_signed = false,
                      int fields = 0);

// ---------------------------------------------------------------------------
// work items (items.cu)
// ---------------------------------------------------------------------------
// Algorithm-1 variable order of mlmc_format.
enum { F_Z = 0, F_CON1 = 1, F_CON2 = 2, F_MUL1 = 3, F_SUM1 = 4, F_MUL2 = 5, F_S = 6 };

bool params_ok(const mlmc_params *p);
// Fields n of Method 2 (icdf_fields, 0 meaning 2).
int m2_fields_of(const mlmc_params *p);
// Approximate-only estimator variants (integer samples, stream 1, packable draws).
bool approx_only_variant(int v);
// Samples per pack (3 with packed draws for approximate-only estimators, else 1).
int pack_lanes(const mlmc_params *p, int variant);
void default_format(const mlmc_params *p, int level, mlmc_format *out);
mlmc::Requant make_rq(int from, int to);
mlmc_status const_fixed(double x, int e, int f, int64_t *out);
bool format_ok_gpu(const mlmc_format &F, bool milstein, int d);
// Proof on the host that only S can saturate (the fast fixed-point datapath),
// for paths of nsteps fine steps; also decides ff.lazy.
bool fast_fixed(const int e[7], const int f[7], int64_t con1, int64_t con1c, int64_t con2, int64_t con3,
                int64_t zmax, bool milstein, int64_t nsteps, mlmc::FastFixed &ff, bool &s64);
int64_t table_zmax_fixed(const double *Z, int d, int method, int fZ, int fields);
int family_of(int variant);
int cost_kind_of(int variant);
// Relative cost per fine path-step of an estimator kind (mlmc_cost_model).
extern double g_cost[4];
double cost_of_variant(int variant);
// Launch shape per (kernel family, scheme, payoff class, level class).
extern std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune;
// Incremented on every change of g_tune (keys of the plan cache).
extern uint64_t g_tune_gen;
int level_class(int level);
// Launch shape (CTA threads, fine path-steps per thread) of a kernel class.
void tuning_for(int family, int scheme, int pc, int level, int *threads, int *spt);

// A work item with its constants and tables resolved (build_item), before
// chunking (chunk_built).
struct BuiltItem {
  mlmc::ItemDesc it;
  int family, scheme, pc;
  size_t smem;
  int kp;               // samples per pack
  double cost_step;     // model cost per fine path-step
  double chunk_cost;    // model cost of one chunk (set by chunk_built)
};
// Where build_item takes the approximate-Normal tables from and how many SMs
// the item is chunked for: the context's cached tables (ctx_tables(), which
// allocate device memory on first use) or mlmc_level_noalloc's fixed scratch.
struct TableSource {
  virtual ~TableSource() {}
  virtual int num_sms() const = 0;
  // largest |value| of the (method, d, fields) table in Z's fixed-point format fZ
  virtual mlmc_status zmax_fixed(int method, int d, int fZ, int fields, int64_t *out) = 0;
  // device table the level kernels read (full signed table for methods 1 and 2,
  // the class lines for method 3)
  virtual mlmc_status device_table(int method, int d, int rep, int fZ, int fields, const void **out) = 0;
  // device copy of Method 2's interval ranks
  virtual mlmc_status m2_perm(int d, int fields, const uint16_t **out) = 0;
};
TableSource &ctx_tables();
// Packed draws of an item of N samples run one sample per thread when the
// packs do not fill one wave of resident threads on num_sms SMs.
bool lane_split(uint64_t N, int num_sms);
// The sample range [first, first + N) of a level keeps every Philox word
// index s 2^l + i and group index below 2^62.
bool sample_range_ok(int level, uint64_t first, uint64_t N);
mlmc_status build_item(const mlmc_work &w, int out_index, void *dump, BuiltItem &b, double &disc, int &unit,
                       int &exact_int, TableSource &src);
// build_item through the per-process cache of built constants.
mlmc_status build_item_cached(const mlmc_work &w, int out_index, void *dump, BuiltItem &b, double &disc, int &unit,
                              int &exact_int);
// Empty that cache and the plan cache (their items point to one device's tables).
void item_cache_clear();
// Empty mlmc_run's cache of host-built plans (plan.cu).
void plan_cache_clear();
// floor: at least four CTAs per SM for this item alone (see chunk_count).
mlmc_status chunk_built(BuiltItem &b, int threads, int spt, int num_sms, bool floor = true);
void make_round_keys(uint64_t seed, mlmc::RoundKeys &rk);
// chunk kind of an item in the merged nested kernel (families 17 / 24), or -1
int merged_kind(const BuiltItem &b);
// Launch one level kernel of a family (or, with occ, query the resident CTAs
// per SM of its device-scheduled kernel).
cudaError_t launch_by_family(int fam, int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             const mlmc::LaunchArgs &a, int *occ);

// ---------------------------------------------------------------------------
// plans (plan.cu)
// ---------------------------------------------------------------------------
// Deterministic sum of each item's chunk partials.
__global__ void finalize_kernel(const mlmc::ItemDesc *items, int n_items, const mlmc::Partial *partials,
                                mlmc::DevSums *out);
double u128_to_double(uint64_t lo, uint64_t hi);
// Plan, launch, read and release in one synchronous call on stream st.
// timed = false: no timing events around the launch, out[i].seconds = 0.
mlmc_status run_sync(const mlmc_work *work, int n_work, uint64_t seed, const mlmc_tuning *tuning,
                     void *const *dumps, mlmc_sums *out, cudaStream_t st, bool launch_chunking,
                     bool timed = true);

}  // namespace mlmc_host
