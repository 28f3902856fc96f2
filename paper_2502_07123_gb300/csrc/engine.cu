// Continuous-batching pricing engine: many adaptive (nested) MLMC requests
// share every level-kernel launch, and one engine iteration is one CUDA-graph
// launch with no host work inside it.
//
// Each admitted request owns a slot of FP64 state in device memory (sums of Y
// and Y^2, sample counts, pending counts per level and estimator) and, built
// on the host once at admission, one work-item template per (level,
// estimator).  An iteration, captured once as a CUDA graph and replayed, is:
//   sched_kernel   - reads every slot's pending counts, chunks each pending
//                    (slot, level, estimator) item exactly as a plan would,
//                    lays the items out by launch group (kernel family,
//                    scheme, payoff class, CTA size, seed) with chunk offsets,
//                    and writes the iteration's work items from the templates;
//   level kernels  - one device-scheduled launch per group, on forked streams,
//                    each a fixed grid of resident CTAs looping over the
//                    group's chunks (level_kernel_dyn);
//   acc_kernel     - sums each item's chunk partials in chunk order and adds
//                    them into its slot;
//   decide_kernel  - per slot: level variances, N = ceil(lambda sqrt(V / C))
//                    (Sec. 2.1 / 2.2), the bias test, a new level or
//                    completion;
// and a copy of the per-slot reports to pinned host memory.  The host admits
// waiting requests between graph launches and reads completed results.  The
// arithmetic, and its order, is that of mlmc_estimate, with every
// floating-point operation rounded separately and every item chunked by its
// own size only, so a request's result does not depend on which other
// requests share its launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "host_api.h"
#include "item.h"
#include "mlmc.h"
#include "reduce.cuh"

using namespace mlmc;
using namespace mlmc_host;

namespace {

constexpr int MAXL = 21;
constexpr int GMAX = 32;                          // launch groups per engine
constexpr unsigned long long NCAP = 1ULL << 34;   // samples of one item per iteration
// bias test once every pending top-up is at most this fraction of its term's
// samples (the value mlmc_estimate uses)
constexpr double ALMOST_DONE = 0.01;

struct SlotState {
  int32_t active, done, L, ne;
  int32_t max_level, exact_mask;       // bit l: the approximate term of level l is exact
  double eps, sqrt_theta_eps, var_target, beta_factor;
  double cost[2];                      // cost per fine path-step of each estimator
  double S1[MAXL][2], S2[MAXL][2];     // discounted sums
  double Vext[MAXL][2];                // extrapolated variance of a level not yet sampled
  unsigned long long N[MAXL][2], dN[MAXL][2];
  double price, se;
  double rem;                          // remaining-bias estimate of the final bias test
};

// What the host reads back after each graph launch, per slot.
struct SlotReport {
  int32_t active, done, L, pad;
  double price, se, rem;
};

// Per (slot, level, estimator) template: what the scheduler needs beside the ItemDesc.
struct TmplMeta {
  int32_t group;          // launch group, -1: no template
  int32_t kp, threads, spt;
  int32_t unit, exact_int, level, est;
  double disc;
};

// Iteration status (device; copied to pinned host memory with the reports).
struct EngStatus {
  uint32_t n_items;                  // work items of the last iteration
  uint32_t overflow;                 // 1: it needed more chunks than the partial array holds
  unsigned long long chunks;         // chunks it needed (all groups)
  unsigned long long path_steps;     // fine path-steps simulated since creation
  int32_t active, done;              // slots active / completed after it
};

__device__ double level_var(const SlotState &s, int l, int k) {
  if (k == 0 && ((s.exact_mask >> l) & 1)) return 0.0;  // an exact mean has no variance
  if (s.N[l][k] == 0) return s.Vext[l][k];
  const double n = __ull2double_rn(s.N[l][k]);
  const double m = __ddiv_rn(s.S1[l][k], n);
  const double v = __dsub_rn(__ddiv_rn(s.S2[l][k], n), __dmul_rn(m, m));
  return v > 0.0 ? v : 0.0;
}

// Per-warp scratch of a slot's decision (shared memory beside the slot's copy):
// per (level, estimator) term, level-major.
struct DecideScratch {
  double v[2 * MAXL];     // floored level variances
  double a[2 * MAXL];     // sqrt(V C); then S1 / N
  double q[2 * MAXL];     // sqrt(V / C); then the variance of the mean
  double lam;
};

// dN = ceil(lambda sqrt(V/C)) - N over all levels <= L and estimators
// (mlmc_estimate's update, operation for operation): each term's divisions and
// square roots on its own lane of the warp, the level-order parts (the floor
// V_l >= V_{l-1} / (2 * 2^beta) from level 2 on, the sum for lambda) on one
// lane.  Dividing by the power of two 2^beta is multiplying by its exact
// reciprocal: the same correctly rounded value.
__device__ void update_dn(SlotState &s, DecideScratch &d, int lane) {
  const int ne = s.ne, T = (s.L + 1) * ne;
  for (int t = lane; t < T; t += 32) d.v[t] = level_var(s, t / ne, t % ne);
  __syncwarp();
  if (lane < ne) {
    const double inv_bf = __ddiv_rn(1.0, s.beta_factor);
    double vprev = 0.0;
    for (int l = 0; l <= s.L; ++l) {
      const int t = l * ne + lane;
      double v = d.v[t];
      if (l >= 2) v = fmax(v, __dmul_rn(__dmul_rn(0.5, vprev), inv_bf));
      vprev = v;
      d.v[t] = fmax(v, 1e-300);
    }
  }
  __syncwarp();
  for (int t = lane; t < T; t += 32) {
    const double C = ldexp(s.cost[t % ne], t / ne);
    d.a[t] = __dsqrt_rn(__dmul_rn(d.v[t], C));
    d.q[t] = __dsqrt_rn(__ddiv_rn(d.v[t], C));
  }
  __syncwarp();
  if (lane == 0) {
    double lam = 0.0;
    for (int t = 0; t < T; ++t) lam = __dadd_rn(lam, d.a[t]);
    d.lam = __ddiv_rn(lam, s.var_target);
  }
  __syncwarp();
  for (int t = lane; t < T; t += 32) {
    const int l = t / ne, k = t % ne;
    const double x = d.v[t] > 0.0 ? __dmul_rn(d.lam, d.q[t]) : 0.0;
    const unsigned long long want = (unsigned long long)ceil(fmin(x, 1e18));
    s.dN[l][k] = want > s.N[l][k] ? want - s.N[l][k] : 0ULL;
  }
  __syncwarp();
}

// Pending work of template t (slot t / il): samples [first, first + N).
__device__ bool pending(const SlotState *slots, const TmplMeta *meta, int il, int t, unsigned long long &first,
                        unsigned long long &N) {
  const TmplMeta &m = meta[t];
  if (m.group < 0) return false;
  const SlotState &S = slots[t / il];
  if (!S.active || S.done || m.level > S.L || m.est >= S.ne) return false;
  const unsigned long long dn = S.dN[m.level][m.est];
  if (dn == 0) return false;
  N = dn < NCAP ? dn : NCAP;
  first = S.N[m.level][m.est];
  return true;
}

// Chunk count and groups per thread of template t's pending work (as a plan chunks it).
__device__ uint64_t pending_chunks(const TmplMeta &m, unsigned long long first, unsigned long long N, int num_sms,
                                   uint32_t *gpt, uint64_t *g0, uint64_t *g1) {
  const uint64_t spc = samples_per_group(m.level, m.kp);
  *g0 = first / spc;
  *g1 = (first + N + spc - 1) / spc;
  return chunk_count(*g1 - *g0, steps_per_group(m.level), m.kp, m.threads, m.spt, num_sms, gpt);
}

// One block of 1024 threads: the iteration's work list, grouped by launch group,
// and its work items (one warp per item: the lanes copy the template, lane 0
// sets the samples and chunking; before, a separate kernel node).
__global__ void __launch_bounds__(1024) sched_kernel(const SlotState *slots, const TmplMeta *meta, const ItemDesc *tmpl,
                                                     int n_tmpl, int il, int n_groups, unsigned long long cap_chunks,
                                                     int num_sms, uint32_t *t_nch, int *run_src, uint32_t *run_nch,
                                                     uint32_t *run_cb, DynLaunch *dyn, EngStatus *status,
                                                     ItemDesc *run, unsigned long long *run_n) {
  __shared__ uint32_t s_cnt[GMAX], s_fill[GMAX], s_ioff[GMAX];
  __shared__ unsigned long long s_chk[GMAX], s_coff[GMAX];
  __shared__ int s_over;
  const int tid = threadIdx.x;
  if (tid < GMAX) { s_cnt[tid] = 0; s_fill[tid] = 0; s_chk[tid] = 0; }
  __syncthreads();
  for (int t = tid; t < n_tmpl; t += blockDim.x) {
    unsigned long long first, N;
    uint32_t nch = 0;
    if (pending(slots, meta, il, t, first, N)) {
      uint32_t gpt;
      uint64_t g0, g1;
      nch = (uint32_t)pending_chunks(meta[t], first, N, num_sms, &gpt, &g0, &g1);
      const int g = meta[t].group;
      atomicAdd(&s_cnt[g], 1u);
      atomicAdd(&s_chk[g], (unsigned long long)nch);
    }
    t_nch[t] = nch;
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t ioff = 0;
    unsigned long long coff = 0;
    for (int g = 0; g < n_groups; ++g) {
      s_ioff[g] = ioff;
      s_coff[g] = coff;
      ioff += s_cnt[g];
      coff += s_chk[g];
    }
    const int over = coff > cap_chunks;
    s_over = over;
    for (int g = 0; g < n_groups; ++g) {
      DynLaunch d;
      d.item_off = s_ioff[g];
      d.n_items = over ? 0u : s_cnt[g];
      d.chunk0 = (uint32_t)s_coff[g];
      d.n_chunks = over ? 0u : (uint32_t)s_chk[g];
      dyn[g] = d;
    }
    status->n_items = over ? 0u : ioff;
    status->overflow = (uint32_t)over;
    status->chunks = coff;
    status->active = 0;
    status->done = 0;
  }
  __syncthreads();
  if (s_over) return;
  for (int t = tid; t < n_tmpl; t += blockDim.x) {
    const uint32_t nch = t_nch[t];
    if (nch == 0) continue;
    const int g = meta[t].group;
    const uint32_t pos = s_ioff[g] + atomicAdd(&s_fill[g], 1u);
    run_src[pos] = t;
    run_nch[pos] = nch;
  }
  __syncthreads();
  // chunk offsets: warp g scans group g in list order
  const int warp = tid >> 5, lane = tid & 31;
  if (warp < n_groups) {
    const uint32_t beg = s_ioff[warp], n = s_cnt[warp];
    unsigned long long base = s_coff[warp];
    for (uint32_t j0 = 0; j0 < n; j0 += 32) {
      const uint32_t j = j0 + lane;
      unsigned long long x = j < n ? run_nch[beg + j] : 0ULL;
      unsigned long long inc = x;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (j < n) run_cb[beg + j] = (uint32_t)(base + inc - x);
      base += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  __syncthreads();
  // the iteration's work items from the templates, one warp per item: the
  // lanes copy the template, lane 0 sets its samples and chunking
  static_assert(sizeof(ItemDesc) % 8 == 0, "item templates are copied in 8-byte words");
  const uint32_t n_items = status->n_items;
  for (uint32_t j = (uint32_t)warp; j < n_items; j += blockDim.x >> 5) {
    const int t = run_src[j];
    const unsigned long long *src = (const unsigned long long *)&tmpl[t];
    unsigned long long *dst = (unsigned long long *)&run[j];
    for (int w = lane; w < (int)(sizeof(ItemDesc) / 8); w += 32) dst[w] = src[w];
    __syncwarp();
    if (lane == 0) {
      unsigned long long first = 0, N = 0;
      pending(slots, meta, il, t, first, N);
      uint32_t gpt;
      uint64_t g0, g1;
      pending_chunks(meta[t], first, N, num_sms, &gpt, &g0, &g1);
      const uint64_t spc = samples_per_group(meta[t].level, meta[t].kp);
      ItemDesc &it = run[j];
      it.first = first;
      it.N = N;
      it.g0 = g0;
      it.g1 = g1;
      it.gf0 = (first + spc - 1) / spc;
      it.gf1 = (first + N) / spc;
      if (it.gf1 < it.gf0) it.gf1 = it.gf0;
      it.groups_per_thread = gpt;
      it.n_chunks = run_nch[j];
      it.chunk_begin = run_cb[j];
      it.out_index = j;
      run_n[j] = N;
    }
    __syncwarp();
  }
}

// Sum each item's chunk partials (one warp per item, chunk order) and add the
// result into its slot (each (slot, level, estimator) appears at most once).
__global__ void acc_kernel(SlotState *slots, const TmplMeta *meta, int il, const int *run_src,
                           const uint32_t *run_nch, const uint32_t *run_cb, const unsigned long long *run_n,
                           const Partial *partials, EngStatus *status) {
  const uint32_t j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (status->overflow || j >= status->n_items) return;
  const DevSums r = warp_sum_partials(partials + run_cb[j], run_nch[j]);
  if ((threadIdx.x & 31) != 0) return;
  const int t = run_src[j];
  const TmplMeta &m = meta[t];
  SlotState &s = slots[t / il];
  double sum, sum2;
  if (m.exact_int) {
    sum = __dmul_rn(m.disc, ldexp(__ll2double_rn(r.isum), -m.unit));
    sum2 = __dmul_rn(__dmul_rn(m.disc, m.disc), ldexp(u128_to_double_rn(r.isum2_lo, r.isum2_hi), -2 * m.unit));
  } else {
    sum = __dmul_rn(m.disc, r.dsum);
    sum2 = __dmul_rn(__dmul_rn(m.disc, m.disc), r.dsum2);
  }
  s.S1[m.level][m.est] = __dadd_rn(s.S1[m.level][m.est], sum);
  s.S2[m.level][m.est] = __dadd_rn(s.S2[m.level][m.est], sum2);
  s.N[m.level][m.est] += run_n[j];
  atomicAdd(&status->path_steps, run_n[j] << m.level);
}

// Per slot: new sample counts, the bias test, a new level, or completion; the
// warp's lanes share the per-term arithmetic (update_dn), the level-order sums
// run on lane 0.  s is the slot's state in shared memory (decide_kernel).
__device__ void decide_slot(SlotState &s, DecideScratch &d, SlotReport &r, EngStatus *status, int lane) {
  if (s.active && !s.done) {
    update_dn(s, d, lane);
    // the bias test once every remaining top-up is within ALMOST_DONE of its
    // term's samples (mlmc_estimate's loop, operation for operation)
    const int ne = s.ne, T = (s.L + 1) * ne;
    bool any = false, small = true;
    for (int t = lane; t < T; t += 32) {
      const int l = t / ne, k = t % ne;
      any |= s.dN[l][k] > 0;
      small &= !(__ull2double_rn(s.dN[l][k]) > __dmul_rn(ALMOST_DONE, __ull2double_rn(s.N[l][k])));
    }
    any = __any_sync(0xffffffffu, any);
    small = __all_sync(0xffffffffu, small);
    if (small) {
      // bias estimate from the last two level means (weak order 1), with the
      // floor |m_l| >= |m_{l-1}| / (2 * 2^alpha) from level 2 on (the division
      // by 2^alpha = 2 as a multiplication by 1/2)
      for (int t = lane; t < T; t += 32) d.a[t] = __ddiv_rn(s.S1[t / ne][t % ne], __ull2double_rn(s.N[t / ne][t % ne]));
      __syncwarp();
      int add = 0, fin = 0;
      double rem = 0.0;
      if (lane == 0) {
        double mprev = 0.0, mL = 0.0, mL1 = 0.0;
        for (int l = 0; l <= s.L; ++l) {
          double ml = 0.0;
          for (int k = 0; k < ne; ++k) ml = __dadd_rn(ml, d.a[l * ne + k]);
          ml = fabs(ml);
          if (l >= 2) ml = fmax(ml, __dmul_rn(__dmul_rn(0.5, mprev), 0.5));
          if (l == s.L - 1) mL1 = ml;
          if (l == s.L) mL = ml;
          mprev = ml;
        }
        rem = fabs(mL);
        rem = fmax(rem, __dmul_rn(fabs(mL1), 0.5));
        if (rem > s.sqrt_theta_eps && s.L < s.max_level) {
          add = 1;
          const int L = ++s.L;
          for (int k = 0; k < ne; ++k) {
            s.N[L][k] = 0; s.dN[L][k] = 0; s.S1[L][k] = 0.0; s.S2[L][k] = 0.0;
            s.Vext[L][k] = __ddiv_rn(fmax(level_var(s, L - 1, k), 1e-300), s.beta_factor);
          }
        } else if (!any) {
          fin = 1;
        }
      }
      add = __shfl_sync(0xffffffffu, add, 0);
      fin = __shfl_sync(0xffffffffu, fin, 0);
      rem = __shfl_sync(0xffffffffu, rem, 0);
      __syncwarp();
      if (add) {
        update_dn(s, d, lane);
      } else if (fin) {
        for (int t = lane; t < T; t += 32) {
          const int l = t / ne, k = t % ne;
          const double n = __ull2double_rn(s.N[l][k]);
          d.a[t] = __ddiv_rn(s.S1[l][k], n);
          d.q[t] = __ddiv_rn(level_var(s, l, k), n);
        }
        __syncwarp();
        if (lane == 0) {
          double pr = 0.0, var = 0.0;
          for (int t = 0; t < T; ++t) {
            pr = __dadd_rn(pr, d.a[t]);
            var = __dadd_rn(var, d.q[t]);
          }
          s.price = pr;
          s.se = __dsqrt_rn(var);
          s.rem = rem;
          s.done = 1;
        }
        __syncwarp();
      }
    }
  }
  if (lane == 0) {
    r.active = s.active;
    r.done = s.done;
    r.L = s.L;
    r.price = s.price;
    r.se = s.se;
    r.rem = s.rem;
    if (s.active && !s.done) atomicAdd(&status->active, 1);
    if (s.active && s.done) atomicAdd(&status->done, 1);
  }
}

// One warp per slot: the slot's state is copied into shared memory by the
// warp's lanes, the decision runs on that copy over the warp (its FP64
// divisions and square roots, one chain per slot on one lane before, took
// ~65 us per iteration on this part), and the copy is written back.
constexpr int DECIDE_WARPS = 4;
static_assert(sizeof(SlotState) % 8 == 0, "the slot state is copied in 8-byte words");
__global__ void __launch_bounds__(DECIDE_WARPS * 32) decide_kernel(SlotState *slots, SlotReport *rep, int n_slots,
                                                                    EngStatus *status) {
  __shared__ SlotState sh[DECIDE_WARPS];
  __shared__ DecideScratch scratch[DECIDE_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * DECIDE_WARPS + warp;
  if (i >= n_slots || status->overflow) return;   // uniform over the warp
  constexpr int WORDS = (int)(sizeof(SlotState) / 8);
  unsigned long long *g = (unsigned long long *)&slots[i];
  unsigned long long *l = (unsigned long long *)&sh[warp];
  for (int w = lane; w < WORDS; w += 32) l[w] = g[w];
  __syncwarp();
  decide_slot(sh[warp], scratch[warp], rep[i], status, lane);
  __syncwarp();
  for (int w = lane; w < WORDS; w += 32) g[w] = l[w];
}

struct Request {
  uint64_t id;
  mlmc_params p;
  std::vector<mlmc_format> formats;   // the request's own copy (params->formats points here)
  double eps;
  int mode;
  uint64_t seed;
  double t_submit, t_admit, t_done;
  int slot;
  int done;
  mlmc_status status;                 // MLMC_OK, or why admission failed
  double price, se;
  int L;
  int exact_mask;                     // bit l: approximate term of level l computed by enumeration
  double rem;                         // final remaining-bias estimate
  std::vector<uint64_t> N;            // samples per (level, estimator) at completion, level-major
};

int exact_mask_of(int mode, int d) {
  if (mode != 5 && mode != 6 && mode != 9 && mode != 10) return 0;
  int m = 0;
  for (int l = 0; l <= 1; ++l)
    if ((d << l) <= 20) m |= 1 << l;
  return m;
}

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

bool mode_variants(int mode, int &ne, int v[2]) {
  switch (mode) {
    case 0: ne = 1; v[0] = MLMC_FP64_EXACT; v[1] = 0; return true;
    case 1: ne = 1; v[0] = MLMC_FP32_EXACT; v[1] = 0; return true;
    case 2: ne = 2; v[0] = MLMC_FIXED_APPROX; v[1] = MLMC_NESTED_CORR_FIXED; return true;
    case 3: ne = 2; v[0] = MLMC_FP16_APPROX; v[1] = MLMC_NESTED_CORR_FP16; return true;
    case 4: ne = 2; v[0] = MLMC_BF16_APPROX; v[1] = MLMC_NESTED_CORR_BF16; return true;
    case 5: ne = 2; v[0] = MLMC_FIXED_APPROX; v[1] = MLMC_NESTED_CORR_FIXED; return true;
    case 6: ne = 2; v[0] = MLMC_FP16_APPROX; v[1] = MLMC_NESTED_CORR_FP16; return true;
    case 7: case 9: ne = 2; v[0] = MLMC_FP16S_APPROX; v[1] = MLMC_NESTED_CORR_FP16S; return true;
    case 8: case 10: ne = 2; v[0] = MLMC_BF16S_APPROX; v[1] = MLMC_NESTED_CORR_BF16S; return true;
    default: return false;
  }
}

// A launch group: the items of one level-kernel launch per iteration.
struct Group {
  int family, scheme, pc, threads;
  size_t smem;
  uint64_t seed;
  RoundKeys rk;
  int refs = 0;           // templates of admitted requests in this group
  int grid = 0;           // resident CTAs of the device-scheduled kernel
  bool in_graph = false;
};

template <class T>
bool dev_alloc(T **p, size_t n) {
  return cudaMalloc((void **)p, sizeof(T) * std::max<size_t>(n, 1)) == cudaSuccess;
}

}  // namespace

struct mlmc_engine {
  int max_slots = 0, max_level = 10, il = 0, iters = 1;
  int num_sms = 0;
  // device state
  SlotState *d_slots = nullptr;
  SlotReport *d_rep = nullptr;
  ItemDesc *d_tmpl = nullptr, *d_run = nullptr;
  TmplMeta *d_meta = nullptr;
  uint32_t *d_tnch = nullptr, *d_run_nch = nullptr, *d_run_cb = nullptr;
  int *d_run_src = nullptr;
  unsigned long long *d_run_n = nullptr;
  DynLaunch *d_dyn = nullptr;
  EngStatus *d_status = nullptr;
  uint32_t *d_iter = nullptr;                  // iterations of the running launch (loop control)
  Partial *d_partials = nullptr;
  unsigned long long cap_chunks = 0;
  // pinned host copies of the reports
  SlotReport *h_rep = nullptr;
  EngStatus *h_status = nullptr;
  // groups and the captured iteration
  std::vector<Group> groups;
  std::vector<std::vector<int>> slot_groups;   // per slot: group of each template (for refs)
  bool dirty = true;
  cudaStream_t cs = nullptr;                   // capture stream
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // host queue
  std::vector<int> slot_req;                   // slot -> index in reqs, -1 if free
  std::deque<size_t> queue;                    // waiting requests (indices into reqs)
  std::vector<Request> reqs;
  std::map<uint64_t, size_t> by_id;
  std::deque<uint64_t> completed;              // ids of completed requests not yet drained
  uint64_t next_id = 1;
  uint64_t steps = 0, launches = 0, path_steps = 0, captures = 0;
};

namespace {

size_t slot_bytes(int il) {
  return sizeof(SlotState) + sizeof(SlotReport) +
         (size_t)il * (2 * sizeof(ItemDesc) + sizeof(TmplMeta) + 4 * sizeof(uint32_t) + sizeof(unsigned long long) +
                       4 * sizeof(Partial));
}

void release(mlmc_engine *e) {
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  for (auto st : e->aux) cudaStreamDestroy(st);
  for (auto ev : e->join) cudaEventDestroy(ev);
  if (e->fork) cudaEventDestroy(e->fork);
  if (e->cs) cudaStreamDestroy(e->cs);
  cudaFree(e->d_slots); cudaFree(e->d_rep); cudaFree(e->d_tmpl); cudaFree(e->d_run); cudaFree(e->d_meta);
  cudaFree(e->d_tnch); cudaFree(e->d_run_nch); cudaFree(e->d_run_cb); cudaFree(e->d_run_src); cudaFree(e->d_run_n);
  cudaFree(e->d_dyn); cudaFree(e->d_status); cudaFree(e->d_partials); cudaFree(e->d_iter);
  if (e->h_rep) cudaFreeHost(e->h_rep);
  if (e->h_status) cudaFreeHost(e->h_status);
}

// One engine iteration, enqueued on the capture stream e->cs (live: the launch
// classes in the graph).
cudaError_t enqueue_iteration(mlmc_engine *e, const std::vector<int> &live) {
  const int n_tmpl = e->max_slots * e->il;
  sched_kernel<<<1, 1024, 0, e->cs>>>(e->d_slots, e->d_meta, e->d_tmpl, n_tmpl, e->il, (int)e->groups.size(),
                                      e->cap_chunks, e->num_sms, e->d_tnch, e->d_run_src, e->d_run_nch,
                                      e->d_run_cb, e->d_dyn, e->d_status, e->d_run, e->d_run_n);
  cudaError_t err = cudaEventRecord(e->fork, e->cs);
  for (size_t i = 0; i < live.size() && err == cudaSuccess; ++i) {
    const Group &G = e->groups[live[i]];
    cudaStream_t ls = e->aux[i];
    LaunchArgs a;
    a.items = e->d_run;
    a.n_items = 0;
    a.chunk0 = 0;
    a.partials = e->d_partials;
    a.rk = G.rk;
    a.dyn = e->d_dyn + live[i];
    a.counters = nullptr;   // acc_kernel sums the partials
    a.dump = 0;
    a.out = nullptr;
    if ((err = cudaStreamWaitEvent(ls, e->fork, 0)) != cudaSuccess) break;
    if ((err = launch_by_family(G.family, G.scheme, G.pc, dim3(G.grid), dim3(G.threads), G.smem, ls, a,
                                nullptr)) != cudaSuccess)
      break;
    if ((err = cudaEventRecord(e->join[i], ls)) != cudaSuccess) break;
    err = cudaStreamWaitEvent(e->cs, e->join[i], 0);
  }
  if (err != cudaSuccess) return err;
  acc_kernel<<<(n_tmpl + 3) / 4, 128, 0, e->cs>>>(e->d_slots, e->d_meta, e->il, e->d_run_src, e->d_run_nch,
                                                  e->d_run_cb, e->d_run_n, e->d_partials, e->d_status);
  decide_kernel<<<(e->max_slots + DECIDE_WARPS - 1) / DECIDE_WARPS, DECIDE_WARPS * 32, 0, e->cs>>>(
      e->d_slots, e->d_rep, e->max_slots, e->d_status);
  return cudaGetLastError();
}

// Copies of the per-slot reports and the status to pinned host memory.
cudaError_t enqueue_reports(mlmc_engine *e) {
  cudaError_t err = cudaMemcpyAsync(e->h_rep, e->d_rep, sizeof(SlotReport) * e->max_slots, cudaMemcpyDeviceToHost,
                                    e->cs);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(e->h_status, e->d_status, sizeof(EngStatus), cudaMemcpyDeviceToHost, e->cs);
  return err;
}

// Keep iterating while a slot is still active, the partial array sufficed and
// fewer than `cap` iterations ran in this launch (the counter is zeroed by the
// host before each launch).
__global__ void loop_control_kernel(cudaGraphConditionalHandle h, const EngStatus *status, uint32_t *iter,
                                    uint32_t cap) {
  const uint32_t k = ++*iter;
  cudaGraphSetConditional(h, (status->active > 0 && !status->overflow && k < cap) ? 1u : 0u);
}

// The whole adaptive run as one graph launch: a conditional WHILE node whose
// body is one iteration plus the loop control, then the report copies.
mlmc_status capture_until_done(mlmc_engine *e, const std::vector<int> &live) {
  cudaGraph_t g = nullptr;
  MLMC_CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t cond = nullptr;
  cudaError_t err = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
  if (err == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    err = cudaGraphAddNode(&cond, g, nullptr, nullptr, 0, &cp);
  }
  if (err == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    err = cudaStreamBeginCaptureToGraph(e->cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
      cudaError_t e2 = enqueue_iteration(e, live);
      if (e2 == cudaSuccess) {
        loop_control_kernel<<<1, 1, 0, e->cs>>>(h, e->d_status, e->d_iter, (uint32_t)(-e->iters));
        e2 = cudaGetLastError();
      }
      cudaGraph_t out = nullptr;
      err = cudaStreamEndCapture(e->cs, &out);
      if (e2 != cudaSuccess) err = e2;
    }
  }
  if (err == cudaSuccess) {
    err = cudaStreamBeginCaptureToGraph(e->cs, g, &cond, nullptr, 1, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
      cudaError_t e2 = enqueue_reports(e);
      cudaGraph_t out = nullptr;
      err = cudaStreamEndCapture(e->cs, &out);
      if (e2 != cudaSuccess) err = e2;
    }
  }
  if (err == cudaSuccess) err = cudaGraphInstantiate(&e->exec, g, 0);
  if (err != cudaSuccess) {
    cudaGraphDestroy(g);
    return MLMC_ECUDA;
  }
  e->graph = g;
  e->dirty = false;
  e->captures += 1;
  return MLMC_OK;
}

// Capture `iters` iterations (and the report copies) as one CUDA graph.
mlmc_status capture(mlmc_engine *e) {
  if (e->exec) { cudaGraphExecDestroy(e->exec); e->exec = nullptr; }
  if (e->graph) { cudaGraphDestroy(e->graph); e->graph = nullptr; }
  std::vector<int> live;
  for (int gi = 0; gi < (int)e->groups.size(); ++gi) {
    Group &G = e->groups[gi];
    G.in_graph = G.refs > 0;
    if (!G.in_graph) continue;
    live.push_back(gi);
    if (G.grid == 0) {
      int nb = 0;
      LaunchArgs q;
      std::memset(&q, 0, sizeof q);
      MLMC_CK(launch_by_family(G.family, G.scheme, G.pc, dim3(1), dim3(G.threads), G.smem, e->cs, q, &nb));
      if (nb < 1) return MLMC_EINVAL;
      G.grid = nb * e->num_sms;
    }
  }
  while (e->aux.size() < live.size()) {
    cudaStream_t st;
    cudaEvent_t ev;
    MLMC_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    e->aux.push_back(st);
    MLMC_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    e->join.push_back(ev);
  }
  if (e->iters < 0) return capture_until_done(e, live);
  MLMC_CK(cudaStreamBeginCapture(e->cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  for (int k = 0; k < e->iters && err == cudaSuccess; ++k) err = enqueue_iteration(e, live);
  if (err == cudaSuccess) err = enqueue_reports(e);
  cudaGraph_t gr = nullptr;
  const cudaError_t end = cudaStreamEndCapture(e->cs, &gr);
  if (err != cudaSuccess || end != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    return MLMC_ECUDA;
  }
  e->graph = gr;
  MLMC_CK(cudaGraphInstantiate(&e->exec, e->graph, 0));
  e->dirty = false;
  e->captures += 1;
  return MLMC_OK;
}

// Group index of a launch class, added if new (MLMC_EINVAL beyond GMAX).
mlmc_status group_of(mlmc_engine *e, const BuiltItem &b, int threads, uint64_t seed, int *gi) {
  for (int i = 0; i < (int)e->groups.size(); ++i) {
    const Group &G = e->groups[i];
    if (G.family == b.family && G.scheme == b.scheme && G.pc == b.pc && G.threads == threads && G.smem == b.smem &&
        G.seed == seed) {
      *gi = i;
      return MLMC_OK;
    }
  }
  Group G;
  G.family = b.family; G.scheme = b.scheme; G.pc = b.pc; G.threads = threads; G.smem = b.smem; G.seed = seed;
  make_round_keys(seed, G.rk);
  if ((int)e->groups.size() < GMAX) {
    e->groups.push_back(G);
    *gi = (int)e->groups.size() - 1;
    return MLMC_OK;
  }
  // all slots taken: reuse one that no admitted request refers to any more
  for (int i = 0; i < (int)e->groups.size(); ++i)
    if (e->groups[i].refs == 0) {
      e->groups[i] = G;
      e->dirty = true;
      *gi = i;
      return MLMC_OK;
    }
  return MLMC_EINVAL;
}

// Admit request idx into free slot sl: templates, metadata and initial state.
mlmc_status admit(mlmc_engine *e, int sl, size_t idx, cudaStream_t st) {
  Request &r = e->reqs[idx];
  int ne, v[2];
  mode_variants(r.mode, ne, v);
  r.p.formats = r.formats.empty() ? nullptr : r.formats.data();
  const int il = e->il;
  std::vector<ItemDesc> tm(il);
  std::vector<TmplMeta> meta(il);
  std::vector<int> gl;
  std::memset(tm.data(), 0, sizeof(ItemDesc) * il);
  for (int t = 0; t < il; ++t) meta[t].group = -1;
  for (int l = 0; l <= e->max_level; ++l)
    for (int k = 0; k < ne; ++k) {
      const bool exact = k == 0 && ((r.exact_mask >> l) & 1);
      mlmc_work w;
      std::memset(&w, 0, sizeof w);
      w.params = &r.p;
      w.level = l;
      w.variant = v[k];
      w.first_sample = 0;
      w.N = exact ? (1ULL << (r.p.icdf_bits << l)) : 0;
      w.stream = -1;
      w.flags = exact ? MLMC_WORK_ENUMERATE : 0;
      BuiltItem b;
      double disc;
      int unit, ei;
      mlmc_status s = build_item(w, 0, nullptr, b, disc, unit, ei, ctx_tables());
      int th, sp, gi = -1;
      if (s == MLMC_OK) {
        tuning_for(b.family, b.scheme, b.pc, l, &th, &sp);
        s = group_of(e, b, th, r.seed, &gi);
      }
      if (s != MLMC_OK) {
        for (int g2 : gl) e->groups[g2].refs -= 1;   // release what this admission took
        return s;
      }
      // hold the class at once, so that a later template of this request cannot reuse it
      Group &G = e->groups[gi];
      if (G.refs++ == 0 && !G.in_graph) e->dirty = true;
      const int t = l * 2 + k;
      tm[t] = b.it;
      TmplMeta &m = meta[t];
      m.group = gi; m.kp = b.kp; m.threads = th; m.spt = sp;
      m.unit = unit; m.exact_int = ei; m.level = l; m.est = k; m.disc = disc;
      gl.push_back(gi);
    }
  e->slot_groups[sl] = gl;
  SlotState h;
  std::memset(&h, 0, sizeof h);
  h.active = 1;
  h.done = 0;
  h.L = 2;
  h.ne = ne;
  h.max_level = e->max_level;
  h.eps = r.eps;
  h.sqrt_theta_eps = std::sqrt(0.5) * r.eps;
  h.var_target = (1.0 - 0.5) * r.eps * r.eps;
  h.beta_factor = std::pow(2.0, r.p.scheme == MLMC_MILSTEIN ? 2.0 : 1.0);
  for (int k = 0; k < ne; ++k) h.cost[k] = cost_of_variant(v[k]);
  h.exact_mask = r.exact_mask;
  for (int l = 0; l <= 2; ++l)
    for (int k = 0; k < ne; ++k)
      h.dN[l][k] = (k == 0 && ((r.exact_mask >> l) & 1)) ? (1ULL << (r.p.icdf_bits << l)) : 10000;
  MLMC_CK(cudaMemcpyAsync(e->d_tmpl + (size_t)sl * il, tm.data(), sizeof(ItemDesc) * il, cudaMemcpyHostToDevice, st));
  MLMC_CK(cudaMemcpyAsync(e->d_meta + (size_t)sl * il, meta.data(), sizeof(TmplMeta) * il, cudaMemcpyHostToDevice,
                          st));
  MLMC_CK(cudaMemcpyAsync(e->d_slots + sl, &h, sizeof h, cudaMemcpyHostToDevice, st));
  // pageable sources: tm, meta and h may go out of scope once cudaMemcpyAsync returns
  return MLMC_OK;
}

void free_slot_groups(mlmc_engine *e, int sl) {
  for (int gi : e->slot_groups[sl]) e->groups[gi].refs -= 1;
  e->slot_groups[sl].clear();
}

}  // namespace

extern "C" {

mlmc_status mlmc_engine_create(mlmc_engine **out, const mlmc_engine_config *cfg) {
  MLMC_API_LOCK();
  if (!out || !cfg || cfg->max_level < 2 || cfg->max_level > MAXL - 1) return MLMC_EINVAL;
  if (cfg->iters_per_launch < -4096 || cfg->iters_per_launch > 64 || cfg->reserved != 0) return MLMC_EINVAL;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  const int il = (cfg->max_level + 1) * 2;
  int slots = cfg->max_slots > 0 ? cfg->max_slots : 256;
  // admission by memory: per-slot state, templates and work-list space must fit the budget
  if (cfg->device_bytes_budget) {
    const uint64_t fit = cfg->device_bytes_budget / slot_bytes(il);
    if (fit == 0) return MLMC_ENOMEM;
    slots = (int)std::min<uint64_t>((uint64_t)slots, fit);
  }
  mlmc_engine *e = new (std::nothrow) mlmc_engine;
  if (!e) return MLMC_ENOMEM;
  e->max_slots = slots;
  e->max_level = cfg->max_level;
  e->il = il;
  e->iters = cfg->iters_per_launch != 0 ? cfg->iters_per_launch : 1;
  e->num_sms = ctx_num_sms();
  const size_t nt = (size_t)slots * il;
  e->cap_chunks = std::max<unsigned long long>(4ULL * nt, 1ULL << 16);
  bool ok = dev_alloc(&e->d_slots, slots) && dev_alloc(&e->d_rep, slots) && dev_alloc(&e->d_tmpl, nt) &&
            dev_alloc(&e->d_run, nt) && dev_alloc(&e->d_meta, nt) && dev_alloc(&e->d_tnch, nt) &&
            dev_alloc(&e->d_run_nch, nt) && dev_alloc(&e->d_run_cb, nt) && dev_alloc(&e->d_run_src, nt) &&
            dev_alloc(&e->d_run_n, nt) && dev_alloc(&e->d_dyn, GMAX) && dev_alloc(&e->d_status, 1) &&
            dev_alloc(&e->d_iter, 1) &&
            dev_alloc(&e->d_partials, e->cap_chunks) &&
            cudaHostAlloc((void **)&e->h_rep, sizeof(SlotReport) * slots, cudaHostAllocDefault) == cudaSuccess &&
            cudaHostAlloc((void **)&e->h_status, sizeof(EngStatus), cudaHostAllocDefault) == cudaSuccess &&
            cudaStreamCreateWithFlags(&e->cs, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) == cudaSuccess;
  if (ok) {
    std::vector<TmplMeta> none(nt);
    for (auto &m : none) { std::memset(&m, 0, sizeof m); m.group = -1; }
    ok = cudaMemset(e->d_slots, 0, sizeof(SlotState) * slots) == cudaSuccess &&
         cudaMemset(e->d_status, 0, sizeof(EngStatus)) == cudaSuccess &&
         cudaMemset(e->d_dyn, 0, sizeof(DynLaunch) * GMAX) == cudaSuccess &&
         cudaMemcpy(e->d_meta, none.data(), sizeof(TmplMeta) * nt, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (!ok) {
    release(e);
    delete e;
    return MLMC_ENOMEM;
  }
  std::memset(e->h_status, 0, sizeof(EngStatus));
  e->slot_req.assign(slots, -1);
  e->slot_groups.assign(slots, {});
  *out = e;
  return MLMC_OK;
}

mlmc_status mlmc_engine_submit(mlmc_engine *e, const mlmc_params *p, double eps, int mode, uint64_t seed,
                               uint64_t *req_id) {
  MLMC_API_LOCK();
  int ne, v[2];
  if (!e || !p || !req_id || !params_ok(p) || !(eps > 0.0) || !std::isfinite(eps) || !mode_variants(mode, ne, v))
    return MLMC_EINVAL;
  if (p->formats && p->n_formats <= e->max_level) return MLMC_EINVAL;
  Request r;
  r.id = e->next_id++;
  r.p = *p;
  if (p->formats) {
    r.formats.assign(p->formats, p->formats + p->n_formats);
  }
  r.eps = eps;
  r.mode = mode;
  r.seed = seed;
  r.t_submit = now_s();
  r.t_admit = r.t_done = 0.0;
  r.slot = -1;
  r.done = 0;
  r.status = MLMC_OK;
  r.price = r.se = 0.0;
  r.L = 0;
  r.exact_mask = exact_mask_of(mode, p->icdf_bits);
  e->reqs.push_back(std::move(r));
  const size_t idx = e->reqs.size() - 1;
  e->by_id[e->reqs[idx].id] = idx;
  e->queue.push_back(idx);
  *req_id = e->reqs[idx].id;
  return MLMC_OK;
}

mlmc_status mlmc_engine_step(mlmc_engine *e, void *stream, int *active_out, int *queued_out) {
  MLMC_API_LOCK();
  if (!e) return MLMC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // 1. admit waiting requests into free slots
  for (int sl = 0; sl < e->max_slots && !e->queue.empty(); ++sl) {
    if (e->slot_req[sl] >= 0) continue;
    const size_t idx = e->queue.front();
    e->queue.pop_front();
    Request &r = e->reqs[idx];
    const mlmc_status s = admit(e, sl, idx, st);
    if (s != MLMC_OK) {
      // the request cannot run (for instance a format its constants do not fit):
      // it completes with this status and the slot stays free
      r.done = 1;
      r.status = s;
      r.price = r.se = std::nan("");
      r.t_done = now_s();
      e->completed.push_back(r.id);
      if (s == MLMC_ECUDA) return s;
      --sl;
      continue;
    }
    e->slot_req[sl] = (int)idx;
    r.slot = sl;
    r.t_admit = now_s();
  }
  int running = 0;
  for (int sl = 0; sl < e->max_slots; ++sl) running += e->slot_req[sl] >= 0;
  // 2. one graph launch: `iters` iterations of every active slot's pending work
  if (running > 0) {
    for (int attempt = 0;; ++attempt) {
      if (e->dirty) {
        const mlmc_status s = capture(e);
        if (s != MLMC_OK) return s;
      }
      if (e->iters < 0) MLMC_CK(cudaMemsetAsync(e->d_iter, 0, sizeof(uint32_t), st));
      MLMC_CK(cudaGraphLaunch(e->exec, st));
      MLMC_CK(cudaStreamSynchronize(st));
      e->launches += 1;
      if (!e->h_status->overflow) break;
      if (attempt >= 4) return MLMC_ENOMEM;
      // more chunks than the partial array holds: grow it and run the iteration again
      const unsigned long long need = std::max(2 * e->h_status->chunks, 2 * e->cap_chunks);
      cudaFree(e->d_partials);
      e->d_partials = nullptr;
      if (!dev_alloc(&e->d_partials, need)) return MLMC_ENOMEM;
      e->cap_chunks = need;
      e->dirty = true;
    }
    e->path_steps = e->h_status->path_steps;
    // 3. completed requests leave their slots
    const double t = now_s();
    for (int sl = 0; sl < e->max_slots; ++sl) {
      const int idx = e->slot_req[sl];
      if (idx < 0) continue;
      const SlotReport &hr = e->h_rep[sl];
      Request &r = e->reqs[idx];
      if (hr.done && !r.done) {
        r.done = 1;
        r.price = hr.price;
        r.se = hr.se;
        r.L = hr.L;
        r.rem = hr.rem;
        r.t_done = t;
        e->completed.push_back(r.id);
        // the request's schedule, read before the slot is cleared (the launch
        // has finished: its stream was synchronised above)
        r.N.assign((size_t)MAXL * 2, 0);
        MLMC_CK(cudaMemcpy(r.N.data(), &e->d_slots[sl].N[0][0], sizeof(unsigned long long) * MAXL * 2,
                           cudaMemcpyDeviceToHost));
        SlotState z;
        std::memset(&z, 0, sizeof z);
        MLMC_CK(cudaMemcpyAsync(e->d_slots + sl, &z, sizeof z, cudaMemcpyHostToDevice, st));
        free_slot_groups(e, sl);
        e->slot_req[sl] = -1;
      }
    }
  }
  e->steps += 1;
  if (active_out) {
    int a = 0;
    for (int sl = 0; sl < e->max_slots; ++sl) a += e->slot_req[sl] >= 0;
    *active_out = a;
  }
  if (queued_out) *queued_out = (int)e->queue.size();
  return MLMC_OK;
}

mlmc_status mlmc_engine_poll(mlmc_engine *e, uint64_t req_id, double *price, double *stderr_out, int *L,
                             int *done, double *latency_s) {
  MLMC_API_LOCK();
  if (!e) return MLMC_EINVAL;
  auto it = e->by_id.find(req_id);
  if (it == e->by_id.end()) return MLMC_EINVAL;
  const Request &r = e->reqs[it->second];
  if (done) *done = r.done;
  if (r.done) {
    if (price) *price = r.price;
    if (stderr_out) *stderr_out = r.se;
    if (L) *L = r.L;
    if (latency_s) *latency_s = r.t_done - r.t_submit;
  }
  return r.status;
}

mlmc_status mlmc_engine_completed(mlmc_engine *e, uint64_t *ids, int cap, int *n) {
  MLMC_API_LOCK();
  if (!e || !n || cap < 0 || (cap > 0 && !ids)) return MLMC_EINVAL;
  int k = 0;
  while (k < cap && !e->completed.empty()) {
    ids[k++] = e->completed.front();
    e->completed.pop_front();
  }
  *n = k;
  return MLMC_OK;
}

mlmc_status mlmc_engine_request_info(mlmc_engine *e, uint64_t req_id, uint64_t *N_l, int cap_levels,
                                     double *bias_estimate) {
  MLMC_API_LOCK();
  if (!e || cap_levels < 0 || (cap_levels > 0 && !N_l)) return MLMC_EINVAL;
  auto it = e->by_id.find(req_id);
  if (it == e->by_id.end()) return MLMC_EINVAL;
  const Request &r = e->reqs[it->second];
  if (!r.done) return MLMC_ENOTREADY;
  if (r.status != MLMC_OK) return r.status;
  for (int l = 0; l < cap_levels; ++l)
    for (int k = 0; k < 2; ++k)
      N_l[2 * l + k] = (l < MAXL && l <= r.L && !r.N.empty()) ? r.N[(size_t)l * 2 + k] : 0;
  if (bias_estimate) *bias_estimate = r.rem;
  return MLMC_OK;
}

mlmc_status mlmc_engine_stats(const mlmc_engine *e, uint64_t *steps, uint64_t *launches, uint64_t *path_steps,
                              int *slots) {
  MLMC_API_LOCK();
  if (!e) return MLMC_EINVAL;
  if (steps) *steps = e->steps;
  if (launches) *launches = e->launches;
  if (path_steps) *path_steps = e->path_steps;
  if (slots) *slots = e->max_slots;
  return MLMC_OK;
}

mlmc_status mlmc_engine_graph_info(const mlmc_engine *e, int *groups, int *captures, int *iters_per_launch,
                                   uint64_t *partial_capacity) {
  MLMC_API_LOCK();
  if (!e) return MLMC_EINVAL;
  if (groups) {
    int n = 0;
    for (const Group &G : e->groups) n += G.in_graph;
    *groups = n;
  }
  if (captures) *captures = (int)e->captures;
  if (iters_per_launch) *iters_per_launch = e->iters;
  if (partial_capacity) *partial_capacity = e->cap_chunks;
  return MLMC_OK;
}

void mlmc_engine_destroy(mlmc_engine *e) {
  MLMC_API_LOCK();
  if (!e) return;
  if (e->cs) cudaStreamSynchronize(e->cs);
  release(e);
  delete e;
}

mlmc_status mlmc_batch_estimate(const mlmc_params *params, const double *eps, int n, int mode, uint64_t seed,
                                int max_level, int iters_per_launch, double *price, double *stderr_out, int *L,
                                int *launches, void *stream) {
  MLMC_API_LOCK();
  if (!params || !eps || n <= 0 || !price) return MLMC_EINVAL;
  mlmc_engine_config cfg;
  std::memset(&cfg, 0, sizeof cfg);
  cfg.max_slots = n;
  cfg.max_level = max_level;
  cfg.iters_per_launch = iters_per_launch;
  mlmc_engine *e = nullptr;
  mlmc_status s = mlmc_engine_create(&e, &cfg);
  if (s != MLMC_OK) return s;
  std::vector<uint64_t> ids(n);
  for (int i = 0; i < n && s == MLMC_OK; ++i) s = mlmc_engine_submit(e, &params[i], eps[i], mode, seed, &ids[i]);
  int active = 1, queued = 1;
  for (int k = 0; s == MLMC_OK && (active > 0 || queued > 0); ++k) {
    if (k >= 100000) { s = MLMC_ETIMEOUT; break; }
    s = mlmc_engine_step(e, stream, &active, &queued);
  }
  for (int i = 0; i < n && s == MLMC_OK; ++i) {
    int done = 0;
    s = mlmc_engine_poll(e, ids[i], &price[i], stderr_out ? &stderr_out[i] : nullptr, L ? &L[i] : nullptr, &done,
                         nullptr);
    if (s == MLMC_OK && !done) s = MLMC_ETIMEOUT;
  }
  if (launches) *launches = (int)e->launches;
  mlmc_engine_destroy(e);
  return s;
}

}  // extern "C"
