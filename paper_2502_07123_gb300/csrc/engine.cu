// Continuous-batching pricing engine: many adaptive (nested) MLMC requests
// share every level-kernel launch.
//
// Each admitted request owns a slot of FP64 state in device memory (sums of Y
// and Y^2, sample counts, pending counts per level and estimator).  One engine
// step gathers the pending (request, level, estimator, count) work of every
// active slot into one batched plan launch; accumulate_kernel then adds the new
// sums into each slot and decide_kernel, on the device, recomputes the level variances, the
// optimal sample counts N = ceil(lambda sqrt(V / C)) (Sec. 2.1 / 2.2) and the
// bias test of the adaptive loop.  The host only moves the pending counts back
// to build the next work list.  The arithmetic, and its order, is that of
// mlmc_estimate, with every floating-point operation rounded separately, so a
// request's result does not depend on which other requests share its launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "host_api.h"
#include "item.h"
#include "mlmc.h"

using namespace mlmc;
using namespace mlmc_host;

namespace {

constexpr int MAXL = 21;

struct SlotState {
  int32_t active, done, L, ne;
  int32_t max_level, exact_mask;       // bit l: the approximate term of level l is exact
  double eps, sqrt_theta_eps, var_target, beta_factor;
  double cost[2];                      // cost per fine path-step of each estimator
  double S1[MAXL][2], S2[MAXL][2];     // discounted sums
  double Vext[MAXL][2];                // extrapolated variance of a level not yet sampled
  unsigned long long N[MAXL][2], dN[MAXL][2];
  double price, se;
};

// What the host reads back after each step.
struct SlotReport {
  int32_t active, done, L, pad;
  unsigned long long dN[MAXL][2];
  double price, se;
};

struct ItemMap {
  int32_t slot, level, est, exact_int, unit, pad;
  double disc;
};

__device__ double u128_to_double_rn(unsigned long long lo, unsigned long long hi) {
  if (hi == 0) return __ull2double_rn(lo);
  const int z = __clzll((long long)hi);
  unsigned long long m = z ? ((hi << z) | (lo >> (64 - z))) : hi;
  const unsigned long long rest = z ? (lo << z) : lo;
  m |= (rest != 0ULL) ? 1ULL : 0ULL;   // sticky bit below the 64 kept bits
  return ldexp(__ull2double_rn(m), 64 - z);
}

__device__ double level_var(const SlotState &s, int l, int k) {
  if (k == 0 && ((s.exact_mask >> l) & 1)) return 0.0;  // an exact mean has no variance
  if (s.N[l][k] == 0) return s.Vext[l][k];
  const double n = __ull2double_rn(s.N[l][k]);
  const double m = __ddiv_rn(s.S1[l][k], n);
  const double v = __dsub_rn(__ddiv_rn(s.S2[l][k], n), __dmul_rn(m, m));
  return v > 0.0 ? v : 0.0;
}

// dN = ceil(lambda sqrt(V/C)) - N over all levels <= L and estimators (mlmc_estimate's update).
// Level variance with the floor V_l >= V_{l-1} / (2 * 2^beta) from level 2 on.
__device__ double floored_var(const SlotState &s, int l, int k, double &vprev) {
  double v = level_var(s, l, k);
  if (l >= 2) v = fmax(v, __ddiv_rn(__dmul_rn(0.5, vprev), s.beta_factor));
  vprev = v;
  return fmax(v, 1e-300);
}

__device__ void update_dn(SlotState &s) {
  double lam = 0.0;
  double vp[2] = {0.0, 0.0};
  for (int l = 0; l <= s.L; ++l)
    for (int k = 0; k < s.ne; ++k) {
      const double V = floored_var(s, l, k, vp[k]);
      const double C = ldexp(s.cost[k], l);
      lam = __dadd_rn(lam, __dsqrt_rn(__dmul_rn(V, C)));
    }
  lam = __ddiv_rn(lam, s.var_target);
  vp[0] = vp[1] = 0.0;
  for (int l = 0; l <= s.L; ++l)
    for (int k = 0; k < s.ne; ++k) {
      const double V = floored_var(s, l, k, vp[k]);
      const double C = ldexp(s.cost[k], l);
      const double x = V > 0.0 ? __dmul_rn(lam, __dsqrt_rn(__ddiv_rn(V, C))) : 0.0;
      const unsigned long long want = (unsigned long long)ceil(fmin(x, 1e18));
      s.dN[l][k] = want > s.N[l][k] ? want - s.N[l][k] : 0ULL;
    }
}

// Add this step's results into the slots (each (slot, level, estimator) appears at most once).
__global__ void accumulate_kernel(SlotState *slots, const ItemMap *map, const DevSums *res, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ItemMap &mp = map[i];
  SlotState &s = slots[mp.slot];
  const DevSums &r = res[i];
  double sum, sum2;
  if (mp.exact_int) {
    sum = __dmul_rn(mp.disc, ldexp(__ll2double_rn(r.isum), -mp.unit));
    sum2 = __dmul_rn(__dmul_rn(mp.disc, mp.disc), ldexp(u128_to_double_rn(r.isum2_lo, r.isum2_hi), -2 * mp.unit));
  } else {
    sum = __dmul_rn(mp.disc, r.dsum);
    sum2 = __dmul_rn(__dmul_rn(mp.disc, mp.disc), r.dsum2);
  }
  s.S1[mp.level][mp.est] = __dadd_rn(s.S1[mp.level][mp.est], sum);
  s.S2[mp.level][mp.est] = __dadd_rn(s.S2[mp.level][mp.est], sum2);
  s.N[mp.level][mp.est] += s.dN[mp.level][mp.est];
}

// Per slot: new sample counts, the bias test, a new level, or completion.
__global__ void decide_kernel(SlotState *slots, SlotReport *rep, int n_slots) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_slots) return;
  SlotState &s = slots[i];
  SlotReport &r = rep[i];
  if (s.active && !s.done) {
    update_dn(s);
    bool any = false;
    for (int l = 0; l <= s.L; ++l)
      for (int k = 0; k < s.ne; ++k) any |= s.dN[l][k] > 0;
    if (!any) {
      // bias estimate from the last two level means (weak order 1), with the
      // floor |m_l| >= |m_{l-1}| / (2 * 2^alpha) from level 2 on
      double mprev = 0.0, mL = 0.0, mL1 = 0.0;
      for (int l = 0; l <= s.L; ++l) {
        double ml = 0.0;
        for (int k = 0; k < s.ne; ++k) ml = __dadd_rn(ml, __ddiv_rn(s.S1[l][k], __ull2double_rn(s.N[l][k])));
        ml = fabs(ml);
        if (l >= 2) ml = fmax(ml, __ddiv_rn(__dmul_rn(0.5, mprev), 2.0));
        if (l == s.L - 1) mL1 = ml;
        if (l == s.L) mL = ml;
        mprev = ml;
      }
      double rem = __ddiv_rn(fabs(mL), 1.0);
      rem = fmax(rem, __ddiv_rn(__ddiv_rn(fabs(mL1), 2.0), 1.0));
      if (rem <= s.sqrt_theta_eps || s.L >= s.max_level) {
        double pr = 0.0, var = 0.0;
        for (int l = 0; l <= s.L; ++l)
          for (int k = 0; k < s.ne; ++k) {
            const double n = __ull2double_rn(s.N[l][k]);
            pr = __dadd_rn(pr, __ddiv_rn(s.S1[l][k], n));
            var = __dadd_rn(var, __ddiv_rn(level_var(s, l, k), n));
          }
        s.price = pr;
        s.se = __dsqrt_rn(var);
        s.done = 1;
      } else {
        const int L = ++s.L;
        for (int k = 0; k < s.ne; ++k) {
          s.N[L][k] = 0; s.dN[L][k] = 0; s.S1[L][k] = 0.0; s.S2[L][k] = 0.0;
          s.Vext[L][k] = __ddiv_rn(fmax(level_var(s, L - 1, k), 1e-300), s.beta_factor);
        }
        update_dn(s);
      }
    }
  }
  r.active = s.active;
  r.done = s.done;
  r.L = s.L;
  for (int l = 0; l < MAXL; ++l) { r.dN[l][0] = s.dN[l][0]; r.dN[l][1] = s.dN[l][1]; }
  r.price = s.price;
  r.se = s.se;
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
  double price, se;
  int L;
  unsigned long long N[MAXL][2];      // samples taken so far (host mirror of the slot's counts)
  int exact_mask;                     // bit l: approximate term of level l computed by enumeration
};

int exact_mask_of(int mode, int d) {
  if (mode != 5 && mode != 6) return 0;
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
    default: return false;
  }
}

}  // namespace

struct mlmc_engine {
  int max_slots = 0, max_level = 10;
  SlotState *d_slots = nullptr;
  SlotReport *d_rep = nullptr;
  ItemMap *d_map = nullptr;
  size_t map_cap = 0;
  std::vector<SlotReport> h_rep;
  std::vector<int> slot_req;                 // slot -> index in reqs, -1 if free
  std::deque<size_t> queue;                  // waiting requests (indices into reqs)
  std::vector<Request> reqs;
  std::map<uint64_t, size_t> by_id;
  uint64_t next_id = 1;
  uint64_t steps = 0, launches = 0, path_steps = 0;
};

extern "C" {

mlmc_status mlmc_engine_create(mlmc_engine **out, const mlmc_engine_config *cfg) {
  if (!out || !cfg || cfg->max_level < 2 || cfg->max_level > MAXL - 1) return MLMC_EINVAL;
  mlmc_status s = ensure_ctx();
  if (s != MLMC_OK) return s;
  int slots = cfg->max_slots > 0 ? cfg->max_slots : 256;
  // admission by memory: the slot table must fit the budget
  if (cfg->device_bytes_budget) {
    const uint64_t per = sizeof(SlotState) + sizeof(SlotReport);
    const uint64_t fit = cfg->device_bytes_budget / per;
    if (fit == 0) return MLMC_ENOMEM;
    slots = (int)std::min<uint64_t>((uint64_t)slots, fit);
  }
  mlmc_engine *e = new (std::nothrow) mlmc_engine;
  if (!e) return MLMC_ENOMEM;
  e->max_slots = slots;
  e->max_level = cfg->max_level;
  if (cudaMalloc(&e->d_slots, sizeof(SlotState) * slots) != cudaSuccess ||
      cudaMalloc(&e->d_rep, sizeof(SlotReport) * slots) != cudaSuccess ||
      cudaMemset(e->d_slots, 0, sizeof(SlotState) * slots) != cudaSuccess) {
    cudaFree(e->d_slots);
    cudaFree(e->d_rep);
    delete e;
    return MLMC_ENOMEM;
  }
  e->h_rep.resize(slots);
  e->slot_req.assign(slots, -1);
  *out = e;
  return MLMC_OK;
}

mlmc_status mlmc_engine_submit(mlmc_engine *e, const mlmc_params *p, double eps, int mode, uint64_t seed,
                               uint64_t *req_id) {
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
  r.price = r.se = 0.0;
  r.L = 0;
  std::memset(r.N, 0, sizeof r.N);
  r.exact_mask = exact_mask_of(mode, p->icdf_bits);
  e->reqs.push_back(std::move(r));
  const size_t idx = e->reqs.size() - 1;
  e->by_id[e->reqs[idx].id] = idx;
  e->queue.push_back(idx);
  *req_id = e->reqs[idx].id;
  return MLMC_OK;
}

mlmc_status mlmc_engine_step(mlmc_engine *e, void *stream, int *active_out, int *queued_out) {
  if (!e) return MLMC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // 1. admit waiting requests into free slots
  for (int sl = 0; sl < e->max_slots && !e->queue.empty(); ++sl) {
    if (e->slot_req[sl] >= 0) continue;
    const size_t idx = e->queue.front();
    e->queue.pop_front();
    Request &r = e->reqs[idx];
    int ne, v[2];
    mode_variants(r.mode, ne, v);
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
    MLMC_CK(cudaMemcpyAsync(e->d_slots + sl, &h, sizeof h, cudaMemcpyHostToDevice, st));
    SlotReport &hr = e->h_rep[sl];
    std::memset(&hr, 0, sizeof hr);
    hr.active = 1;
    hr.L = 2;
    for (int l = 0; l <= 2; ++l)
      for (int k = 0; k < ne; ++k) hr.dN[l][k] = h.dN[l][k];
    e->slot_req[sl] = (int)idx;
    r.slot = sl;
    r.t_admit = now_s();
  }
  // 2. one batched launch over the pending work of every active slot
  std::vector<mlmc_work> work;
  std::vector<ItemMap> map;
  int active = 0;
  for (int sl = 0; sl < e->max_slots; ++sl) {
    const int idx = e->slot_req[sl];
    if (idx < 0) continue;
    Request &r = e->reqs[idx];
    if (r.done) continue;
    ++active;
    int ne, v[2];
    mode_variants(r.mode, ne, v);
    r.p.formats = r.formats.empty() ? nullptr : r.formats.data();
    const SlotReport &hr = e->h_rep[sl];
    for (int l = 0; l <= hr.L; ++l)
      for (int k = 0; k < ne; ++k)
        if (hr.dN[l][k] > 0) {
          mlmc_work w;
          std::memset(&w, 0, sizeof w);
          w.params = &r.p;
          w.level = l;
          w.variant = v[k];
          w.N = hr.dN[l][k];
          w.first_sample = r.N[l][k];
          w.stream = -1;
          w.flags = (k == 0 && ((r.exact_mask >> l) & 1)) ? MLMC_WORK_ENUMERATE : 0;
          work.push_back(w);
          ItemMap m;
          std::memset(&m, 0, sizeof m);
          m.slot = sl;
          m.level = l;
          m.est = k;
          map.push_back(m);
        }
  }
  (void)active;
  if (!work.empty()) {
    // one launch per distinct seed (the key of Philox); requests sharing a seed are
    // told apart by the request id in their counters
    std::map<uint64_t, std::vector<size_t>> by_seed;
    for (size_t i = 0; i < work.size(); ++i) by_seed[e->reqs[e->slot_req[map[i].slot]].seed].push_back(i);
    for (auto &kv : by_seed) {
      const std::vector<size_t> &ix = kv.second;
      std::vector<mlmc_work> w;
      for (size_t i : ix) w.push_back(work[i]);
      mlmc_plan *pl = nullptr;
      mlmc_status s = plan_create_transient(&pl, w.data(), (int)w.size(), kv.first, nullptr);
      if (s != MLMC_OK) return s;
      s = plan_launch_on(pl, st);
      if (s != MLMC_OK) { plan_release(pl); return s; }
      std::vector<ItemMap> m(ix.size());
      for (size_t j = 0; j < ix.size(); ++j) {
        m[j] = map[ix[j]];
        plan_item_scale(pl, (int)j, &m[j].disc, &m[j].unit, &m[j].exact_int);
      }
      if (m.size() > e->map_cap) {
        cudaFree(e->d_map);
        e->d_map = nullptr;
        e->map_cap = std::max(m.size(), 2 * e->map_cap);
        MLMC_CK(cudaMalloc(&e->d_map, sizeof(ItemMap) * e->map_cap));
      }
      MLMC_CK(cudaMemcpyAsync(e->d_map, m.data(), sizeof(ItemMap) * m.size(), cudaMemcpyHostToDevice, st));
      accumulate_kernel<<<(unsigned)((m.size() + 127) / 128), 128, 0, st>>>(e->d_slots, e->d_map,
                                                                            plan_out_device(pl), (int)m.size());
      MLMC_CK(cudaGetLastError());
      MLMC_CK(cudaStreamSynchronize(st));
      plan_release(pl);
      e->launches += 1;
    }
    for (size_t i = 0; i < work.size(); ++i) {
      e->path_steps += work[i].N << work[i].level;
      e->reqs[e->slot_req[map[i].slot]].N[map[i].level][map[i].est] += work[i].N;
    }
  }
  // 3. decisions on the device, pending counts back to the host
  decide_kernel<<<(e->max_slots + 127) / 128, 128, 0, st>>>(e->d_slots, e->d_rep, e->max_slots);
  MLMC_CK(cudaGetLastError());
  MLMC_CK(cudaMemcpyAsync(e->h_rep.data(), e->d_rep, sizeof(SlotReport) * e->max_slots, cudaMemcpyDeviceToHost,
                          st));
  MLMC_CK(cudaStreamSynchronize(st));
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
      r.t_done = t;
      // free the slot
      SlotState z;
      std::memset(&z, 0, sizeof z);
      MLMC_CK(cudaMemcpyAsync(e->d_slots + sl, &z, sizeof z, cudaMemcpyHostToDevice, st));
      e->slot_req[sl] = -1;
    }
  }
  MLMC_CK(cudaStreamSynchronize(st));
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
  return MLMC_OK;
}

mlmc_status mlmc_engine_stats(const mlmc_engine *e, uint64_t *steps, uint64_t *launches, uint64_t *path_steps,
                              int *slots) {
  if (!e) return MLMC_EINVAL;
  if (steps) *steps = e->steps;
  if (launches) *launches = e->launches;
  if (path_steps) *path_steps = e->path_steps;
  if (slots) *slots = e->max_slots;
  return MLMC_OK;
}

void mlmc_engine_destroy(mlmc_engine *e) {
  if (!e) return;
  cudaFree(e->d_slots);
  cudaFree(e->d_rep);
  cudaFree(e->d_map);
  delete e;
}

}  // extern "C"
