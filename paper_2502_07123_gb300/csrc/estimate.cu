// The adaptive MLMC driver mlmc_estimate: the Giles (2008) loop to RMS error
// eps, in the form of Giles (2015) that tests the bias once the remaining
// top-ups are small, with the nested variant of Sec. 2.2 (approximate levels
// plus corrections), host-driven over synchronous plans.
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

namespace {

struct EstPlan {
  int n;          // estimators per level
  int variant[2];
  bool exact_low; // approximate terms of levels 0-1 computed exactly by enumeration
};

// Levels whose approximate level difference is a finite sum over 2^(d 2^l) <= 2^20 cells.
constexpr int EXACT_MAX_BITS = 20;
// The bias test runs once every pending top-up is at most this fraction of its
// term's samples (Giles 2015's form of the loop); a bound on the rounds.
constexpr double ALMOST_DONE = 0.01;
constexpr int MAX_ROUNDS = 100000;

bool est_plan(int mode, EstPlan &e) {
  switch (mode) {
    case 0: e = {1, {MLMC_FP64_EXACT, 0}, false}; return true;
    case 1: e = {1, {MLMC_FP32_EXACT, 0}, false}; return true;
    case 2: e = {2, {MLMC_FIXED_APPROX, MLMC_NESTED_CORR_FIXED}, false}; return true;
    case 3: e = {2, {MLMC_FP16_APPROX, MLMC_NESTED_CORR_FP16}, false}; return true;
    case 4: e = {2, {MLMC_BF16_APPROX, MLMC_NESTED_CORR_BF16}, false}; return true;
    case 5: e = {2, {MLMC_FIXED_APPROX, MLMC_NESTED_CORR_FIXED}, true}; return true;
    case 6: e = {2, {MLMC_FP16_APPROX, MLMC_NESTED_CORR_FP16}, true}; return true;
    case 7: e = {2, {MLMC_FP16S_APPROX, MLMC_NESTED_CORR_FP16S}, false}; return true;
    case 8: e = {2, {MLMC_BF16S_APPROX, MLMC_NESTED_CORR_BF16S}, false}; return true;
    case 9: e = {2, {MLMC_FP16S_APPROX, MLMC_NESTED_CORR_FP16S}, true}; return true;
    case 10: e = {2, {MLMC_BF16S_APPROX, MLMC_NESTED_CORR_BF16S}, true}; return true;
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
  // One synchronous round per pass: the pending samples of every term, new
  // optimal counts, and (once every remaining top-up is within ALMOST_DONE of
  // its term's samples) the bias test, which may add a level whose first
  // samples then run in the same round as those top-ups.  The run ends when
  // nothing is pending and the bias test passed (or L = max_level).
  for (int round = 0;; ++round) {
    if (round >= MAX_ROUNDS) return MLMC_ETIMEOUT;
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
    if (!work.empty()) {
      res.resize(work.size());
      // (the rounds' device times are not used: no timing events)
      s = run_sync(work.data(), (int)work.size(), seed, nullptr, nullptr, res.data(), g.st, false, false);
      if (s != MLMC_OK) return s;
      for (size_t j = 0; j < work.size(); ++j) {
        const int l = idx[j].first, k = idx[j].second;
        S1[l][k] += res[j].sum;
        S2[l][k] += res[j].sum2;
        N[l][k] += work[j].N;
      }
    }
    update_dn();
    bool any = false, small = true;
    for (int l = 0; l <= L; ++l)
      for (int k = 0; k < ne; ++k) {
        any |= dN[l][k] > 0;
        small &= !((double)dN[l][k] > ALMOST_DONE * (double)N[l][k]);
      }
    if (!small) continue;
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
    if (rem > std::sqrt(theta) * eps && L < max_level) {
      L += 1;
      N.push_back(std::vector<uint64_t>(ne, 0));
      dN.push_back(std::vector<uint64_t>(ne, 0));
      S1.push_back(std::vector<double>(ne, 0.0));
      S2.push_back(std::vector<double>(ne, 0.0));
      std::vector<double> ve(ne);
      for (int k = 0; k < ne; ++k) ve[k] = std::max(level_var(L - 1, k), 1e-300) / std::pow(2.0, beta);
      Vext.push_back(ve);
      update_dn();
      continue;
    }
    if (!any) break;
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
