// Offline bit-width optimisation of the fixed-point path of one level
// (Sec. 4-6), host code.
//
// Error model (Sec. 4.2): V_indep(d) = 1/12 sum_t A_t 4^(e_t - d_t) (eq.
// optimistic), V_corr(d) = (sum_t B_t 2^(e_t - d_t - 1))^2 (eq. pessimistic),
// for the variable types t = Z, con1, con2, mul1, sum1, mul2, S of
// Algorithm 1 with exponents e_t (|x| < 2^e_t) and bit-widths d_t.
// Cost model (Sec. 5, eq. cost_sq): C~(d) = steps (1/2 sum_t M_t d_t^2 +
// sum_t M'_t d_t) per sample, steps = fine + coarse steps; the exact sample
// costs C = 2^l c_rng.  Level cost (eq. level_cost2):
// F(d) = sqrt(V C~(d)) + sqrt(V_indep(d) C).
// Lagrange solve (Sec. 6.1, eq. Lagr): for a multiplier lambda every d_t is
// the root of (ln 4 / 12) A_t 4^(e_t - d_t) = lambda steps (M_t d_t + M'_t);
// a golden-section search over log(lambda) minimises F(d(lambda)).
// Integer rounding (Sec. 6.2): round down, then add one bit at a time to the
// variable with the largest variance decrease per unit cost (eq. ratio_lagr)
// until V_indep is at or below the real solution's.
// Table size (Sec. 4.3, eq. extended): the smallest d_lut whose term
// A_Z MSE(d_lut) does not exceed V_indep of the integer widths (the 1/12 of
// the printed formula belongs to the uniform rounding model and is not
// applied to a mean square error).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "mlmc.h"

namespace {

constexpr int NV = 7;
constexpr double D_LO = 1.0, D_HI = 60.0;
// operands per time step of Algorithm 1 (mul1 = con2 Z, sum1 = con1 + mul1,
// mul2 = S sum1, S = S + mul2), variable order Z, con1, con2, mul1, sum1, mul2, S
const double kMul[NV] = {1, 0, 1, 0, 1, 0, 1};
const double kAdd[NV] = {0, 1, 0, 1, 0, 1, 1};

struct Model {
  double A[NV], B[NV], M[NV], Mp[NV];
  int e[NV];
  double steps, V, C;

  double vind(const double *d) const {
    double s = 0.0;
    for (int t = 0; t < NV; ++t) s += A[t] * std::exp2(2.0 * (e[t] - d[t]));
    return s / 12.0;
  }
  double vcorr(const double *d) const {
    double s = 0.0;
    for (int t = 0; t < NV; ++t) s += B[t] * std::exp2((double)e[t] - d[t] - 1.0);
    return s * s;
  }
  double cost(const double *d) const {
    double s = 0.0;
    for (int t = 0; t < NV; ++t) s += 0.5 * M[t] * d[t] * d[t] + Mp[t] * d[t];
    return steps * s;
  }
  double level_cost(const double *d) const { return std::sqrt(V * cost(d)) + std::sqrt(vind(d) * C); }

  // d_t(lambda): the decreasing left side meets the increasing right side once
  void widths(double lambda, double *d) const {
    const double k = std::log(4.0) / 12.0;
    for (int t = 0; t < NV; ++t) {
      auto g = [&](double x) { return k * A[t] * std::exp2(2.0 * (e[t] - x)) - lambda * steps * (M[t] * x + Mp[t]); };
      if (g(D_LO) <= 0.0) { d[t] = D_LO; continue; }
      if (g(D_HI) >= 0.0) { d[t] = D_HI; continue; }
      double lo = D_LO, hi = D_HI;
      while (hi - lo > 1e-12) {
        const double mid = 0.5 * (lo + hi);
        (g(mid) > 0.0 ? lo : hi) = mid;
      }
      d[t] = 0.5 * (lo + hi);
    }
  }
  double cost_at_loglambda(double x) const {
    double d[NV];
    widths(std::exp(x), d);
    return level_cost(d);
  }
};

int exponent_of(double maxabs) {
  if (!(maxabs > 0.0)) return 0;
  return (int)std::floor(std::log2(maxabs)) + 1;
}

}  // namespace

extern "C" mlmc_status mlmc_optimise_level(int level, const mlmc_sensitivity *s, const mlmc_opt_config *cfg,
                                           mlmc_opt_result *out) {
  if (!s || !out || level < 0 || level > 20 || !(s->var > 0.0)) return MLMC_EINVAL;
  mlmc_opt_config c;
  std::memset(&c, 0, sizeof c);
  if (cfg) c = *cfg;
  if (c.lut_max_bits < 0 || c.lut_max_bits > 16) return MLMC_EINVAL;
  Model md;
  bool any_op = false;
  for (int t = 0; t < NV; ++t) any_op |= c.mul[t] != 0.0 || c.add[t] != 0.0;
  for (int t = 0; t < NV; ++t) {
    if (!(s->A[t] >= 0.0) || !(s->B[t] >= 0.0) || !(s->maxabs[t] >= 0.0)) return MLMC_EINVAL;
    md.A[t] = s->A[t];
    md.B[t] = s->B[t];
    md.e[t] = exponent_of(s->maxabs[t]);
    md.M[t] = any_op ? c.mul[t] : kMul[t];
    md.Mp[t] = any_op ? c.add[t] : kAdd[t];
    if (md.M[t] < 0.0 || md.Mp[t] < 0.0) return MLMC_EINVAL;
  }
  const int n = 1 << level;
  md.steps = n + (level > 0 ? n / 2 : 0);
  md.V = s->var;
  md.C = std::ldexp(c.c_rng > 0.0 ? c.c_rng : 1e4, level);
  // golden-section search over log(lambda)
  const double gr = (std::sqrt(5.0) - 1.0) / 2.0;
  double a = std::log(1e-40), b = std::log(1e10);
  double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
  double f1 = md.cost_at_loglambda(x1), f2 = md.cost_at_loglambda(x2);
  for (int it = 0; it < 200; ++it) {
    if (f1 <= f2) {
      b = x2; x2 = x1; f2 = f1;
      x1 = b - gr * (b - a);
      f1 = md.cost_at_loglambda(x1);
    } else {
      a = x1; x1 = x2; f1 = f2;
      x2 = a + gr * (b - a);
      f2 = md.cost_at_loglambda(x2);
    }
  }
  const double lambda = std::exp(0.5 * (a + b));
  double dr[NV], di[NV];
  md.widths(lambda, dr);
  // greedy integer rounding
  const double target = md.vind(dr);
  for (int t = 0; t < NV; ++t) di[t] = std::floor(dr[t]);
  for (int guard = 0; md.vind(di) > target && guard < 64 * NV; ++guard) {
    const double v0 = md.vind(di), c0 = md.cost(di);
    int bt = 0;
    double best = -1.0;
    for (int t = 0; t < NV; ++t) {
      di[t] += 1.0;
      const double r = (v0 - md.vind(di)) / (md.cost(di) - c0);
      di[t] -= 1.0;
      if (r > best) { best = r; bt = t; }
    }
    di[bt] += 1.0;
  }
  std::memset(out, 0, sizeof *out);
  for (int t = 0; t < NV; ++t) {
    out->e[t] = md.e[t];
    out->d[t] = (int32_t)di[t];
    out->d_real[t] = dr[t];
    out->format.e[t] = (int8_t)md.e[t];
    out->format.f[t] = (int8_t)std::max(0, (int)di[t] - md.e[t]);
  }
  out->lambda = lambda;
  out->v_indep_real = target;
  out->v_indep = md.vind(di);
  out->v_corr = md.vcorr(di);
  out->cost_lp = md.cost(di);
  out->cost_exact = md.C;
  out->level_cost_ratio = std::sqrt(out->cost_lp / md.C) + std::sqrt(out->v_indep / md.V);
  out->lut_bits = 0;
  out->mse_term = 0.0;
  if (c.lut_mse) {
    const int top = c.lut_max_bits > 0 ? c.lut_max_bits : 16;
    for (int dl = 2; dl <= top; ++dl)
      if (s->A[0] * c.lut_mse[dl] <= out->v_indep) {
        out->lut_bits = dl;
        out->mse_term = s->A[0] * c.lut_mse[dl];
        break;
      }
  }
  return MLMC_OK;
}

static_assert(sizeof(mlmc_sensitivity) == 200, "mlmc_sensitivity layout");
static_assert(sizeof(mlmc_opt_config) == 136, "mlmc_opt_config layout");
static_assert(sizeof(mlmc_opt_result) == 200, "mlmc_opt_result layout");
