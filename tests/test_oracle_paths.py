"""Pins of the oracle's path simulation, payoffs and estimators against closed forms
and invariants of the method."""
import math

import numpy as np
import pytest
from scipy.stats import norm

from oracle import core, driver
from paper_2502_07123_gb300 import workloads as W


def black_scholes_call(S0, K, r, sig, T):
    d1 = (math.log(S0 / K) + (r + 0.5 * sig * sig) * T) / (sig * math.sqrt(T))
    d2 = d1 - sig * math.sqrt(T)
    return S0 * norm.cdf(d1) - K * math.exp(-r * T) * norm.cdf(d2)


def black_scholes_digital(S0, K, r, sig, T):
    d2 = (math.log(S0 / K) + (r - 0.5 * sig * sig) * T) / (sig * math.sqrt(T))
    return math.exp(-r * T) * norm.cdf(d2)


def test_black_scholes_reference_values():
    # textbook values for the paper's test case at the money
    assert abs(black_scholes_call(100, 100, 0.05, 0.2, 1) - 10.450583572185565) < 1e-9
    assert abs(black_scholes_digital(100, 100, 0.05, 0.2, 1) - 0.5323248154537634) < 1e-9


@pytest.mark.parametrize("scheme", [W.EULER, W.MILSTEIN])
def test_mean_terminal_value_closed_form(scheme):
    """E[Z] = 0 (and E[Z^2 - 1] = 0) give E[S_N] = S0 (1 + r h)^N exactly for both schemes;
    the coarse path has E[S^c] = S0 (1 + 2 r h)^(N/2)."""
    p = W.params(scheme=scheme, sigma=0.3)
    lev, N = 3, 40_000
    _, dump = core.level(p, lev, 0, N, core.FP64_EXACT, 17, dump=True)
    h = p["T"] / 2**lev
    for col, ref in (("sf", p["S0"] * (1 + p["r"] * h) ** 8), ("sc", p["S0"] * (1 + 2 * p["r"] * h) ** 4)):
        x = dump[col]
        se = x.std() / math.sqrt(N)
        assert abs(x.mean() - ref) < 4 * se, (col, x.mean(), ref, se)


@pytest.mark.parametrize("scheme,lo,hi", [(W.EULER, -1.3, -0.7), (W.MILSTEIN, -2.4, -1.6)])
def test_level_variance_decay(scheme, lo, hi):
    """V_l = Var[P_l - P_{l-1}] decays like h (Euler-Maruyama) or h^2 (Milstein) for the call."""
    p = W.params(scheme=scheme)
    V = []
    for lev in range(2, 7):
        s, _ = core.level(p, lev, 0, 20_000, core.FP64_EXACT, 11)
        m = s["sum"] / s["n"]
        V.append(s["sum2"] / s["n"] - m * m)
    slope = np.polyfit(np.arange(2, 7), np.log2(V), 1)[0]
    assert lo < slope < hi


def test_telescoping_sum_matches_finest_level():
    """eq. classic_MLMC_iden: sum_l E[P_l - P_{l-1}] = E[P_L], by independent estimates."""
    p = W.params()
    L, N = 4, 40_000
    tot, var = 0.0, 0.0
    for lev in range(L + 1):
        s, _ = core.level(p, lev, 0, N, core.FP64_EXACT, 100 + lev)
        m = s["sum"] / N
        tot += m
        var += (s["sum2"] / N - m * m) / N
    _, dump = core.level(p, L, 0, N, core.FP64_EXACT, 999, dump=True)
    direct = dump["pf"].mean()
    var += dump["pf"].var() / N
    assert abs(tot - direct) < 4 * math.sqrt(var)


def test_nested_coupling_shares_uniforms():
    """The correction sample uses the same J for its exact and approximate paths (Sec. 3):
    its exact part equals the plain exact sample and its approximate part the approximate
    sample drawn from the same stream."""
    p = W.params(payoff=W.ASIAN)
    lev = 3
    fmt = W.default_format(p, lev)
    _, corr = core.level(p, lev, 50, 300, core.CORR_FIXED, 5, fmt=fmt, dump=True)
    _, ex = core.level(p, lev, 50, 300, core.FP64_EXACT, 5, stream=0, dump=True)
    _, ap = core.level(p, lev, 50, 300, core.FIXED_APPROX, 5, stream=0, fmt=fmt, dump=True)
    assert np.array_equal(corr["pf"], ex["pf"]) and np.array_equal(corr["pc"], ex["pc"])
    assert np.array_equal(corr["qf"], ap["qf"]) and np.array_equal(corr["qc"], ap["qc"])
    unit = fmt["f"][6] + lev + 1
    y_nested = corr["y"] + (ap["qf"] - ap["qc"]) * 2.0**-unit
    assert np.allclose(y_nested, ex["pf"] - ex["pc"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("variant", [core.FIXED_APPROX, core.FP16_APPROX])
def test_approximate_path_tracks_exact_path(variant):
    """With shared uniforms the low-precision path stays close to the exact path:
    |S~ - S| is small relative to S (the error is driven by the table MSE and rounding)."""
    p = W.params()
    lev = 4
    fmt = W.default_format(p, lev)
    _, ap = core.level(p, lev, 0, 2000, variant, 8, stream=0, fmt=fmt, dump=True)
    _, ex = core.level(p, lev, 0, 2000, core.FP64_EXACT, 8, stream=0, dump=True)
    rel = np.abs(ap["af"] - ex["sf"]) / ex["sf"]
    assert np.median(rel) < (2e-3 if variant == core.FIXED_APPROX else 1e-2)
    assert np.max(rel) < 0.05


def test_nested_estimator_expectation():
    """eq. chap:nested_exp: E[dP~] + E[dP - dP~] = E[dP], checked with independent samples."""
    p = W.params()
    lev = 3
    fmt = W.default_format(p, lev)
    N = 40_000
    sa, _ = core.level(p, lev, 0, N, core.FIXED_APPROX, 21, fmt=fmt)
    sc, _ = core.level(p, lev, 0, N, core.CORR_FIXED, 21, fmt=fmt)
    se_, _ = core.level(p, lev, 0, N, core.FP64_EXACT, 22)
    ma, mc, me = sa["sum"] / N, sc["sum"] / N, se_["sum"] / N
    va = sa["sum2"] / N - ma * ma
    vc = sc["sum2"] / N - mc * mc
    ve = se_["sum2"] / N - me * me
    assert abs(ma + mc - me) < 4 * math.sqrt((va + vc + ve) / N)
    assert vc < 0.05 * va      # the correction has a far smaller variance (Sec. 2.2)


@pytest.mark.parametrize("payoff,bs", [(W.EURO, black_scholes_call), (W.DIGITAL, black_scholes_digital)])
def test_adaptive_mlmc_black_scholes(payoff, bs):
    p = W.params(payoff=payoff)
    eps = 0.05 if payoff == W.EURO else 0.01
    res = driver.mlmc(eps, p, 2024, mode=driver.PLAIN_FP64, L_min=2, N_init=2000)
    ref = bs(p["S0"], p["K"], p["r"], p["sigma"], p["T"])
    # variance <= eps^2/2 and bias <= eps/sqrt(2) by construction; 3 standard errors + bias
    assert abs(res["price"] - ref) < 3 * math.sqrt(res["var"]) + eps / math.sqrt(2)
    assert res["var"] <= 0.5 * eps * eps * 1.0001


def test_adaptive_nested_mlmc_black_scholes():
    p = W.params()
    eps = 0.05
    res = driver.mlmc(eps, p, 77, mode=driver.NESTED_FIXED, L_min=2, N_init=2000,
                      cost={core.FIXED_APPROX: 0.4, core.CORR_FIXED: 1.4},
                      fmt_of_level=lambda lev: W.default_format(p, lev))
    ref = black_scholes_call(p["S0"], p["K"], p["r"], p["sigma"], p["T"])
    assert abs(res["price"] - ref) < 3 * math.sqrt(res["var"]) + eps / math.sqrt(2)
    # far more approximate than correction samples on the coarse levels (Sec. 2.2)
    assert res["N"][0][0] > 5 * res["N"][0][1]


def test_adaptive_nested_exact_low_levels_black_scholes():
    """Mode with the approximate terms of levels 0-1 computed by enumeration."""
    p = W.params()
    eps = 0.05
    res = driver.mlmc(eps, p, 77, mode=driver.NESTED_FIXED_EXACT_LOW, N_init=2000,
                      cost={core.FIXED_APPROX: 0.9, core.CORR_FIXED: 1.9},
                      fmt_of_level=lambda lev: W.default_format(p, lev))
    ref = black_scholes_call(p["S0"], p["K"], p["r"], p["sigma"], p["T"])
    assert abs(res["price"] - ref) < 3 * math.sqrt(res["var"]) + eps / math.sqrt(2)
    assert res["N"][0][0] == 1 << 10 and res["N"][1][0] == 1 << 20


# ---------------------------------------------------------------------------
# Exact-path Asian and lookback payoffs.  These payoffs come from the workload
# configurations, not from the paper, and have no closed form for the price
# under Euler-Maruyama in general; each pin below is a case the mathematics
# fixes: means that E[Z] = 0 and E[Z^2 - 1] = 0 determine, deterministic paths,
# and the first two levels, whose expectations reduce to one-dimensional
# integrals of the Normal density.
# ---------------------------------------------------------------------------
def _call_on_normal(mu, s):
    """E[(mu + s Z)^+] for a standard Normal Z."""
    return mu * norm.cdf(mu / s) + s * norm.pdf(mu / s)


def _put_on_normal(k, mu, s):
    """E[(k - (mu + s Z))^+]."""
    return (k - mu) * norm.cdf((k - mu) / s) + s * norm.pdf((k - mu) / s)


def _trapezoid_mean(S0, a, n):
    """E of the trapezoidal average over n steps of a path with E[S_i] = S0 a^i."""
    return (0.5 * S0 + sum(S0 * a**i for i in range(1, n)) + 0.5 * S0 * a**n) / n


@pytest.mark.parametrize("scheme", [W.EULER, W.MILSTEIN])
@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_asian_average_mean_closed_form(scheme, level):
    """With K = 0 the Asian payoff is the trapezoidal average itself, whose mean is
    fixed by E[S_i] = S0 (1 + r h)^i on the fine grid and S0 (1 + 2 r h)^k on the
    coarse one (both schemes).  A wrong end weight or a dropped inner point moves
    the mean by S0 / (2n) or more, far beyond four standard errors."""
    p = W.params(payoff=W.ASIAN, scheme=scheme, K=0.0, sigma=0.3)
    N = 40_000
    _, dump = core.level(p, level, 0, N, core.FP64_EXACT, 41 + level, dump=True)
    n, h = 2**level, p["T"] / 2**level
    ref_f = _trapezoid_mean(p["S0"], 1 + p["r"] * h, n)
    se = dump["pf"].std() / math.sqrt(N)
    assert abs(dump["pf"].mean() - ref_f) < 4 * se, (dump["pf"].mean(), ref_f, se)
    if level > 0:
        ref_c = _trapezoid_mean(p["S0"], 1 + 2 * p["r"] * h, n // 2)
        se = dump["pc"].std() / math.sqrt(N)
        assert abs(dump["pc"].mean() - ref_c) < 4 * se, (dump["pc"].mean(), ref_c, se)
    else:
        assert np.all(dump["pc"] == 0.0)


@pytest.mark.parametrize("level", [0, 1, 3, 5])
@pytest.mark.parametrize("r", [0.05, -0.05])
def test_deterministic_paths_asian_and_lookback(level, r):
    """sigma = 0: S_i = S0 (1 + r h)^i exactly, so the average, the minimum (S0 when
    r > 0, S_N when r < 0) and both payoffs have closed forms on each grid."""
    n, T, S0 = 2**level, 1.0, 100.0
    h = T / n
    a, ac = 1 + r * h, 1 + 2 * r * h
    for K in (95.0, 105.0):
        p = W.params(payoff=W.ASIAN, sigma=0.0, r=r, K=K)
        _, dump = core.level(p, level, 0, 8, core.FP64_EXACT, 3, dump=True)
        ref_f = max(_trapezoid_mean(S0, a, n) - K, 0.0)
        assert np.allclose(dump["pf"], ref_f, rtol=1e-12, atol=1e-12)
        if level > 0:
            assert np.allclose(dump["pc"], max(_trapezoid_mean(S0, ac, n // 2) - K, 0.0), rtol=1e-12, atol=1e-12)
    p = W.params(payoff=W.LOOKBACK, sigma=0.0, r=r)
    _, dump = core.level(p, level, 0, 8, core.FP64_EXACT, 3, dump=True)
    ref_f = S0 * (a**n - 1) if r > 0 else 0.0
    assert np.allclose(dump["pf"], ref_f, rtol=1e-12, atol=1e-12)
    if level > 0:
        ref_c = S0 * (ac ** (n // 2) - 1) if r > 0 else 0.0
        assert np.allclose(dump["pc"], ref_c, rtol=1e-12, atol=1e-12)


def test_lookback_level0_is_call_struck_at_S0():
    """One step: S_1 - min(S0, S_1) = max(S_1 - S0, 0) sample by sample, with mean
    S0 E[(r T + sigma sqrt(T) Z)^+] (Euler-Maruyama)."""
    p = W.params(payoff=W.LOOKBACK, sigma=0.3)
    N = 100_000
    _, dump = core.level(p, 0, 0, N, core.FP64_EXACT, 5, dump=True)
    assert np.array_equal(dump["pf"], np.maximum(dump["sf"] - p["S0"], 0.0))
    ref = p["S0"] * _call_on_normal(p["r"] * p["T"], p["sigma"] * math.sqrt(p["T"]))
    se = dump["pf"].std() / math.sqrt(N)
    assert abs(dump["pf"].mean() - ref) < 4 * se


def test_level1_asian_and_lookback_by_quadrature():
    """Level 1 (two fine steps, one coarse step), Euler-Maruyama: with
    a_i = 1 + r h + sigma sqrt(h) Z_i the fine payoffs are functions of (a_1, a_2)
    that are linear in a_2 for fixed a_1, so their means are one-dimensional
    integrals over Z_1 of closed-form Normal expectations; the coarse step has
    a_c = 1 + r T + sigma sqrt(T) Z'."""
    from scipy.integrate import quad
    S0, K, r, sig, T = 100.0, 100.0, 0.05, 0.3, 1.0
    h = T / 2
    mu, s = 1 + r * h, sig * math.sqrt(h)
    N = 100_000

    def over_z1(f):
        return quad(lambda z: f(mu + s * z) * norm.pdf(z), -9, 9, epsabs=1e-12, epsrel=1e-12, limit=400)[0]

    # lookback: S0 E[a1 a2 - min(1, a1, a1 a2)]; E[min(m, a1 a2)] = m - a1 E[(m / a1 - a2)^+]
    def lb_inner(a1):
        m = min(1.0, a1)
        return m - a1 * _put_on_normal(m / a1, mu, s)
    lb_f = S0 * (mu * mu - over_z1(lb_inner))
    lb_c = S0 * _call_on_normal(r * T, sig * math.sqrt(T))
    # Asian: average (S0/2 + S1 + S2/2) / 2 - K = A + B a2 with B = S0 a1 / 4
    def as_inner(a1):
        A, B = S0 * (0.5 + a1) / 2 - K, S0 * a1 / 4
        return B * _call_on_normal(A / B + mu, s)
    as_f = over_z1(as_inner)
    as_c = 0.5 * S0 * _call_on_normal(2 + r * T - 2 * K / S0, sig * math.sqrt(T))
    for payoff, rf, rc in ((W.LOOKBACK, lb_f, lb_c), (W.ASIAN, as_f, as_c)):
        p = W.params(payoff=payoff, sigma=sig, K=K)
        _, dump = core.level(p, 1, 0, N, core.FP64_EXACT, 9 + payoff, dump=True)
        for col, ref in (("pf", rf), ("pc", rc)):
            x = dump[col]
            se = x.std() / math.sqrt(N)
            assert abs(x.mean() - ref) < 4 * se, (payoff, col, x.mean(), ref, se)
        y = dump["pf"] - dump["pc"]
        assert abs(y.mean() - (rf - rc)) < 4 * y.std() / math.sqrt(N)


def test_lookback_fine_level_discrete_monitoring():
    """Level 6 against the continuously monitored floating-strike lookback
    (Goldman-Sosin-Gatto) with the Broadie-Glasserman-Kou shift of the minimum,
    m_discrete ~ m_continuous exp(beta sigma sqrt(h)), beta = -zeta(1/2)/sqrt(2 pi):
    E[S_N - min] ~ S0 (1 + r h)^N - E[m_cont] exp(beta sigma sqrt(h)).  The tolerance is
    four standard errors plus 8h for the O(h) remainder of the shift and the Euler
    weak error; the minimum over the coarse grid instead of the fine one would be
    off by about 0.5 here, over twice the tolerance."""
    S0, r, sig, T, lev = 100.0, 0.05, 0.2, 1.0, 6
    a1 = (r + sig * sig / 2) * math.sqrt(T) / sig
    a2 = a1 - sig * math.sqrt(T)
    a3 = (-r + sig * sig / 2) * math.sqrt(T) / sig
    price = (S0 * norm.cdf(a1) - S0 * sig * sig / (2 * r) * norm.cdf(-a1)
             - S0 * math.exp(-r * T) * (norm.cdf(a2) - sig * sig / (2 * r) * norm.cdf(-a3)))
    e_min = S0 * math.exp(r * T) - math.exp(r * T) * price     # E[min over [0, T]]
    beta = 0.5825971579390106
    h, n = T / 2**lev, 2**lev
    ref = S0 * (1 + r * h) ** n - e_min * math.exp(beta * sig * math.sqrt(h))
    N = 100_000
    _, dump = core.level(W.params(payoff=W.LOOKBACK), lev, 0, N, core.FP64_EXACT, 3, dump=True)
    se = dump["pf"].std() / math.sqrt(N)
    assert abs(dump["pf"].mean() - ref) < 4 * se + 8 * h, (dump["pf"].mean(), ref, se)
