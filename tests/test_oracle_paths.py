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
