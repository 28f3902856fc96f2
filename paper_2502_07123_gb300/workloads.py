"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds inputs only: market parameters, level / sample-count
schedules, seeds and the per-level fixed-point format tables (bit widths).
It contains none of the method's arithmetic (no random-number generation,
inverse CDF, path step, payoff or sum), so that the CUDA path and the CPU
oracle can both take their inputs from here without sharing any computation.

Market parameters follow the paper's test case (European call on GBM with
r = 0.05, sigma = 0.2, T = 1, Sec. 4.4) with S0 = K = 100.
"""
import math

import numpy as np

# payoff / scheme / variant codes (same numbering as include/mlmc.h)
EURO, DIGITAL, ASIAN, LOOKBACK = 0, 1, 2, 3
EULER, MILSTEIN = 0, 1
FP64_EXACT, FP32_EXACT, FP16_APPROX, BF16_APPROX, FIXED_APPROX, CORR_FIXED, CORR_FP16, CORR_BF16 = range(8)
# binary16 / bfloat16 increments with S in FP32
FP16S_APPROX, BF16S_APPROX, CORR_FP16S, CORR_BF16S = range(8, 12)

# Fixed-point variable order of Algorithm 1
FORMAT_VARS = ("Z", "con1", "con2", "mul1", "sum1", "mul2", "S")

#: the paper's GBM test case (Sec. 4.4), at the money
GBM = dict(S0=100.0, K=100.0, r=0.05, sigma=0.2, T=1.0, payoff=EURO, scheme=EULER)

SEED_PLAIN = 20250211
SEED_NESTED = 20250212


def params(**over):
    p = dict(GBM)
    p.update(over)
    return p


def _bitlen(x: float, f: int) -> int:
    """Integer bits e such that |x| < 2^e (at least 1 - f so that e + f >= 1)."""
    if x <= 0.0:
        return 1 - f
    return max(int(math.floor(math.log2(x))) + 1, 1 - f)


def _bitlen_rounded(x: float, f: int) -> int:
    """Integer bits e such that x rounded to f fractional bits stays below 2^e:
    x + 2^-(f+1) < 2^e."""
    return _bitlen(x + math.ldexp(1.0, -(f + 1)), f)


def default_format(p: dict, level: int) -> dict:
    """Per-level fixed-point formats (e_i, f_i) for the Algorithm-1 variables.

    The paper's optimised bit widths survive only as a lost figure (Fig. 4), so
    this is a stated schedule: fractional bits grow by one per level (the
    d_S,l+1 = d_S,l + 1 trend of Sec. 6.3) and follow the size ordering of
    Sec. 6.3 (con1 ~ h, con2/mul1/sum1/mul2 ~ sqrt(h), S ~ 1), clamped to
    [10, 24], with S (and mul2) capped at 21 fractional bits, and at 30 - e_S
    (not below 10) where S's integer bits would make it wider than 30 bits.  Integer bits bound each variable's magnitude (for the rounded
    constants con1, con2, S0 and K: their values rounded to f bits):
      Z     : |Z~| < 8 for every table size d <= 16 (coarse sums are exact),
      con1  : max(|r| 2h, sigma^2 h / 2) (the Milstein constant shares it),
      con2  : sigma sqrt(h),
      mul1  : max(16 sigma sqrt(h), 128 sigma^2 h)   (|coarse Z~| < 16),
      sum1  : |r| 2h + mul1 bound,
      S     : max(S0 exp(|r| T + 6 sigma sqrt(T)), K),
      mul2  : e_S + e_sum1.
    """
    r, sig, T, S0, K = p["r"], p["sigma"], p["T"], p["S0"], p["K"]
    h = T / float(1 << level)
    f = {
        "Z": 12,
        "con1": 16 + level,
        "con2": 14 + level,
        "mul1": 12 + level,
        "sum1": 12 + level,
        "mul2": 12 + level,
        "S": 14 + level,
    }
    f = {k: min(24, max(10, v)) for k, v in f.items()}
    # S keeps at most 21 fractional bits (the 32-bit fixed-point datapath holds
    # e_S + f_S <= 30 for the test case's e_S = 9), mul2 no more than S
    f["S"] = min(f["S"], 21)
    f["mul2"] = min(f["mul2"], f["S"])
    mul1_bound = max(16.0 * sig * math.sqrt(h), 128.0 * sig * sig * h)
    e = {
        "Z": 3,
        "con1": _bitlen_rounded(max(abs(r) * 2.0 * h, 0.5 * sig * sig * h), f["con1"]),
        "con2": _bitlen_rounded(sig * math.sqrt(h), f["con2"]),
        "mul1": _bitlen(mul1_bound, f["mul1"]),
        "sum1": _bitlen(abs(r) * 2.0 * h + mul1_bound, f["sum1"]),
        "S": _bitlen_rounded(max(S0 * math.exp(abs(r) * T + 6.0 * sig * math.sqrt(T)), K), f["S"]),
    }
    if e["S"] + f["S"] > 30:
        # a wide S (high volatility, long maturity) gives up fractional bits down
        # to 10 so that S keeps to 30 bits
        f["S"] = max(10, 30 - e["S"])
        f["mul2"] = min(f["mul2"], f["S"])
        e["S"] = _bitlen_rounded(max(S0 * math.exp(abs(r) * T + 6.0 * sig * math.sqrt(T)), K), f["S"])
    e["mul2"] = e["S"] + e["sum1"]
    return {"e": [e[v] for v in FORMAT_VARS], "f": [f[v] for v in FORMAT_VARS]}


def uniform_format(p: dict, level: int, frac_bits: int) -> dict:
    """Same integer bits as default_format, one fractional width for every variable."""
    fm = default_format(p, level)
    return {"e": list(fm["e"]), "f": [frac_bits] * 7}


# --------------------------------------------------------------------------
# Workload configurations
# --------------------------------------------------------------------------
def plain_fp64_config():
    """Plain MLMC, FP64, exact Normals: EM European call, levels 0..5, 10^4 samples per level."""
    return dict(name="plain-fp64-em-euro-l0-5-n1e4", params=params(), levels=list(range(6)),
                N=[10_000] * 6, variant=FP64_EXACT, seed=SEED_PLAIN)


def nested_counts(level: int) -> tuple:
    """(N~_l, N^Delta_l) of the nested workload: N~ from 10^7 at l = 0 falling by 2^-1.5
    per level with a floor of 10^4; N^Delta = 10^4 on every level."""
    n_approx = max(10_000, int(round(1e7 * 2.0 ** (-1.5 * level))))
    return n_approx, 10_000


def nested_config():
    """Nested MLMC: European and digital call, EM, levels 0..8, Method-1 table with d = 10,
    approximate paths in fixed point (default_format) with packed draws (three table
    indices per 32-bit word), correction = FP32 exact - fixed (one word per step)."""
    items = []
    for payoff in (EURO, DIGITAL):
        p = params(payoff=payoff)
        for lev in range(9):
            n_a, n_c = nested_counts(lev)
            items.append(dict(params=p, level=lev, N=n_a, variant=FIXED_APPROX, request=payoff))
            items.append(dict(params=p, level=lev, N=n_c, variant=CORR_FIXED, request=payoff))
    return dict(name="nested-fixed-em-euro+digital-l0-8", items=items, d=10, method=1,
                seed=SEED_NESTED, rng_pack=1)


def sweep_points():
    """Level-kernel sweep (Milstein; European, Asian, lookback; three volatilities)."""
    pts = []
    for payoff in (EURO, ASIAN, LOOKBACK):
        for sig in (0.1, 0.2, 0.4):
            pts.append(params(payoff=payoff, sigma=sig, scheme=MILSTEIN))
    return pts


def batched_options(n=256, seed=7, eps_range=(1e-4, 1e-2)):
    """Batched workload: n independent options; payoff mix European / digital / Asian;
    accuracies log-uniform in eps_range."""
    rng = np.random.default_rng(seed)
    S0 = rng.uniform(80, 120, n)
    K = rng.uniform(80, 120, n)
    sig = rng.uniform(0.1, 0.5, n)
    T = rng.uniform(0.25, 2.0, n)
    pay = rng.integers(0, 3, n)
    eps = np.exp(rng.uniform(math.log(eps_range[0]), math.log(eps_range[1]), n))
    return [dict(S0=float(S0[i]), K=float(K[i]), r=0.05, sigma=float(sig[i]), T=float(T[i]),
                 payoff=int(pay[i]), scheme=EULER, eps=float(eps[i])) for i in range(n)]


def poisson_arrivals(rate, n=10_000, seed=11):
    """Arrival times (seconds) of a Poisson stream of n requests."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))
