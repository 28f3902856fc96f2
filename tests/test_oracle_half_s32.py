"""Pins of the oracle's half-precision variants with S in FP32 (the approximate
path's increments in binary16 / bfloat16, one IEEE rounding per operation, and
S, its running average and minimum in FP32).

* Replay: the increments rounded by the oracle's half rounding (itself pinned
  against numpy float16 and torch bfloat16 conversions) and S updated with
  numpy float32 arithmetic (IEEE single, one rounding per operation) give the
  oracle's terminal values and integer payoffs bit for bit.
* The FP32 S path tracks the exact path far more closely than the all-half
  path, and its correction has the smaller variance.
* eq. chap:nested_exp with the new variants: E[dP~] + E[dP - dP~] = E[dP]."""
import math

import numpy as np
import pytest

from oracle import core, tables
from paper_2502_07123_gb300 import workloads as W


def _replay(p, lev, s, variant, seed, d=10):
    """Terminal values and FP32 payoffs (units 2^-24) of sample s by the rules above."""
    rnd = core.round_fp16 if core.approx_rep(variant) == "fp16" else core.round_bf16
    r1 = lambda x: float(rnd(np.array([x]))[0])
    n = 1 << lev
    h = p["T"] / n
    c1, c1c = r1(p["r"] * h), r1(p["r"] * 2 * h)
    c2, c3 = r1(p["sigma"] * math.sqrt(h)), r1(0.5 * p["sigma"] ** 2 * h)
    tab = tables.table(d, 1, core.approx_rep(variant))
    J = core.draws(seed, 0, lev, core.default_stream(variant), np.full(n, s, dtype=np.uint64), np.arange(n))
    f32 = np.float32
    mil = p["scheme"] == W.MILSTEIN

    def inc(z, c, m):
        sum1 = r1(c + r1(c2 * z))
        if mil:
            sum1 = r1(sum1 + r1(c3 * r1(r1(z * z) - m)))
        return f32(sum1)

    S = Sc = f32(p["S0"])
    accf, accc = [], []
    zprev = 0.0
    for i in range(n):
        j = int(J[i]) >> (32 - d)
        z = float(tab[j]) if j < (1 << (d - 1)) else -float(tab[(1 << d) - 1 - j])
        S = f32(S + f32(S * inc(z, c1, 1.0)))
        accf.append(S)
        if lev > 0 and i & 1:
            Sc = f32(Sc + f32(Sc * inc(r1(zprev + z), c1c, 2.0)))
            accc.append(Sc)
        zprev = z
    K = f32(p["K"])

    def pay(path, s0):
        x = path[-1]
        if p["payoff"] == W.EURO:
            P = max(f32(x - K), f32(0))
        elif p["payoff"] == W.DIGITAL:
            P = f32(1) if x > K else f32(0)
        elif p["payoff"] == W.ASIAN:
            acc = f32(0.5) * f32(s0)
            for v in path[:-1]:
                acc = f32(acc + v)
            tot = f32(acc + f32(f32(0.5) * x))
            P = max(f32(f32(tot * f32(1.0 / len(path))) - K), f32(0))
        else:
            P = f32(x - min([f32(s0)] + path))
        return int(np.rint(float(f32(P * f32(16777216.0)))))
    qf = pay(accf, p["S0"])
    qc = pay(accc, p["S0"]) if lev > 0 else 0
    return float(S), (float(Sc) if lev > 0 else 0.0), qf, qc


@pytest.mark.parametrize("variant", [core.FP16S_APPROX, core.BF16S_APPROX])
@pytest.mark.parametrize("scheme", [W.EULER, W.MILSTEIN])
@pytest.mark.parametrize("payoff", [W.EURO, W.DIGITAL, W.ASIAN, W.LOOKBACK])
@pytest.mark.parametrize("lev", [0, 1, 3])
def test_fp32_s_path_replay(variant, scheme, payoff, lev):
    p = W.params(scheme=scheme, payoff=payoff, sigma=0.3)
    seed, first, N = 11 + lev, 5, 24
    _, dump = core.level(p, lev, first, N, variant, seed, dump=True)
    for t in range(N):
        af, ac, qf, qc = _replay(p, lev, first + t, variant, seed)
        assert dump["af"][t] == af and dump["ac"][t] == ac, (t, dump["af"][t], af)
        assert dump["qf"][t] == qf and dump["qc"][t] == qc, (t, dump["qf"][t], qf, dump["qc"][t], qc)


@pytest.mark.parametrize("half,s32,near_fixed,factor", [(core.FP16_APPROX, core.FP16S_APPROX, 1.3, 1.8),
                                                        (core.BF16_APPROX, core.BF16S_APPROX, 3.0, 4.0)])
def test_fp32_s_tracks_the_exact_path(half, s32, near_fixed, factor):
    """With S in FP32 the approximate path's distance from the exact path is set
    by the table and the increments' precision (binary16: as the fixed-point
    path's, within 30%; bfloat16's 8-bit significand: within 3x), no longer by
    the rounding of S, which the all-half paths pay for."""
    p = W.params()
    lev, N = 5, 4000
    _, ex = core.level(p, lev, 0, N, core.FP64_EXACT, 8, stream=0, dump=True)
    _, a = core.level(p, lev, 0, N, half, 8, stream=0, dump=True)
    _, b = core.level(p, lev, 0, N, s32, 8, stream=0, dump=True)
    _, f = core.level(p, lev, 0, N, core.FIXED_APPROX, 8, stream=0, dump=True, fmt=W.default_format(p, lev))
    err = lambda d: np.median(np.abs(d["af"] - ex["sf"]) / ex["sf"])
    assert err(b) < near_fixed * err(f), (err(b), err(f))
    assert err(a) > factor * err(b), (err(a), err(b))


@pytest.mark.parametrize("approx,corr,half_corr", [(core.FP16S_APPROX, core.CORR_FP16S, core.CORR_FP16),
                                                   (core.BF16S_APPROX, core.CORR_BF16S, core.CORR_BF16)])
def test_nested_expectation_with_fp32_s(approx, corr, half_corr):
    p = W.params()
    lev, N = 3, 40_000
    sa, _ = core.level(p, lev, 0, N, approx, 31)
    sc, _ = core.level(p, lev, 0, N, corr, 31)
    se_, _ = core.level(p, lev, 0, N, core.FP64_EXACT, 32)
    sh, _ = core.level(p, lev, 0, N, half_corr, 31)
    ma, mc, me = sa["sum"] / N, sc["sum"] / N, se_["sum"] / N
    va, vc, ve = (x["sum2"] / N - m * m for x, m in ((sa, ma), (sc, mc), (se_, me)))
    assert abs(ma + mc - me) < 4 * math.sqrt((va + vc + ve) / N)
    vh = sh["sum2"] / N - (sh["sum"] / N) ** 2
    assert vc < 0.5 * vh     # the FP32 S correction varies less than the all-half one
