"""Pin of the oracle's fixed-point emulation against exact rational arithmetic.

Algorithm 1 (Sec. 4.1) is replayed on tiny inputs with fractions.Fraction, using
the definition of the number format (x~ = n 2^-f, |n| <= 2^(e+f) - 1) and of
round-to-nearest (ties toward +infinity, the stated reading): every
intermediate is rounded once from its exact rational value.  The oracle, which
works with shifted 128-bit integers, must agree bit for bit, and every rounding
error must respect eq. bound_rounding_error, |delta x| <= 2^(-f-1).
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import core, tables
from paper_2502_07123_gb300 import workloads as W

V_Z, V_CON1, V_CON2, V_MUL1, V_SUM1, V_MUL2, V_S = range(7)


class Fx:
    def __init__(self, fmt):
        self.e, self.f = fmt["e"], fmt["f"]
        self.sat = False

    def rd(self, x, v):
        f = self.f[v]
        n = math.floor(x * 2**f + Fr(1, 2))
        q = Fr(n, 2**f)
        assert abs(q - x) <= Fr(1, 2 ** (f + 1))          # eq. bound_rounding_error
        lim = 2 ** (self.e[v] + f) - 1
        if abs(n) > lim:
            self.sat = True
            q = Fr(lim if n > 0 else -lim, 2**f)
        return q


def const(x, f):
    return Fr(math.floor(math.ldexp(x, f) + 0.5), 2**f)


def brute_sample(p, lev, fmt, ztab, J_row, d):
    fx = Fx(fmt)
    h = math.ldexp(p["T"], -lev)
    f = fmt["f"]
    con1 = const(p["r"] * h, f[V_CON1])
    con1c = const(p["r"] * (2.0 * h), f[V_CON1])
    con2 = const(p["sigma"] * math.sqrt(h), f[V_CON2])
    con3 = const(0.5 * p["sigma"] * p["sigma"] * h, f[V_CON1])
    S0 = const(p["S0"], f[V_S])
    K = const(p["K"], f[V_S])
    mil = p["scheme"] == W.MILSTEIN

    def step(S, z, c1, m):
        mul1 = fx.rd(con2 * z, V_MUL1)
        acc = c1 + mul1
        if mil:
            acc += fx.rd(con3 * (z * z - m), V_MUL1)
        sum1 = fx.rd(acc, V_SUM1)
        mul2 = fx.rd(S * sum1, V_MUL2)
        return fx.rd(S + mul2, V_S)

    def zt(J):
        j = J >> (32 - d)
        half = 1 << (d - 1)
        idx, neg = (j, False) if j < half else ((1 << d) - 1 - j, True)
        v = Fr(float(ztab[idx]))
        return -v if neg else v

    S, Sc = S0, S0
    fine, coarse = [S0], [S0]
    zprev = None
    for i, J in enumerate(J_row):
        z = zt(int(J))
        S = step(S, z, con1, 1)
        fine.append(S)
        if lev > 0 and i % 2 == 1:
            Sc = step(Sc, zprev + z, con1c, 2)
            coarse.append(Sc)
        zprev = z

    def payoff(path, unit_steps):
        x = path[-1]
        if p["payoff"] == W.EURO:
            return max(x - K, 0)
        if p["payoff"] == W.DIGITAL:
            return Fr(1) if x > K else Fr(0)
        if p["payoff"] == W.ASIAN:
            n = len(path) - 1
            avg = (path[0] / 2 + sum(path[1:-1]) + path[-1] / 2) / n
            return max(avg - K, 0)
        return x - min(path)

    pf = payoff(fine, None)
    pc = payoff(coarse, None) if lev > 0 else Fr(0)
    return S, (Sc if lev > 0 else Fr(0)), pf, pc, fx.sat


CASES = []
rng = np.random.default_rng(12)
for lev in (0, 1, 2):
    for payoff in (W.EURO, W.DIGITAL, W.ASIAN, W.LOOKBACK):
        for scheme in (W.EULER, W.MILSTEIN):
            CASES.append((lev, payoff, scheme, int(rng.integers(6, 21)), int(rng.integers(0, 1000))))


@pytest.mark.parametrize("pack", [0, 1])
@pytest.mark.parametrize("lev,payoff,scheme,fbits,seed", CASES)
def test_fixed_point_matches_rationals(lev, payoff, scheme, fbits, seed, pack):
    p = W.params(payoff=payoff, scheme=scheme, sigma=0.3)
    fmt = W.default_format(p, lev)
    r = np.random.default_rng(seed)
    fmt["f"] = [int(x) for x in r.integers(max(4, fbits - 4), fbits + 5, 7)]
    d = 8
    N = 64
    sums, dump = core.level(p, lev, 1000, N, core.FIXED_APPROX, seed, d=d, fmt=fmt, dump=True, pack=pack)
    ztab = tables.table(d, 1, "fixed", fmt["f"][V_Z])
    n = 1 << lev
    s_idx = np.repeat(np.arange(1000, 1000 + N, dtype=np.uint64), n)
    steps = np.tile(np.arange(n, dtype=np.uint32), N)
    if pack:
        J = core.draws_packed(seed, 0, lev, 1, s_idx, steps, d).reshape(N, n)
    else:
        J = core.draws(seed, 0, lev, 1, s_idx, steps).reshape(N, n)
    unit = sums["unit"]
    tot = 0
    for t in range(N):
        S, Sc, pf, pc, sat = brute_sample(p, lev, fmt, ztab, J[t], d)
        assert Fr(float(dump["af"][t])) == S
        if lev > 0:
            assert Fr(float(dump["ac"][t])) == Sc
        assert Fr(int(dump["qf"][t]), 2**unit) == pf
        assert Fr(int(dump["qc"][t]), 2**unit) == pc
        assert bool(dump["sat"][t]) == sat
        tot += int(dump["qf"][t]) - int(dump["qc"][t])
    assert sums["isum"] == tot


def test_saturation_is_counted():
    p = W.params()
    fmt = W.default_format(p, 2)
    fmt["e"][V_S] = 7          # |S| < 128: GBM paths from 100 leave this range often
    fmt["e"][V_MUL2] = 7 + fmt["e"][V_SUM1]
    sums, dump = core.level(p, 2, 0, 2000, core.FIXED_APPROX, 3, d=10, fmt=fmt, dump=True)
    assert 0 < sums["saturations"] == int(dump["sat"].sum()) < 2000
    assert np.all(dump["af"] <= 128.0)
