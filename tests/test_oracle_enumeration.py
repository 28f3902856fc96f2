"""Exact expectation of the approximate level difference on levels 0 and 1:
the approximate Normal takes 2^d values, so E[dP~_l] is the mean over the
2^(d 2^l) combinations of table cells.  Pinned by brute force over the cells
(Python loop on a tiny table) and against the Monte Carlo estimate."""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import core
from paper_2502_07123_gb300 import workloads as W


def test_enumeration_draws_cover_every_cell_once():
    p = W.params()
    d = 6
    _, dump = core.level(p, 1, 0, 1 << (2 * d), core.FIXED_APPROX, 1, d=d, fmt=W.default_format(p, 1),
                         dump=True, enumerate=1)
    pairs = set()
    for s in range(1 << (2 * d)):
        pairs.add((s & 63, s >> 6))
    assert len(pairs) == 1 << (2 * d)


@pytest.mark.parametrize("payoff", [W.EURO, W.DIGITAL])
def test_level0_expectation_by_brute_force(payoff):
    """Level 0: E[P~] = 2^-d sum over j of payoff(S0 + rd(S0 rd(con1 + rd(con2 z_j)))),
    written out with rationals from the Algorithm-1 definition."""
    p = W.params(payoff=payoff)
    d = 8
    fmt = W.default_format(p, 0)
    s, _ = core.level(p, 0, 0, 1 << d, core.FIXED_APPROX, 1, d=d, fmt=fmt, enumerate=1)
    from oracle import tables
    from tests.test_oracle_fixed import brute_sample
    zt = tables.table(d, 1, "fixed", fmt["f"][0])
    tot = Fr(0)
    for j in range(1 << d):
        J = j << (32 - d)
        _, _, pf, pc, _ = brute_sample(p, 0, fmt, zt, [J], d)
        tot += pf - pc
    assert Fr(s["isum"], 2 ** s["unit"]) == tot


def test_exact_level_matches_monte_carlo():
    p = W.params()
    for lev in (0, 1):
        fmt = W.default_format(p, lev)
        d = 10 if lev == 0 else 8
        ex, _ = core.level(p, lev, 0, 1 << (d << lev), core.FIXED_APPROX, 1, d=d, fmt=fmt, enumerate=1)
        N = 200_000
        mc, _ = core.level(p, lev, 0, N, core.FIXED_APPROX, 5, d=d, fmt=fmt)
        n_ex = 1 << (d << lev)
        m_ex = ex["sum"] / n_ex
        m = mc["sum"] / N
        v = mc["sum2"] / N - m * m
        assert abs(m - m_ex) < 4 * math.sqrt(v / N)


def test_enumeration_rejected_where_undefined():
    p = W.params()
    with pytest.raises(core.OracleError):
        core.level(p, 2, 0, 10, core.FIXED_APPROX, 1, fmt=W.default_format(p, 2), enumerate=1)
    with pytest.raises(core.OracleError):
        core.level(p, 0, 0, 10, core.CORR_FIXED, 1, fmt=W.default_format(p, 0), enumerate=1)
