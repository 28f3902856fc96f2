"""Pins of the oracle's Method 2 (Sec. 3.2): the iteration counts and MSE
relations the paper prints, least-squares optimality at the converged
permutation, antisymmetry, the MSE decomposition against Monte Carlo with
the coupled uniform, and the coupling of the exact path in the level
estimator."""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import ndtri

from oracle import core, tables as T
from paper_2502_07123_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_claims.json")))


def _band(key, x):
    lo, hi = GOLD[key]["band"]
    assert lo <= x <= hi, (key, x)


def test_paper_iteration_counts_and_mse_relations():
    r10, r12 = T.m2_optimise(10), T.m2_optimise(12)
    _band("m2_iterations_d10", r10["iterations"])
    _band("m2_iterations_d12", r12["iterations"])
    for d in (8, 10, 12):
        r = T.m2_optimise(d)
        assert r["mse"] < 0.9 * r["mse0"]                       # the optimisation helps
        _band("m2_vs_m1_dminus1", r["mse"] / float(T.moments_m1(d - 1)[1]))
        _band("m2_vs_m1_same_d", r["mse"] / float(T.moments_m1(d)[1]))
    # MSE divided by about 2 per bit (4 per field-bit pair)
    ratio = T.m2_optimise(8)["mse"] / T.m2_optimise(10)["mse"]
    assert 3.0 <= ratio <= 5.5


@pytest.mark.parametrize("d", [4, 6, 10])
def test_least_squares_optimal_at_fixed_point(d):
    r = T.m2_optimise(d)
    A = T.m2_design(d, 2)
    t = T.m1_full(d)[r["pi"]]
    resid = t - A @ r["x"]
    assert np.abs(A.T @ resid).max() < 1e-10 * (1 << d)
    assert sorted(r["pi"].tolist()) == list(range(1 << d))
    np.testing.assert_array_equal(T.m2_rank(r["values"]), r["pi"])
    v = r["values"]
    np.testing.assert_array_equal(v[::-1], -v)                  # Z~_{2^d-1-j} = -Z~_j
    np.testing.assert_allclose(v, A @ r["x"], rtol=0, atol=1e-13)


def test_n_fields_general():
    """n = 3, 4, 6 fields: the iteration stops (converged or back in an earlier
    permutation), beats its start, and returns the ranking of its own values;
    the sums are A x, antisymmetric, and identical for indices whose fields are
    the same values in another order."""
    for d, n in ((9, 3), (12, 3), (8, 4), (12, 4), (12, 6)):
        r = T.m2_optimise(d, n)
        assert r["iterations"] < 1000
        assert r["mse"] < r["mse0"]
        v = r["values"]
        np.testing.assert_array_equal(T.m2_rank(v), r["pi"])
        assert sorted(r["pi"].tolist()) == list(range(1 << d))
        np.testing.assert_allclose(v, T.m2_design(d, n) @ r["x"], rtol=0, atol=1e-13)
        np.testing.assert_array_equal(v[::-1], -v)
        b = d // n
        j = np.arange(1 << d)
        fields = [(j >> (b * (n - 1 - i))) & ((1 << b) - 1) for i in range(n)]
        rolled = sum(fields[(i + 1) % n] << (b * (n - 1 - i)) for i in range(n))
        np.testing.assert_array_equal(v[rolled], v)


def test_two_field_sums_are_the_plain_sum():
    """For n = 2 the ordered net-count sum is x_a +- x_b as written."""
    d = 10
    r = T.m2_optimise(d)
    x, b = r["x"], d // 2
    for jj in range(0, 1 << d, 37):
        f1, f2 = jj >> b, jj & ((1 << b) - 1)
        a = x[f1] if f1 < (1 << (b - 1)) else -x[(1 << b) - 1 - f1]
        c = x[f2] if f2 < (1 << (b - 1)) else -x[(1 << b) - 1 - f2]
        assert r["values"][jj] == a + c


def test_mse_against_monte_carlo_with_coupled_uniform():
    d = 8
    r = T.m2_optimise(d)
    rng = np.random.default_rng(3)
    J = rng.integers(0, 2 ** 32, 2_000_000, dtype=np.uint64)
    j = J >> (32 - d)
    Jp = (r["pi"][j].astype(np.uint64) << np.uint64(32 - d)) | (J & np.uint64((1 << (32 - d)) - 1))
    U = (Jp.astype(np.float64) + 0.5) * 2.0 ** -32
    err = ndtri(U) - r["values"][j]
    mc = float(np.mean(err * err))
    se = float(np.std(err * err)) / math.sqrt(len(err))
    assert abs(mc - r["mse"]) < 5 * se
    # the coupled uniform is uniform: every interval is hit as often as before
    counts = np.bincount((Jp >> np.uint64(32 - d)).astype(np.int64), minlength=1 << d)
    ref = np.bincount(j.astype(np.int64), minlength=1 << d)
    np.testing.assert_array_equal(np.sort(counts), np.sort(ref))


def test_representation_tables():
    d, fZ = 10, 12
    r = T.m2_optimise(d)
    fixed = T.m2_table(d, "fixed", fZ)
    xq = [T.round_fixed(v, fZ) for v in r["x"]]
    for jj in (0, 5, 77, 511, 512, 1000):
        f1, f2 = jj >> 5, jj & 31
        a = xq[f1] if f1 < 16 else -xq[31 - f1]
        b = xq[f2] if f2 < 16 else -xq[31 - f2]
        assert fixed[jj] == math.ldexp(a + b, -fZ)
    np.testing.assert_array_equal(fixed[::-1], -fixed)
    h = T.m2_table(d, "fp16")
    assert np.all(h.astype(np.float16).astype(np.float64) == h)
    np.testing.assert_array_equal(T.table(d, 2, "fixed", fZ), fixed[:512])


def test_coupling_in_the_level_estimator():
    """With Method 2 the correction's exact path reads J' (interval pi(j)); the
    coupled corrections have a small variance (about the Method-1 one at d - 1),
    while the identity E[Y~] + E[Y^Delta] = E[Y] holds."""
    p = W.params()
    lev, N = 3, 20000
    fm = W.default_format(p, lev)
    c2, _ = core.level(p, lev, 0, N, core.CORR_FIXED, 4, d=10, method=2, fmt=fm)
    c1, _ = core.level(p, lev, 0, N, core.CORR_FIXED, 4, d=9, method=1, fmt=fm)
    v2 = c2["sum2"] / N - (c2["sum"] / N) ** 2
    v1 = c1["sum2"] / N - (c1["sum"] / N) ** 2
    assert 0.5 * v1 < v2 < 1.5 * v1
    # exact part of one correction sample against the FP64 path on the moved uniforms
    _, dump = core.level(p, lev, 7, 1, core.CORR_FIXED, 4, d=10, method=2, fmt=fm, dump=True)
    pi = T.m2_optimise(10)["pi"]
    S = p["S0"]
    h = p["T"] / 8
    for i in range(8):
        J = int(core.draws(4, 0, lev, 0, np.array([7], np.uint64), np.array([i], np.uint32))[0])
        Jp = (int(pi[J >> 22]) << 22) | (J & ((1 << 22) - 1))
        z = float(core.exact_normal(np.array([Jp], np.uint32))[0])
        S = S + p["r"] * S * h + p["sigma"] * S * math.sqrt(h) * z
    assert dump[0]["sf"] == pytest.approx(S, rel=1e-14)
