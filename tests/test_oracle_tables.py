"""Pins of the oracle's approximate inverse-CDF tables (Sec. 3.1 Method 1, Sec. 3.3 Method 3)."""
import json
import math
import os

import mpmath as mp
import numpy as np
import pytest
from scipy import integrate
from scipy.special import ndtri

from oracle import core, tables

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_claims.json")))


def test_m1_table_size_d10():
    assert len(tables.m1_exact(10)) == GOLD["m1_table_entries_d10"]["value"]


@pytest.mark.parametrize("d,ks", [(6, range(32)), (10, [0, 1, 2, 17, 100, 300, 510, 511])])
def test_m1_matches_quadrature(d, ks):
    """Z_k = 2^d * integral of Phi^{-1} over [k 2^-d, (k+1) 2^-d] (Sec. 3.1), by adaptive quadrature."""
    z = tables.m1_fp64(d)
    for k in ks:
        a, b = k * 2.0**-d, (k + 1) * 2.0**-d
        val, err = integrate.quad(ndtri, a, b, epsabs=1e-15, epsrel=1e-13, limit=400)
        ref = val * 2.0**d
        tol = 1e-8 if k == 0 else 1e-11
        assert abs(z[k] - ref) <= tol * abs(ref), (k, z[k], ref)


@pytest.mark.parametrize("d", [4, 8, 10, 12])
def test_m1_total_integral(d):
    """sum_k 2^-d Z_k = integral_0^{1/2} Phi^{-1} = -phi(0) = -1/sqrt(2 pi)."""
    with mp.workdps(40):
        s = mp.fsum(tables.m1_exact(d)) / mp.mpf(2) ** d
        assert abs(s + 1 / mp.sqrt(2 * mp.pi)) < mp.mpf(10) ** -30


def test_m1_mse_monte_carlo_and_conditional_mean():
    """MSE = 1 - E[Z~^2] (Z~ is the conditional mean of Z given j), checked against a Monte
    Carlo estimate that uses the oracle's own index/sign rule and exact inverse CDF."""
    d = 10
    rng = np.random.default_rng(99)
    J = rng.integers(0, 2**32, 1 << 21, dtype=np.uint64).astype(np.uint32)
    Z = core.exact_normal(J)
    Zt = core.approx_normal(J, d, tables.m1_fp64(d))
    diff = Z - Zt
    ez2, mse = tables.moments_m1(d)
    se = np.std(diff**2) / math.sqrt(diff.size)
    assert abs(np.mean(diff**2) - float(mse)) < 5 * se
    # conditional-mean property: the error is orthogonal to Z~ and has zero mean
    se2 = np.std(diff * Zt) / math.sqrt(diff.size)
    assert abs(np.mean(diff * Zt)) < 5 * se2
    assert abs(np.mean(diff)) < 5 * np.std(diff) / math.sqrt(diff.size)
    # a wrong sign or mirrored index would give an MSE of order 1
    assert np.mean(diff**2) < 2e-4


def test_m1_mse_halves_per_bit():
    lo, hi = GOLD["m1_mse_ratio_per_bit"]["band"]
    d0, d1 = GOLD["m1_mse_ratio_per_bit"]["d_range"]
    prev = None
    for d in range(d0, d1 + 1):
        _, mse = tables.moments_m1(d)
        if prev is not None:
            assert lo <= float(prev / mse) <= hi, d
        prev = mse


def test_m3_two_point_classes_exact_and_size():
    for d in (6, 10, 12):
        coef = tables.m3_exact(d)
        assert len(coef) == d - 1
        Z = tables.m1_exact(d)
        with mp.workdps(40):
            for k in range(4):
                a, b = coef[tables.m3_class_of(k)]
                assert abs(a + b * k - Z[k]) < mp.mpf(10) ** -30


def test_m3_least_squares_normal_equations():
    d = 10
    Z = tables.m1_exact(d)
    with mp.workdps(40):
        for c, (a, b) in enumerate(tables.m3_exact(d)):
            ks = [k for k in range(len(Z)) if tables.m3_class_of(k) == c]
            res = [a + b * k - Z[k] for k in ks]
            assert abs(mp.fsum(res)) < mp.mpf(10) ** -28
            assert abs(mp.fsum(r * k for r, k in zip(res, ks))) < mp.mpf(10) ** -25


def test_mse_dyadic_identity_by_quadrature():
    """eq. mse_dyadic: integral (Zbar_j - Phi^{-1})^2 = 2^-d (Zbar_j - Z_j)^2 + integral (Z_j - Phi^{-1})^2."""
    d = 8
    z1 = tables.m1_fp64(d)
    coef = tables.m3_coefficients_fp64(d)
    for k in (1, 5, 40, 127):
        a, b = coef[tables.m3_class_of(k)]
        zbar = a + b * k
        u0, u1 = k * 2.0**-d, (k + 1) * 2.0**-d
        lhs = integrate.quad(lambda u: (zbar - ndtri(u)) ** 2, u0, u1, epsabs=1e-16, epsrel=1e-12)[0]
        rhs = 2.0**-d * (zbar - z1[k]) ** 2 + \
            integrate.quad(lambda u: (z1[k] - ndtri(u)) ** 2, u0, u1, epsabs=1e-16, epsrel=1e-12)[0]
        assert abs(lhs - rhs) <= 1e-9 * rhs


def test_m3_against_m1_claims():
    r10 = float(tables.mse_m3(10) / tables.moments_m1(10)[1])
    r12 = float(tables.mse_m3(12) / tables.moments_m1(12)[1])
    assert GOLD["m3_over_m1_mse_d10"]["band"][0] < r10 < GOLD["m3_over_m1_mse_d10"]["band"][1]
    assert GOLD["m3_over_m1_mse_d12"]["band"][0] < r12 < GOLD["m3_over_m1_mse_d12"]["band"][1]
    for d in (4, 8, 12):
        assert tables.mse_m3(d) >= tables.moments_m1(d)[1]


def test_m3_mse_plateaus():
    """The dyadic MSE stops falling (Sec. 3.4): its decrements shrink geometrically while the
    Method-1 MSE keeps halving, and the limit stays a sizeable fraction of the d = 12 value."""
    m = [float(tables.mse_m3(d)) for d in range(9, 14)]
    dec = [m[i] - m[i + 1] for i in range(len(m) - 1)]
    ratios = [dec[i + 1] / dec[i] for i in range(len(dec) - 1)]
    assert all(0.3 < q < 0.6 for q in ratios)
    limit = m[-1] - dec[-1] * ratios[-1] / (1 - ratios[-1])
    assert limit > 0.5 * m[-2] * 0.5 and limit > 0.0


def test_table_representations():
    d = 10
    z64 = tables.m1_fp64(d)
    fx = tables.table(d, 1, "fixed", 12)
    assert np.all(np.ldexp(fx, 12) == np.round(np.ldexp(fx, 12)))
    assert np.max(np.abs(fx - z64)) <= 2.0**-13
    f16 = tables.table(d, 1, "fp16")
    assert np.array_equal(f16, z64.astype(np.float16).astype(np.float64))
    for method in (1, 3):
        for rep in ("fp32", "fp16", "bf16", "fixed"):
            t = tables.table(d, method, rep, 12)
            assert t.shape == (512,)
            # Method 1 values are interval means of Phi^{-1} on [0, 1/2]: negative and increasing;
            # the Method-3 line of the widest class may cross zero near u = 1/2
            if method == 1:
                assert np.all(t < 0) and np.all(np.diff(t) >= 0)
            assert np.max(np.abs(t - z64)) < 0.05
