"""Pins of the oracle's error-model statistics and bit-width optimiser
(Sec. 4.2-4.3 and 6): adjoint sensitivities against finite differences,
closed forms on level 0, the forward pass against the plain FP64 level
estimator, the Lagrange / golden-section / greedy-rounding steps against
their defining conditions and brute force, the model bound against the
oracle's own fixed-point corrections, and the level-cost savings the paper
prints."""
import json
import math
import os

import numpy as np
import pytest
from scipy.stats import norm

from oracle import core, optimiser as O, tables
from paper_2502_07123_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_claims.json")))
P = W.params()


def _in_the_money_samples(lev, k=3, seed=5):
    out = []
    s = 0
    while len(out) < k:
        dp, xb = core.sens_probe(P, lev, seed, 0, s, -1, -1, 0.0, True)
        if abs(xb[6, :]).max() > 0:        # the fine or the coarse path ends in the money
            out.append(s)
        s += 1
    return out


@pytest.mark.parametrize("lev", [0, 1, 2, 4])
def test_adjoint_matches_finite_differences(lev):
    """Every instance's sensitivity equals the central difference of DeltaP."""
    ni = core.sens_instances(lev)
    for s in _in_the_money_samples(lev, 2):
        _, xb = core.sens_probe(P, lev, 5, 0, s, -1, -1, 0.0, True)
        scale = abs(xb).max()
        for t in range(7):
            for i in range(ni):
                h = 1e-7
                fd = (core.sens_probe(P, lev, 5, 0, s, t, i, h) - core.sens_probe(P, lev, 5, 0, s, t, i, -h)) / (2 * h)
                assert abs(fd - xb[t, i]) <= 1e-5 * scale, (lev, s, O.VARS[t], i, fd, xb[t, i])


def test_level0_closed_forms():
    """Level 0: DeltaP = e^{-rT} max(S0 (1 + con1 + con2 Z) - K, 0); the second
    moments of the con1, con2 and S0 sensitivities have closed forms."""
    N = 200_000
    r = core.sensitivities(P, 0, 0, N, 11, per_instance=True)
    h = P["T"]
    con1, con2 = P["r"] * h, P["sigma"] * math.sqrt(h)
    disc = math.exp(-P["r"] * P["T"])
    zs = (P["K"] / P["S0"] - 1.0 - con1) / con2
    tail = 1.0 - norm.cdf(zs)
    ez2 = zs * norm.pdf(zs) + tail                      # E[Z^2 1{Z > z*}]
    ez = norm.pdf(zs)                                    # E[Z 1{Z > z*}]
    a = 1.0 + con1
    exact = {
        "con1": disc ** 2 * P["S0"] ** 2 * tail,
        "con2": disc ** 2 * P["S0"] ** 2 * ez2,
        "S0": disc ** 2 * (a * a * tail + 2 * a * con2 * ez + con2 * con2 * ez2),
    }
    got = {"con1": r["inst"][1, 0] / N, "con2": r["inst"][2, 0] / N, "S0": r["inst"][6, -1] / N}
    # Monte Carlo error: the sensitivities are bounded by disc S0 (1 + con1 + 5 con2) and 5 disc S0
    for k in exact:
        bound = 6 * (disc * P["S0"] * 3.0) ** 2 / math.sqrt(N)
        assert abs(got[k] - exact[k]) < bound, (k, got[k], exact[k])
        assert abs(got[k] / exact[k] - 1.0) < 0.02, (k, got[k], exact[k])


def test_forward_pass_matches_fp64_level_estimator():
    """The forward sweep is the FP64 exact level difference on the same uniforms
    (stream 0, as the correction estimator draws them)."""
    for lev in (0, 1, 3):
        N = 3000
        r = core.sensitivities(P, lev, 0, N, 7, per_instance=False)
        s, _ = core.level(P, lev, 0, N, core.FP64_EXACT, 7, stream=0)
        disc = math.exp(-P["r"] * P["T"])
        assert abs(r["sum_dp"] - disc * s["sum"]) <= 1e-11 * (abs(disc * s["sum"]) + N)
        assert abs(r["sum_dp2"] - disc * disc * s["sum2"]) <= 1e-11 * (disc * disc * s["sum2"] + N)


def test_maxima_and_type_sums():
    lev = 3
    r = core.sensitivities(P, lev, 0, 500, 3, per_instance=True)
    h = P["T"] / 8
    assert r["maxabs"][1] == pytest.approx(P["r"] * 2 * h, rel=0, abs=0)
    assert r["maxabs"][2] == pytest.approx(P["sigma"] * math.sqrt(h), rel=1e-15)
    assert r["maxabs"][6] >= P["S0"]
    np.testing.assert_allclose(r["A"], r["inst"].sum(axis=1), rtol=1e-12)
    # sum1 and mul1 errors enter DeltaP identically (sum1 = con1 + mul1)
    np.testing.assert_allclose(r["A"][3], r["A"][4], rtol=1e-14)


def _stats(lev, N, seed=5):
    r = core.sensitivities(P, lev, 0, N, seed, per_instance=True)
    A = list(r["A"] / N)
    B = list(np.sqrt(r["inst"] / N).sum(axis=1))
    V = r["sum_dp2"] / N - (r["sum_dp"] / N) ** 2
    return A, B, list(r["maxabs"]), V


MSE = {d: float(tables.moments_m1(d)[1]) for d in range(2, 17)}


def test_lagrange_solution_is_stationary_and_optimal():
    lev = 2
    A, B, mx, V = _stats(lev, 3000)
    o = O.optimise_level(lev, A, B, mx, V)
    e, d, lam = o["e"], o["d_real"], o["lambda"]
    st = O.steps_of(lev)
    for t in range(7):
        lhs = O.LN4 / 12 * A[t] * 4.0 ** (e[t] - d[t])
        rhs = lam * st * (O.M_MUL[t] * d[t] + O.M_ADD[t])
        assert abs(lhs - rhs) <= 1e-9 * rhs, O.VARS[t]
    # lambda = sqrt(V V_indep / (C C~)) at the optimum (Sec. 6.1)
    C = (1 << lev) * 1e4
    assert lam == pytest.approx(math.sqrt(V * O.v_indep(A, e, d) / (C * O.cost_lp(d, lev))), rel=1e-4)
    # a local minimum of the level cost, and better than every uniform bit-width (Fig. 5)
    F0 = O.level_cost(V, C, A, e, d, lev)
    rng = np.random.default_rng(0)
    for _ in range(200):
        dd = list(np.array(d) + rng.normal(0, 0.3, 7))
        assert O.level_cost(V, C, A, e, dd, lev) >= F0 * (1 - 1e-12)
    for u in range(1, 40):
        assert O.level_cost(V, C, A, e, [float(u)] * 7, lev) > F0


def test_lagrange_against_brute_force_two_variables():
    """Two variables: the golden-section / Lagrange optimum equals a grid search."""
    A = [3.0, 0.0, 0.0, 0.0, 0.0, 0.0, 40.0]
    e = [2, 0, 0, 0, 0, 0, 8]
    mx = [2.0 ** (x - 1) + 1e-9 for x in e]
    lev, V = 1, 2.0
    o = O.optimise_level(lev, A, [0.0] * 7, mx, V)
    C = (1 << lev) * 1e4
    best, arg = float("inf"), None
    for dz in np.arange(1.0, 30.0, 0.02):
        for ds in np.arange(1.0, 30.0, 0.02):
            d = [dz, 1.0, 1.0, 1.0, 1.0, 1.0, ds]
            f = O.level_cost(V, C, A, e, d, lev)
            if f < best:
                best, arg = f, (dz, ds)
    assert O.level_cost(V, C, A, e, o["d_real"], lev) <= best * (1 + 1e-9)
    assert abs(o["d_real"][0] - arg[0]) < 0.05 and abs(o["d_real"][6] - arg[1]) < 0.05


def test_greedy_rounding_is_feasible_and_tight():
    lev = 3
    A, B, mx, V = _stats(lev, 2000)
    o = O.optimise_level(lev, A, B, mx, V)
    d_int, d_real, e = o["d"], o["d_real"], o["e"]
    assert O.v_indep(A, e, d_int) <= O.v_indep(A, e, d_real)
    assert all(di >= math.floor(dr) for di, dr in zip(d_int, d_real))
    assert sum(d_int) - sum(math.floor(x) for x in d_real) <= 7
    # removing the last greedy bit breaks the constraint
    added = [i for i in range(7) if d_int[i] > math.floor(d_real[i])]
    if added:
        assert any(O.v_indep(A, e, [d_int[j] - (j == i) for j in range(7)]) > O.v_indep(A, e, d_real)
                   for i in added)


def test_paper_level_cost_savings_and_trends():
    """Fig. 5 discussion: about 7x at level 0, 5x at level 1 against standard MLMC;
    Sec. 6.3: one more bit of S per level."""
    res = {}
    for lev in (0, 1, 2, 4, 6):
        A, B, mx, V = _stats(lev, 4000 if lev < 5 else 1500)
        res[lev] = O.optimise_level(lev, A, B, mx, V, c_rng=GOLD["c_rng"]["value"])
    lo, hi = GOLD["level_cost_saving_l0"]["band"]
    assert lo <= 1.0 / res[0]["level_cost_ratio"] <= hi
    lo, hi = GOLD["level_cost_saving_l1"]["band"]
    assert lo <= 1.0 / res[1]["level_cost_ratio"] <= hi
    slope = (res[6]["d_real"][6] - res[2]["d_real"][6]) / 4.0
    lo, hi = GOLD["d_S_per_level"]["band"]
    assert lo <= slope <= hi


def test_model_bounds_the_fixed_point_corrections():
    """Sec. 4.4: the simulated Var[DeltaP - DeltaP~] of the fixed-point path with the
    optimised widths respects the pessimistic bound with the approximate-Normal term
    (eq. extended) and is of the order of the optimistic one."""
    lev = 2
    A, B, mx, V = _stats(lev, 20000)
    o = O.optimise_level(lev, A, B, mx, V, mse_of_lut=lambda dl: MSE[dl])
    e, d = o["e"], o["d"]
    fmt = {"e": list(e), "f": [max(0, di - ei) for di, ei in zip(d, e)]}
    lut = o["lut_bits"]
    N = 20000
    s, _ = core.level(P, lev, 0, N, core.CORR_FIXED, 9, d=lut, method=1, fmt=fmt)
    disc = math.exp(-P["r"] * P["T"])
    m = disc * s["sum"] / N
    var = disc * disc * s["sum2"] / N - m * m
    v_corr_ext = (math.sqrt(o["v_corr"]) + B[0] * math.sqrt(MSE[lut])) ** 2
    v_indep_ext = o["v_indep"] + A[0] * MSE[lut]
    assert var <= v_corr_ext
    assert 0.1 * v_indep_ext <= var <= 10 * v_indep_ext
