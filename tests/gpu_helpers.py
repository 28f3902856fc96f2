"""Shared helpers of the GPU parity tests (comparison rules and tolerances)."""
import numpy as np

from oracle import core

# FP32 exact path: 1e-5 relative per path (terminal value and path functionals)
RTOL_F32 = 1e-5
# FP64 exact path: GPU normcdfinv / fused multiply-adds against the oracle's Newton inverse
RTOL_F64 = 1e-12

APPROX_ONLY = core.APPROX_ONLY_VARIANTS
CORR = core.CORR_VARIANTS


def exact_rtol(variant):
    return RTOL_F64 if variant == core.FP64_EXACT else RTOL_F32


def compare_samples(variant, p, g, o):
    """Element-wise parity of one dump against the oracle's dump of the same samples."""
    assert g.shape == o.shape
    if core.has_approx(variant):
        # integer / IEEE-emulated work: bit-exact
        for f in ("qf", "qc", "af", "ac", "sat"):
            bad = np.nonzero(g[f] != o[f])[0]
            assert bad.size == 0, (f, bad[:5], g[f][bad[:5]], o[f][bad[:5]])
    if core.has_exact(variant):
        rt = exact_rtol(variant)
        for f in ("sf", "sc"):
            err = np.abs(g[f] - o[f])
            assert np.all(err <= rt * np.abs(o[f]) + 1e-300), (f, float(np.max(err / np.maximum(np.abs(o[f]), 1e-300))))
        scale = np.maximum(np.abs(o["sf"]), p["K"]) + np.abs(o["sc"])
        for f in ("pf", "pc"):
            err = np.abs(g[f] - o[f])
            if p["payoff"] == core.DIGITAL:
                s = o["sf"] if f == "pf" else o["sc"]
                near = np.abs(s - p["K"]) <= 4 * rt * np.abs(s)
                assert np.all((err == 0) | near), f
            else:
                assert np.all(err <= 4 * rt * scale), (f, float(np.max(err / scale)))
    # the sample value
    if variant in APPROX_ONLY:
        assert np.array_equal(g["y"], o["y"])
    else:
        tol = y_tolerance(variant, p, o)
        err = np.abs(g["y"] - o["y"])
        assert np.all(err <= tol), float(np.max(err - tol))


def y_tolerance(variant, p, o):
    """Per-sample bound on |Y_gpu - Y_oracle| from the oracle's records o: zero for
    the integer estimators; for real ones 8 rt times the path scale (terminal
    values against the strike), a digital payoff either way where S_N is within
    the path bound of K, and for corrections the FP32 rounding of the
    approximate part."""
    if variant in APPROX_ONLY:
        return np.zeros(len(o))
    rt = exact_rtol(variant)
    scale = np.maximum(np.abs(o["sf"]), p["K"]) + np.abs(o["sc"])
    tol = 8 * rt * scale
    if p["payoff"] == core.DIGITAL:
        near = (np.abs(o["sf"] - p["K"]) <= 4 * rt * o["sf"]) | (np.abs(o["sc"] - p["K"]) <= 4 * rt * np.abs(o["sc"]))
        tol = np.where(near, 1.0 + 1e-9, tol)
    if variant in CORR:
        tol = tol + 2.0**-22 * np.abs(o["y"] - (o["pf"] - o["pc"])) + 1e-30
    return tol


def schedule_bounds(mode, p, dumps, N, d=10):
    """Bounds on |price_gpu - price_oracle| and |var_gpu - var_oracle| for a
    schedule N[l][k] priced by the oracle with per-sample records `dumps`
    (oracle.driver.price_on_schedule(..., dump=True)): the mean of each term's
    per-sample bounds, and the bound those imply for its variance estimate;
    enumerated terms (exact low levels) carry no variance."""
    import math
    from oracle import driver
    plan = driver.estimator_plan(mode)
    exact = driver.exact_levels(mode, d)
    disc = math.exp(-p["r"] * p["T"])
    tol_p, tol_v, terms = 0.0, 0.0, 0
    for lev, row in enumerate(N):
        for k, n in enumerate(row[:len(plan)]):
            terms += 1
            dm_rec = dumps[lev][k]
            t = disc * y_tolerance(plan[k], p, dm_rec)
            y = disc * dm_rec["y"]
            dm = float(np.sum(t)) / n
            tol_p += dm
            if not (k == 0 and lev in exact):
                m_ = float(np.mean(y))
                d2 = float(np.sum((2 * np.abs(y) + t) * t)) / n
                tol_v += (d2 + (2 * abs(m_) + dm) * dm) / n
    return tol_p, tol_v, terms
