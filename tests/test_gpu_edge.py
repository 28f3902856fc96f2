"""Edge cases through the C ABI against the oracle: empty and one-sample
items, the deepest levels, the smallest and largest table sizes, a
zero-volatility market (every sample identical; zero variance; the
adaptive driver must still terminate on the deterministic price), a zero
strike, and the size limits (rejected before any launch)."""
import math

import numpy as np
import pytest

from oracle import core
from paper_2502_07123_gb300 import workloads as W
from tests.gpu_helpers import compare_samples

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2502_07123_gb300 import mlmc
    return mlmc


def _P(m, p, lev_max=12, d=10, method=1, pack=0):
    return m.make_params(p, d=d, method=method, formats=[W.default_format(p, k) for k in range(lev_max + 1)],
                         rng_pack=pack)


def test_empty_items_and_single_samples(m):
    p = W.params()
    P = _P(m, p)
    items = [dict(params=P, level=3, variant=W.FIXED_APPROX, N=0),
             dict(params=P, level=2, variant=W.CORR_FIXED, N=1, first_sample=77),
             dict(params=P, level=0, variant=W.FP32_EXACT, N=0),
             dict(params=P, level=5, variant=W.FIXED_APPROX, N=1, first_sample=5)]
    for _ in range(2):                         # twice: the per-item counters reset
        r = m.mlmc_run(items, 31)
        assert r[0]["n"] == 0 and r[0]["sum"] == 0.0 and r[0]["isum"] == 0 and r[0]["sum2"] == 0.0
        assert r[2]["n"] == 0 and r[2]["sum"] == 0.0
        o1, _ = core.level(p, 2, 77, 1, core.CORR_FIXED, 31, fmt=W.default_format(p, 2))
        o3, _ = core.level(p, 5, 5, 1, core.FIXED_APPROX, 31, fmt=W.default_format(p, 5))
        assert r[3]["isum"] == o3["isum"]
        assert r[1]["sum"] == pytest.approx(math.exp(-p["r"] * p["T"]) * o1["sum"], rel=1e-4, abs=1e-6)
    assert m.mlmc_level(4, 0, P, W.FP32_EXACT, 1)["sum"] == 0.0


@pytest.mark.parametrize("level", [10, 12])
@pytest.mark.parametrize("variant", [core.FP32_EXACT, core.FIXED_APPROX, core.CORR_FIXED, core.FP16_APPROX])
def test_deep_levels(m, level, variant):
    p = W.params(payoff=W.EURO)
    fm = [W.default_format(p, k) for k in range(level + 1)]
    P = m.make_params(p, d=10, method=1, formats=fm)
    _, od = core.level(p, level, 3, 40, variant, 8, fmt=fm[level], dump=True)
    _, gd = m.mlmc_level_dump(level, 40, P, variant, 8, 3)
    compare_samples(variant, p, gd, od)


@pytest.mark.parametrize("d", [2, 3, 14])
@pytest.mark.parametrize("variant", [core.FIXED_APPROX, core.CORR_FIXED, core.CORR_FP16])
def test_table_size_extremes(m, d, variant):
    p = W.params(payoff=W.DIGITAL)
    fm = [W.default_format(p, k) for k in range(3)]
    P = m.make_params(p, d=d, method=1, formats=fm)
    _, od = core.level(p, 2, 0, 500, variant, 12, d=d, fmt=fm[2], dump=True)
    _, gd = m.mlmc_level_dump(2, 500, P, variant, 12, 0)
    compare_samples(variant, p, gd, od)


def test_zero_volatility(m):
    """sigma = 0: every path is S0 (1 + r h)^n; corrections and level variances vanish
    on the exact path, and the adaptive driver stops at the deterministic price."""
    p = W.params(sigma=0.0)
    P = _P(m, p, 10)
    g = m.mlmc_level_dump(3, 64, P, W.FP32_EXACT, 5)[1]
    sf = p["S0"] * (1 + p["r"] / 8) ** 8
    np.testing.assert_allclose(g["sf"], sf, rtol=1e-6)
    assert np.all(g["sf"] == g["sf"][0])
    _, od = core.level(p, 3, 0, 64, core.CORR_FIXED, 5, fmt=W.default_format(p, 3), dump=True)
    _, gd = m.mlmc_level_dump(3, 64, P, W.CORR_FIXED, 5)
    compare_samples(core.CORR_FIXED, p, gd, od)
    for mode in (1, 2, 5):
        r = m.mlmc_estimate(1e-3, P, mode, 3, 10)
        L = r["L"]
        exact_em = math.exp(-p["r"] * p["T"]) * max(p["S0"] * (1 + p["r"] / 2 ** L) ** (2 ** L) - p["K"], 0.0)
        assert math.isfinite(r["price"]) and r["stderr"] < 1e-3
        assert abs(r["price"] - exact_em) < 2e-3, (mode, r, exact_em)


def test_zero_strike(m):
    """K = 0: the call is the forward; E[e^{-rT} S_N] = S0 (1 + r h)^N e^{-rT} on level L."""
    p = W.params(K=0.0)
    P = _P(m, p, 10)
    r = m.mlmc_estimate(0.02, P, 5, 9, 10)
    assert abs(r["price"] - p["S0"]) < 4 * r["stderr"] + 0.02


def test_size_limits_rejected(m):
    P = _P(m, W.params())
    with pytest.raises(m.MLMCError) as e:
        m.mlmc_level(2, (1 << 58) + 1, P, W.FP32_EXACT, 1)
    assert e.value.status == m.EINVAL
    with pytest.raises(m.MLMCError) as e:
        m.mlmc_level(10, 100, P, W.FP32_EXACT, 1, first_sample=(1 << 50))
    assert e.value.status == m.EINVAL
    with pytest.raises(m.MLMCError) as e:
        m.mlmc_level(21, 100, P, W.FP32_EXACT, 1)
    assert e.value.status == m.EINVAL


def test_calls_from_several_threads(m):
    """Concurrent calls from host threads are serialised by the library and give
    the results of the same calls made one after another."""
    import threading
    p = W.params()
    P = _P(m, p, 8, pack=1)
    cases = [(lev, v) for lev in (1, 3, 6) for v in (W.FIXED_APPROX, W.CORR_FIXED, W.FP32_EXACT)]
    seq = [m.mlmc_level(lev, 20_000, P, v, 99) for lev, v in cases]
    out = [None] * len(cases)

    def work(i):
        lev, v = cases[i]
        out[i] = m.mlmc_level(lev, 20_000, P, v, 99)

    ts = [threading.Thread(target=work, args=(i,)) for i in range(len(cases))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for a, b in zip(seq, out):
        assert a["sum"] == b["sum"] and a["sum2"] == b["sum2"]


def test_plan_launch_items_partition_the_work(m):
    # every item with samples is in exactly one level-kernel launch, whose
    # family and path-steps its items account for; empty items are in none
    p = W.params()
    P = _P(m, p, pack=1)
    items = [dict(params=P, level=lev, variant=v, N=n)
             for lev, n in ((0, 400_000), (2, 400_000), (5, 1_000), (7, 0))
             for v in (W.FIXED_APPROX, W.CORR_FIXED, W.FP32_EXACT)]
    plan = m.Plan(items, 9)
    try:
        seen = []
        for k in range(plan.info()["kernels"]):
            fam, n_items, _, ps = plan.launch_info(k)
            idx = plan.launch_items(k)
            assert len(idx) == n_items > 0
            assert ps == sum(items[i]["N"] << items[i]["level"] for i in idx)
            variants = {items[i]["variant"] for i in idx}
            if fam in (17, 24):
                # the merged nested launch: 32-bit fixed-point approximate and correction chunks
                assert variants <= {W.FIXED_APPROX, W.CORR_FIXED} and len(variants) == 2
            else:
                assert len(variants) == 1
            seen += idx
        assert sorted(seen) == [i for i, it in enumerate(items) if it["N"] > 0]
        with pytest.raises(m.MLMCError):
            plan.launch_items(plan.info()["kernels"])
    finally:
        plan.close()


def test_plan_elapsed_brackets_the_launch(m):
    # mlmc_plan_elapsed: the whole launch's device time; a one-kernel plan is
    # timed by the same events as its kernel, a plan of several launches by
    # events around all of them (and its items with no samples read zero)
    p = W.params()
    P = _P(m, p, pack=1)
    one = m.Plan([dict(params=P, level=3, variant=W.FIXED_APPROX, N=300_000)], 5)
    several = m.Plan([dict(params=P, level=lev, variant=v, N=n)
                      for lev, n in ((0, 400_000), (4, 20_000), (6, 0))
                      for v in (W.FIXED_APPROX, W.FP32_EXACT)], 5)
    try:
        with pytest.raises(m.MLMCError) as e:
            one.elapsed_ms()
        assert e.value.status == m.ENOTREADY
        one.launch()
        assert one.info()["kernels"] == 1
        assert one.elapsed_ms() == one.kernel_time(0)[1] > 0.0
        several.launch()
        k = several.info()["kernels"]
        assert k >= 2
        total = several.elapsed_ms()
        assert all(0.0 < several.kernel_time(j)[1] <= total for j in range(k))
        res = several.results()
        assert all(r["n"] == 0 and r["sum"] == 0.0 and r["sum2"] == 0.0 for r in res[4:])
    finally:
        one.close()
        several.close()


def test_worklist_and_raw_results(m):
    # a marshalled-once work list and the structured-array results give the
    # same sums as the list-of-dicts call
    p = W.params()
    P = _P(m, p, pack=1)
    items = [dict(params=P, level=lev, variant=v, N=2000 + lev, first_sample=lev)
             for lev in (0, 2, 5) for v in (W.FIXED_APPROX, W.CORR_FIXED, W.FP32_EXACT)]
    a = m.mlmc_run(items, 21)
    wl = m.WorkList(items)
    b = m.mlmc_run(wl, 21)
    raw = m.mlmc_run(wl, 21, raw=True)
    plan = m.Plan(wl, 21)
    try:
        plan.launch()
        c = plan.results(raw=True)
    finally:
        plan.close()
    for i, x in enumerate(a):
        assert x["isum"] == b[i]["isum"] and x["isum2"] == b[i]["isum2"] and x["sum"] == b[i]["sum"]
        assert raw[i]["sum"] == x["sum"] and raw[i]["sum2"] == x["sum2"] and raw[i]["isum"] == x["isum"]
        assert (int(raw[i]["isum2_hi"]) << 64 | int(raw[i]["isum2_lo"])) == x["isum2"]
        assert c[i]["sum"] == x["sum"] and c[i]["n"] == x["n"]


@pytest.mark.parametrize("sigma,family", [(0.2, 24), (0.6, 17)])
def test_merged_nested_launch_equals_separate_items(m, sigma, family):
    # approximate (packed and one sample per thread) and correction items of the
    # 32-bit fixed-point datapath share one launch of the merged kernel (family
    # 17, or 24 in its pre-scaled form); each item's sums equal those of the item run alone: integer sums bit
    # for bit, real sums to FP64 rounding (the chunkings differ).  With sigma 0.6
    # the coarse increments of the low levels are too large for the pre-scaled
    # product (|sum1| < 2^(rs2 - 1)), so the launch keeps the funnel-shift form.
    p = W.params(payoff=W.DIGITAL, sigma=sigma)
    P = _P(m, p, pack=1)
    items = [dict(params=P, level=0, variant=W.FIXED_APPROX, N=300_001, first_sample=7),
             dict(params=P, level=3, variant=W.FIXED_APPROX, N=5_000),
             dict(params=P, level=6, variant=W.FIXED_APPROX, N=40_000),
             dict(params=P, level=1, variant=W.CORR_FIXED, N=20_000, first_sample=3),
             dict(params=P, level=7, variant=W.CORR_FIXED, N=3_000)]
    plan = m.Plan(items, 21)
    try:
        assert plan.info()["kernels"] == 1 and plan.launch_info(0)[0] == family
        plan.launch()
        res = plan.results()
    finally:
        plan.close()
    for it, r in zip(items, res):
        one = m.mlmc_level(it["level"], it["N"], P, it["variant"], 21, it.get("first_sample", 0))
        if it["variant"] == W.FIXED_APPROX:
            assert r["isum"] == one["isum"] and r["isum2"] == one["isum2"] and r["sum"] == one["sum"]
        else:
            assert abs(r["sum"] - one["sum"]) <= 1e-12 * (r["n"] * r["sum2"]) ** 0.5
            assert abs(r["sum2"] - one["sum2"]) <= 1e-12 * r["sum2"]


def test_run_plan_cache_follows_the_work_list(m):
    # mlmc_run keeps host-built plans by the contents of the work list: the same
    # list gives the same bits, and a parameter changed in place (the same ctypes
    # objects, so the same pointers) gives the result of the new parameters
    p = W.params()
    P = _P(m, p, pack=1)
    items = [dict(params=P, level=2, variant=W.FIXED_APPROX, N=50_000),
             dict(params=P, level=4, variant=W.CORR_FIXED, N=3_000)]
    work = m.WorkList(items)

    def sums(res):   # everything but the launch's device time
        return [{k: v for k, v in r.items() if k != "seconds"} for r in res]
    a = sums(m.mlmc_run(work, 5))
    assert sums(m.mlmc_run(work, 5)) == a
    P.K = 102.0      # within the format table built for K = 100
    c = m.mlmc_run(work, 5)
    ref = m.mlmc_level(2, 50_000, P, W.FIXED_APPROX, 5)
    assert c[0]["isum"] == ref["isum"] and c[0]["isum2"] == ref["isum2"] and c[0]["isum"] != a[0]["isum"]
    P.K = p["K"]
    assert sums(m.mlmc_run(work, 5)) == a


def test_item_lookup_over_many_items(m):
    # a launch of 1500 items (three rounds of the CTAs' warp-ballot item
    # lookup): every item's exact integer sums equal the item run alone
    p = W.params()
    P = _P(m, p, pack=1)
    rng = np.random.default_rng(5)
    items = []
    for i in range(1500):
        lev = int(rng.integers(0, 4))
        items.append(dict(params=P, level=lev, variant=W.FIXED_APPROX, N=int(rng.integers(1, 400)),
                          first_sample=int(rng.integers(0, 10_000))))
    plan = m.Plan(items, 13)
    try:
        assert plan.info()["kernels"] == 1
        assert plan.launch_info(0)[1] == len(items)
        plan.launch()
        res = plan.results()
    finally:
        plan.close()
    for k in rng.choice(len(items), 60, replace=False):
        it = items[k]
        one = m.mlmc_level(it["level"], it["N"], P, W.FIXED_APPROX, 13, it["first_sample"])
        assert res[k]["isum"] == one["isum"] and res[k]["isum2"] == one["isum2"], k


def test_run_replay_follows_the_seed(m):
    # mlmc_run replays a cached single-launch plan as a CUDA graph; a new seed
    # (new round keys in the kernel's parameters) is captured again, so each
    # seed's sums equal those computed item by item
    p = W.params()
    P = _P(m, p, pack=1)
    items = [dict(params=P, level=1, variant=W.FIXED_APPROX, N=30_000),
             dict(params=P, level=3, variant=W.FIXED_APPROX, N=7_000, first_sample=11)]
    for seed in (5, 6, 5, 6):
        res = m.mlmc_run(items, seed)
        for it, r in zip(items, res):
            one = m.mlmc_level(it["level"], it["N"], P, W.FIXED_APPROX, seed, it.get("first_sample", 0))
            assert r["isum"] == one["isum"] and r["isum2"] == one["isum2"], seed
