"""Continuous-batching engine: each request's result is the same alone, in a
mix of other requests, and through mlmc_estimate (same algorithm and
arithmetic, work of other requests only shares the launches); prices agree
with Black-Scholes within their error bars; admission respects slots and the
memory budget."""
import math

import numpy as np
import pytest

from paper_2502_07123_gb300 import workloads as W
from tests.test_oracle_paths import black_scholes_call, black_scholes_digital

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


def _P(m, p, request, pack=1):
    return m.make_params(p, d=10, method=1, formats=[W.default_format(p, lev) for lev in range(11)],
                         request=request, rng_pack=pack)


def _run(eng, rids):
    out = {}
    for _ in range(10_000):
        active, queued = eng.step()
        for r in rids:
            if r not in out:
                res = eng.poll(r)
                if res is not None:
                    out[r] = res
        if len(out) == len(rids):
            return out
    raise AssertionError("engine did not finish")


@pytest.mark.parametrize("mode,scheme,payoff", [(1, W.EULER, W.EURO), (2, W.EULER, W.EURO), (9, W.EULER, W.EURO),
                                                (5, W.EULER, W.EURO), (2, W.MILSTEIN, W.ASIAN)])
def test_engine_equals_estimate_and_is_mix_independent(m, mode, scheme, payoff):
    """The device-side decision (a warp per slot) takes mlmc_estimate's FP64
    operations in mlmc_estimate's order: the same request gives the same price,
    standard error and L alone, in a mix, and through mlmc_estimate (exact low
    levels in mode 5; Milstein's variance decay 2^-2 in the last case)."""
    pA = W.params(payoff=payoff, scheme=scheme)
    eps = 0.02
    ref = m.mlmc_estimate(eps, _P(m, pA, 17), mode, 5, 10)
    # alone
    eng = m.Engine(max_slots=8, max_level=10)
    rid = eng.submit(_P(m, pA, 17), eps, mode, 5)
    alone = _run(eng, [rid])[rid]
    eng.close()
    assert alone["price"] == ref["price"] and alone["stderr"] == ref["stderr"] and alone["L"] == ref["L"]
    # in a mix of 40 other requests (different options, accuracies, payoffs), admitted over time
    opts = W.batched_options(40, seed=3)
    eng = m.Engine(max_slots=16, max_level=10)
    others = []
    for i, o in enumerate(opts[:20]):
        others.append(eng.submit(_P(m, o, 100 + i), max(o["eps"], 5e-3) * 4, mode, 5))
    eng.step()
    eng.step()
    ridA = eng.submit(_P(m, pA, 17), eps, mode, 5)
    for i, o in enumerate(opts[20:]):
        others.append(eng.submit(_P(m, o, 200 + i), max(o["eps"], 5e-3) * 4, mode, 5))
    res = _run(eng, [ridA] + others)
    st = eng.stats()
    eng.close()
    mixed = res[ridA]
    assert mixed["price"] == alone["price"] and mixed["stderr"] == alone["stderr"] and mixed["L"] == alone["L"]
    assert st["launches"] < st["steps"] * 2   # many requests per launch


def test_engine_prices_match_black_scholes(m):
    eng = m.Engine(max_slots=32, max_level=10)
    cases = []
    rng = np.random.default_rng(4)
    for i in range(24):
        p = W.params(S0=float(rng.uniform(80, 120)), K=float(rng.uniform(80, 120)),
                     sigma=float(rng.uniform(0.1, 0.4)), T=float(rng.uniform(0.25, 2.0)),
                     payoff=int(rng.integers(0, 2)))
        eps = float(np.exp(rng.uniform(np.log(0.01), np.log(0.05))))
        rid = eng.submit(_P(m, p, i), eps, 2, 11)
        cases.append((rid, p, eps))
    res = _run(eng, [c[0] for c in cases])
    eng.close()
    z = []
    for rid, p, eps in cases:
        f = black_scholes_call if p["payoff"] == W.EURO else black_scholes_digital
        ref = f(p["S0"], p["K"], p["r"], p["sigma"], p["T"])
        r = res[rid]
        assert abs(r["price"] - ref) < 4 * r["stderr"] + eps / math.sqrt(2), (p, r, ref)
        z.append((r["price"] - ref) / eps)
    assert math.sqrt(np.mean(np.square(z))) < 1.5   # RMS error about eps


def test_engine_admission_by_slots_and_memory(m):
    eng = m.Engine(max_slots=3, max_level=8)
    assert eng.stats()["slots"] == 3
    rids = [eng.submit(_P(m, W.params(), i), 0.05, 1, 9) for i in range(7)]
    a, q = eng.step()
    assert a <= 3 and q == 4
    res = _run(eng, rids)
    assert len(res) == 7
    eng.close()
    with pytest.raises(m.MLMCError) as e:
        m.Engine(max_slots=4, max_level=8, device_bytes_budget=64)
    assert e.value.status == m.ENOMEM
    small = m.Engine(max_slots=100, max_level=8, device_bytes_budget=1 << 20)
    assert 1 <= small.stats()["slots"] < 100
    small.close()


def test_engine_graph_iterations_and_partial_growth(m):
    """One graph launch per step (captured once per new launch class); an
    iteration that needs more chunks than the partial array holds grows the
    array and reruns, with the same result as mlmc_estimate."""
    pA = W.params(payoff=W.EURO)
    eps = 4e-4      # about 5e9 approximate samples on level 0: > 65536 chunks in one iteration
    ref = m.mlmc_estimate(eps, _P(m, pA, 3), 2, 21, 10)
    eng = m.Engine(max_slots=1, max_level=10)
    cap0 = eng.graph_info()["partial_capacity"]
    rid = eng.submit(_P(m, pA, 3), eps, 2, 21)
    res = _run(eng, [rid])[rid]
    gi = eng.graph_info()
    st = eng.stats()
    eng.close()
    assert res["price"] == ref["price"] and res["stderr"] == ref["stderr"] and res["L"] == ref["L"]
    assert gi["partial_capacity"] > cap0
    assert 2 <= gi["groups"] <= 4         # approximate (packed) and correction kernels, 32- or 64-bit S
    assert gi["captures"] <= 1 + 5        # first capture plus one per growth of the partial array
    assert st["launches"] >= st["steps"]


@pytest.mark.parametrize("iters", [1, 4])
def test_batch_estimate_equals_estimate(m, iters):
    """mlmc_batch_estimate: a mixed batch (payoffs, accuracies, options) in one
    engine; each result equals mlmc_estimate of that request alone."""
    opts = W.batched_options(12, seed=5)
    plist, eps = [], []
    for i, o in enumerate(opts):
        plist.append(_P(m, o, 300 + i))
        eps.append(max(o["eps"], 4e-3) * 5)
    out = m.mlmc_batch_estimate(plist, eps, 5, 13, max_level=10, iters_per_launch=iters)
    for i in range(len(opts)):
        ref = m.mlmc_estimate(eps[i], plist[i], 5, 13, 10)
        assert out["price"][i] == ref["price"] and out["stderr"][i] == ref["stderr"], i
        assert out["L"][i] == ref["L"]
    assert out["launches"] >= 1
    if iters > 1:
        single = m.mlmc_batch_estimate(plist, eps, 5, 13, max_level=10, iters_per_launch=1)
        assert out["launches"] < single["launches"]


def test_engine_rejects_unfit_request_without_failing_others(m):
    """A request whose fixed-point formats cannot hold its constants completes
    with MLMC_EOVERFLOW; the others run."""
    p = W.params()
    bad = [dict(e=list(f["e"]), f=list(f["f"])) for f in (W.default_format(p, lev) for lev in range(11))]
    bad[1]["e"][6] = 2        # S in 2 integer bits cannot hold S0 = 100
    eng = m.Engine(max_slots=4, max_level=10)
    r_bad = eng.submit(m.make_params(p, d=10, method=1, formats=bad, request=1), 0.05, 2, 3)
    r_ok = eng.submit(_P(m, p, 2), 0.05, 2, 3)
    with pytest.raises(m.MLMCError) as e:
        _run(eng, [r_bad, r_ok])
    assert e.value.status == m.EOVERFLOW
    res = _run(eng, [r_ok])
    eng.close()
    assert math.isfinite(res[r_ok]["price"])


def test_engine_reuses_launch_classes_across_seeds(m):
    """Launch classes include the seed: an engine serving one request at a time
    with 40 different seeds reuses the classes of finished requests."""
    p = W.params()
    eng = m.Engine(max_slots=1, max_level=10)
    for seed in range(40):
        rid = eng.submit(_P(m, p, 1), 0.05, 5, 1000 + seed)
        res = _run(eng, [rid])[rid]
        assert math.isfinite(res["price"])
    assert eng.graph_info()["groups"] <= 32
    eng.close()


def test_batch_in_one_device_loop(m):
    """iters_per_launch < 0: the whole batch runs as one graph launch whose
    conditional WHILE node iterates on the device until every request is
    done; the results equal mlmc_estimate's."""
    opts = W.batched_options(10, seed=8)
    plist = [_P(m, o, 400 + i) for i, o in enumerate(opts)]
    eps = [max(o["eps"], 4e-3) * 5 for o in opts]
    out = m.mlmc_batch_estimate(plist, eps, 5, 17, max_level=10, iters_per_launch=-4096)
    for i in range(len(opts)):
        ref = m.mlmc_estimate(eps[i], plist[i], 5, 17, 10)
        assert out["price"][i] == ref["price"] and out["stderr"][i] == ref["stderr"], i
    assert out["launches"] <= 3      # one, plus a relaunch per growth of the partial array


@pytest.mark.parametrize("mode", [3, 5, 6])
def test_engine_mixed_methods_equal_estimate(m, mode):
    """Requests with Methods 1, 2 and 3 (and packed / unpacked draws) share the
    engine's launches; each result equals mlmc_estimate's."""
    p = W.params(payoff=W.EURO)
    reqs = []
    for i, (method, pack) in enumerate(((1, 1), (2, 1), (3, 0), (2, 0))):
        P = m.make_params(p, d=10, method=method, formats=[W.default_format(p, k) for k in range(11)],
                          request=50 + i, rng_pack=pack)
        reqs.append(P)
    eng = m.Engine(max_slots=8, max_level=10)
    rids = [eng.submit(P, 0.03, mode, 23) for P in reqs]
    res = _run(eng, rids)
    eng.close()
    for P, rid in zip(reqs, rids):
        ref = m.mlmc_estimate(0.03, P, mode, 23, 10)
        assert res[rid]["price"] == ref["price"] and res[rid]["stderr"] == ref["stderr"]


def test_engine_completed_drains_each_request_once(m):
    """mlmc_engine_completed hands out every finished request exactly once, in
    the step it finished (a failed admission included), and only finished ones."""
    p = W.params()
    bad = [dict(e=list(f["e"]), f=list(f["f"])) for f in (W.default_format(p, lev) for lev in range(11))]
    bad[1]["e"][6] = 2        # S in 2 integer bits cannot hold S0 = 100
    eng = m.Engine(max_slots=3, max_level=10)
    rids = [eng.submit(_P(m, W.params(sigma=0.1 + 0.05 * i), 60 + i), 0.05 - 0.004 * i, 5, 31) for i in range(6)]
    r_bad = eng.submit(m.make_params(p, d=10, method=1, formats=bad, request=99), 0.05, 5, 31)
    assert eng.completed() == []
    seen = []
    for _ in range(10_000):
        eng.step()
        got = eng.completed(cap=2)
        got += eng.completed()           # the rest of this step's completions
        for rid in got:
            assert rid not in seen
            if rid != r_bad:
                assert eng.poll(rid) is not None
            else:
                with pytest.raises(m.MLMCError) as e:
                    eng.poll(rid)
                assert e.value.status == m.EOVERFLOW
        for rid in set(rids) - set(seen) - set(got):
            assert eng.poll(rid) is None   # not handed out: not finished
        seen += got
        if len(seen) == len(rids) + 1:
            break
    assert sorted(seen) == sorted(rids + [r_bad])
    assert eng.completed() == []
    eng.close()
