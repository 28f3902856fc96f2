"""Serving accuracy against the FP64 oracle (the batched / serving workload).

Requests drawn as the batched workload (European, digital and Asian calls
with uneven S0, K, sigma, T and accuracies) run together in one
continuous-batching engine with fewer slots than requests, so that requests
are admitted while others run.  Each request's schedule
(mlmc_engine_request_info) is then priced by the oracle on the same samples
(packed draws, enumerated low levels of mode 5), and the engine's price and
variance must agree within the per-sample FP32 path bound
(gpu_helpers.schedule_bounds).  A request that stopped at max_level reports
a bias estimate; one that met its bias test reports one at most eps/sqrt(2)."""
import math

import pytest

from oracle import driver
from paper_2502_07123_gb300 import workloads as W
from tests.gpu_helpers import schedule_bounds

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


def test_engine_requests_equal_oracle_on_their_schedules(m):
    max_level, mode, seed = 10, driver.NESTED_FIXED_EXACT_LOW, 31
    opts = W.batched_options(10, seed=23, eps_range=(3e-2, 8e-2))
    fmts = [[W.default_format(o, lev) for lev in range(max_level + 1)] for o in opts]
    eng = m.Engine(max_slots=3, max_level=max_level)
    rids = [eng.submit(m.make_params(o, d=10, method=1, formats=fmts[i], request=i, rng_pack=1), o["eps"], mode,
                       seed) for i, o in enumerate(opts)]
    done = {}
    for _ in range(10000):
        if len(done) == len(opts):
            break
        eng.step()
        for i, r in enumerate(rids):
            if i not in done:
                res = eng.poll(r)
                if res is not None:
                    done[i] = (res, eng.request_info(r))
    eng.close()
    assert len(done) == len(opts)
    payoffs = set()
    for i, o in enumerate(opts):
        res, info = done[i]
        N = info["N"]
        assert len(N) == res["L"] + 1
        payoffs.add(o["payoff"])
        orc = driver.price_on_schedule(o, seed, mode, N, fmt_of_level=lambda lev: fmts[i][lev], request=i, pack=1,
                                       dump=True)
        tol_p, tol_v, terms = schedule_bounds(mode, o, orc["dumps"], N)
        assert abs(res["price"] - orc["price"]) <= tol_p + 1e-12 * terms * (abs(orc["price"]) + 1.0), \
            (i, res["price"], orc["price"], tol_p)
        var = res["stderr"] ** 2
        assert abs(var - orc["var"]) <= tol_v + 1e-10 * orc["var"], (i, var, orc["var"], tol_v)
        assert var <= 0.5 * o["eps"] ** 2 * (1 + 1e-9)
        if res["L"] < max_level:
            assert info["bias_estimate"] <= o["eps"] / math.sqrt(2) * (1 + 1e-12)
    assert payoffs == {W.EURO, W.DIGITAL, W.ASIAN}
