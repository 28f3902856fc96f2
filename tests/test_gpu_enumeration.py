"""Exact approximate terms on levels 0 and 1 (enumeration of the table cells)
on the GPU: exact integer sums equal the oracle's; the adaptive modes built on
them agree between mlmc_estimate and the engine and with Black-Scholes."""
import math

import pytest

from oracle import core
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


@pytest.mark.parametrize("variant", [core.FIXED_APPROX, core.FP16_APPROX])
@pytest.mark.parametrize("level,d", [(0, 10), (0, 14), (1, 8), (1, 10)])
@pytest.mark.parametrize("payoff", [W.EURO, W.DIGITAL, W.ASIAN, W.LOOKBACK])
def test_enumeration_sums_bit_exact(m, variant, level, d, payoff):
    p = W.params(payoff=payoff, scheme=W.MILSTEIN if payoff == W.ASIAN else W.EULER)
    fmts = [W.default_format(p, lev) for lev in range(2)]
    P = m.make_params(p, d=d, method=1, formats=fmts, rng_pack=1)
    n = 1 << (d << level)
    res = m.mlmc_run([dict(params=P, level=level, variant=variant, N=n, flags=m.WORK_ENUMERATE)], seed=3)[0]
    o, _ = core.level(p, level, 0, n, variant, 3, d=d, fmt=fmts[level], enumerate=1)
    assert res["isum"] == o["isum"] and res["isum2"] == o["isum2"]


def test_enumeration_rejects_bad_items(m):
    p = W.params()
    P = m.make_params(p, d=10, method=1)
    for item in (dict(level=2, N=1 << 40), dict(level=0, N=1000), dict(level=0, N=1024, first_sample=1)):
        with pytest.raises(m.MLMCError) as e:
            m.mlmc_run([dict(params=P, variant=m.FIXED_APPROX, flags=m.WORK_ENUMERATE, **item)], seed=1)
        assert e.value.status == m.EINVAL
    with pytest.raises(m.MLMCError):
        m.mlmc_run([dict(params=P, level=0, N=1024, variant=m.NESTED_CORR_FIXED, flags=m.WORK_ENUMERATE)], seed=1)


@pytest.mark.parametrize("mode", [5, 6])
@pytest.mark.parametrize("payoff,bs", [(W.EURO, black_scholes_call), (W.DIGITAL, black_scholes_digital)])
def test_exact_low_modes(m, mode, payoff, bs):
    p = W.params(payoff=payoff)
    P = m.make_params(p, d=10, method=1, formats=[W.default_format(p, lev) for lev in range(11)], rng_pack=1)
    eps = 0.01 if payoff == W.EURO else 0.002
    est = m.mlmc_estimate(eps, P, mode, 21, 10)
    assert est["N"][0][0] == 1 << 10 and est["N"][1][0] == 1 << 20
    ref = bs(p["S0"], p["K"], p["r"], p["sigma"], p["T"])
    assert abs(est["price"] - ref) < 4 * est["stderr"] + eps / math.sqrt(2)
    eng = m.Engine(max_slots=4, max_level=10)
    rid = eng.submit(P, eps, mode, 21)
    while True:
        eng.step()
        r = eng.poll(rid)
        if r is not None:
            break
    eng.close()
    assert r["price"] == est["price"] and r["stderr"] == est["stderr"] and r["L"] == est["L"]
