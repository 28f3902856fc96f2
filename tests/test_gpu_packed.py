"""Packed draws (three lockstep samples per Philox word) of the approximate-only
estimators: every datapath against the oracle's packed definition, sample by
sample and in the exact integer sums, across chunk boundaries and ragged ends."""
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


CASES = [(v, s, pay, lev, d) for v in (core.FIXED_APPROX, core.FP16_APPROX, core.BF16_APPROX)
         for s in (W.EULER, W.MILSTEIN) for pay in (W.EURO, W.DIGITAL, W.ASIAN, W.LOOKBACK)
         for lev, d in ((0, 10), (1, 9), (2, 10), (3, 10), (6, 9))]


@pytest.mark.parametrize("variant,scheme,payoff,level,d", CASES)
def test_packed_samples(m, variant, scheme, payoff, level, d):
    p = W.params(scheme=scheme, payoff=payoff, sigma=0.3)
    fmts = [W.default_format(p, lev) for lev in range(level + 1)]
    method = 3 if (level + payoff) % 2 else 1
    seed, first, N = 77 + level, 5, 293        # ragged at both ends of the packs
    P = m.make_params(p, d=d, method=method, formats=fmts, request=2, rng_pack=1)
    gs, gd = m.mlmc_level_dump(level, N, P, variant, seed, first)
    os_, od = core.level(p, level, first, N, variant, seed, request=2, d=d, method=method,
                         fmt=fmts[level], dump=True, pack=1)
    compare_samples(variant, p, gd, od)
    assert gs["isum"] == os_["isum"] and gs["isum2"] == os_["isum2"]


@pytest.mark.parametrize("level", [0, 1, 2, 4, 8])
def test_packed_multichunk_sums(m, level):
    p = W.params()
    fmts = [W.default_format(p, lev) for lev in range(level + 1)]
    P = m.make_params(p, d=10, method=1, formats=fmts, rng_pack=1)
    N, first = (100_003 if level < 4 else 3_001), 2
    res = m.mlmc_run([dict(params=P, level=level, variant=m.FIXED_APPROX, first_sample=first, N=N)], seed=11,
                     tuning=dict(threads=32, steps_per_thread=1))[0]
    o, _ = core.level(p, level, first, N, core.FIXED_APPROX, 11, fmt=fmts[level], pack=1)
    assert res["isum"] == o["isum"] and res["isum2"] == o["isum2"] and res["saturations"] == o["saturations"]


def test_packing_rules(m):
    p = W.params()
    P12 = m.make_params(p, d=12, method=1, rng_pack=1)
    with pytest.raises(m.MLMCError) as e:
        m.mlmc_level(2, 100, P12, m.FIXED_APPROX, 1)      # 32 // 12 != 3 fields
    assert e.value.status == m.EINVAL
    # exact and correction estimators ignore the flag (they need all 32 bits of J)
    Pp = m.make_params(p, d=10, method=1, rng_pack=1)
    Pu = m.make_params(p, d=10, method=1, rng_pack=0)
    for v in (m.FP32_EXACT, m.NESTED_CORR_FIXED):
        a = m.mlmc_level(3, 2000, Pp, v, 5)
        b = m.mlmc_level(3, 2000, Pu, v, 5)
        assert a["sum"] == b["sum"] and a["sum2"] == b["sum2"]


# Items with at least one wave of packs run three lockstep lanes per thread; on
# the binary16 / bfloat16 datapaths lanes 0 and 1 share paired (x2) instructions.
WIDE = [(v, s, pay) for v in (core.FP16_APPROX, core.BF16_APPROX) for s in (W.EULER, W.MILSTEIN)
        for pay in (W.EURO, W.DIGITAL, W.ASIAN, W.LOOKBACK)]


@pytest.mark.parametrize("variant,scheme,payoff", WIDE)
def test_packed_half_pairs(m, variant, scheme, payoff):
    p = W.params(scheme=scheme, payoff=payoff, sigma=0.3)
    level, first, N = 3, 7, 400_003                    # > 6 x 128 x 152 packs: not lane-split
    method = 3 if payoff % 2 else 1
    P = m.make_params(p, d=10, method=method, request=3, rng_pack=1)
    gs, gd = m.mlmc_level_dump(level, N, P, variant, 21, first)
    os_, od = core.level(p, level, first, N, variant, 21, request=3, d=10, method=method, dump=True, pack=1)
    assert gs["isum"] == os_["isum"] and gs["isum2"] == os_["isum2"]
    compare_samples(variant, p, gd, od)


# Packed fixed point with a narrow S format (|S| < 128 while S0 = 100): packs
# whose S leaves the range run again on the clamped datapath, and their
# saturations are counted; sigma = 0.6 lets sum1 fall below -1 on level 0,
# where every pack runs clamped from the start.
@pytest.mark.parametrize("sigma", [0.25, 0.6])
@pytest.mark.parametrize("scheme", [W.EULER, W.MILSTEIN])
@pytest.mark.parametrize("level,N", [(0, 20_011), (1, 20_011), (3, 400_003)])
def test_packed_fixed_saturating(m, sigma, scheme, level, N):
    p = W.params(sigma=sigma, scheme=scheme)
    fmts = [W.default_format(p, lev) for lev in range(level + 1)]
    fmts[level]["e"][6] = 7
    fmts[level]["e"][5] = 7 + fmts[level]["e"][4]
    P = m.make_params(p, d=10, method=1, formats=fmts, rng_pack=1)
    first = 5
    gs, gd = m.mlmc_level_dump(level, N, P, m.FIXED_APPROX, 33, first)
    os_, od = core.level(p, level, first, N, core.FIXED_APPROX, 33, d=10, method=1, fmt=fmts[level], dump=True,
                         pack=1)
    assert os_["saturations"] > 0
    assert gs["isum"] == os_["isum"] and gs["isum2"] == os_["isum2"]
    assert gs["saturations"] == os_["saturations"]
    compare_samples(core.FIXED_APPROX, p, gd, od)
    # the same samples without per-sample records: the lazy path (groups redone
    # clamped when S leaves its range) gives the same integer sums and counts
    ls = m.mlmc_level(level, N, P, m.FIXED_APPROX, 33, first)
    assert ls["isum"] == os_["isum"] and ls["isum2"] == os_["isum2"]
    assert ls["saturations"] == os_["saturations"]
