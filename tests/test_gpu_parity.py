"""Parity of the CUDA path (through the C ABI) with the CPU oracle on identical samples."""
import math

import numpy as np
import pytest

from oracle import core, tables
from paper_2502_07123_gb300 import workloads as W
from tests.gpu_helpers import APPROX_ONLY, CORR, compare_samples

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


def test_philox_words_bit_exact(m):
    rng = np.random.default_rng(0)
    for seed in (0, 1, 2**64 - 1, 0x0123456789ABCDEF):
        ctr = rng.integers(0, 2**32, (4096, 4), dtype=np.uint64).astype(np.uint32)
        ctr[:8] = 0
        ctr[8:16] = 0xFFFFFFFF
        g = m.mlmc_philox(ctr, seed)
        o = core.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        assert np.array_equal(g, o)


@pytest.mark.parametrize("d", [2, 6, 10, 12, 14])
@pytest.mark.parametrize("method", [1, 3])
def test_icdf_tables_bit_exact(m, d, method):
    if method == 3 and d < 3:
        pytest.skip("Method 3 needs d >= 3")
    reps = [("fp32", m.REP_FP32), ("fp16", m.REP_FP16), ("bf16", m.REP_BF16), ("fixed", m.REP_FIXED)]
    for name, rep in reps:
        for fZ in ((12, 20) if name == "fixed" else (0,)):
            g = m.mlmc_icdf_table(method, d, rep, fZ)
            o = tables.table(d, method, name, fZ)
            bad = np.nonzero(g != o)[0]
            assert bad.size == 0, (name, fZ, bad[:4], g[bad[:4]], o[bad[:4]])
    if method == 1:
        # FP64 values: GPU normcdfinv / expm1 against the 40-digit closed form.  The
        # difference of adjacent quantiles loses about d bits, so the bound scales with 2^d.
        g = m.mlmc_icdf_table(1, d, m.REP_FP64)
        o = tables.m1_fp64(d)
        rel = np.abs(g - o) / np.abs(o)
        assert np.max(rel) <= 2.0**d * 1e-15, float(np.max(rel))


VARIANTS = [core.FP64_EXACT, core.FP32_EXACT, core.FP16_APPROX, core.BF16_APPROX, core.FIXED_APPROX,
            core.CORR_FIXED, core.CORR_FP16, core.CORR_BF16, core.FP16S_APPROX, core.BF16S_APPROX,
            core.CORR_FP16S, core.CORR_BF16S]
CASES = [(v, s, pay, lev) for v in VARIANTS for s in (W.EULER, W.MILSTEIN)
         for pay in (W.EURO, W.DIGITAL, W.ASIAN, W.LOOKBACK) for lev in (0, 1, 2, 5)]


@pytest.mark.parametrize("variant,scheme,payoff,level", CASES)
def test_sample_parity(m, variant, scheme, payoff, level):
    p = W.params(scheme=scheme, payoff=payoff, sigma=0.3)
    fmts = [W.default_format(p, lev) for lev in range(level + 1)]
    method = 3 if (level + payoff) % 2 else 1
    seed, first, N = 1000 + level, 13, 301
    P = m.make_params(p, d=10, method=method, formats=fmts, request=3)
    gs, gd = m.mlmc_level_dump(level, N, P, variant, seed, first)
    os_, od = core.level(p, level, first, N, variant, seed, request=3, d=10, method=method,
                         fmt=fmts[level], dump=True)
    compare_samples(variant, p, gd, od)
    if variant in APPROX_ONLY:
        assert gs["isum"] == os_["isum"] and gs["isum2"] == os_["isum2"]
        assert gs["saturations"] == os_["saturations"]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("level", [0, 1, 3, 7])
def test_multichunk_sums(m, variant, level):
    """Many small CTAs and a ragged tail: integer sums equal the oracle's, real sums
    are the FP64 sums of samples that match the oracle's one by one."""
    p = W.params(payoff=W.EURO)
    fmts = [W.default_format(p, lev) for lev in range(level + 1)]
    P = m.make_params(p, d=10, method=1, formats=fmts)
    N = 4097 if level < 5 else 777
    first = 5
    res = m.mlmc_run([dict(params=P, level=level, variant=variant, first_sample=first, N=N)], seed=77,
                     tuning=dict(threads=32, steps_per_thread=1))[0]
    o, od = core.level(p, level, first, N, variant, 77, fmt=fmts[level], dump=True)
    disc = math.exp(-p["r"] * p["T"])
    assert res["n"] == N
    if variant in APPROX_ONLY:
        assert res["isum"] == o["isum"] and res["isum2"] == o["isum2"]
        assert res["sum"] == disc * o["sum"]
    else:
        # real samples: each agrees with the oracle's within the path bound, and
        # the product kernel's sums are the FP64 sums of exactly these samples
        _, gd = m.mlmc_level_dump(level, N, P, variant, 77, first)
        compare_samples(variant, p, gd, od)
        y = gd["y"]
        assert abs(res["sum"] - disc * math.fsum(y.tolist())) <= 1e-12 * disc * np.sum(np.abs(y))
        assert abs(res["sum2"] - disc * disc * math.fsum((y * y).tolist())) <= 1e-12 * disc * disc * np.sum(y * y)


@pytest.mark.parametrize("variant", [core.FP16S_APPROX, core.BF16S_APPROX])
@pytest.mark.parametrize("payoff", [W.EURO, W.ASIAN, W.LOOKBACK])
@pytest.mark.parametrize("level,N", [(0, 4001), (1, 3001), (3, 1001), (6, 301), (4, 200_001)])
def test_fp32_s_packed_draws(m, variant, payoff, level, N):
    """Half increments with FP32 S, three samples per Philox word (and, for deep
    items below one wave, one of them per thread): records and exact integer
    sums equal the oracle's."""
    p = W.params(payoff=payoff, scheme=W.MILSTEIN if level % 2 else W.EULER, sigma=0.25)
    P = m.make_params(p, d=10, method=3 if level == 3 else 1, rng_pack=1)
    method = 3 if level == 3 else 1
    seed, first = 70 + level, 2
    gs, gd = m.mlmc_level_dump(level, N, P, variant, seed, first)
    os_, od = core.level(p, level, first, N, variant, seed, d=10, method=method, dump=True, pack=1)
    compare_samples(variant, p, gd, od)
    run = m.mlmc_level(level, N, P, variant, seed, first)
    assert run["isum"] == os_["isum"] and run["isum2"] == os_["isum2"]
