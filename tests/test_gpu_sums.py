"""Real-valued estimator sums (the level estimator of Sec. 2.1 and the nested
sums of Sec. 2.2, eq. var_nested).

The product level kernels (the ones plans, mlmc_level and mlmc_run launch)
write sums of Y and Y^2.  For the estimators whose samples are real numbers
(FP32 / FP64 exact paths and the nested corrections) these sums must equal
the FP64 sums of the very same samples' values within 1e-12 of sum |Y| (and
of sum Y^2), whatever the chunking: many small CTAs with a ragged tail, the
default shape, and sample counts spanning several CTAs.  The per-sample values
are read through the record-writing kernel (mlmc_level_dump) and are checked
against the oracle sample by sample in test_gpu_parity.py; this file checks
only that the reduction neither loses nor distorts any sample.  With a bound
of 1e-12 sum |Y|, leaving out the partial sums of any CTA that holds a sample
with |Y| above that bound fails the test.
"""
import math

import numpy as np
import pytest

from oracle import core
from paper_2502_07123_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module")
def m():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2502_07123_gb300 import mlmc
    return mlmc


def check_sums(res, y, disc):
    """res: discounted sums of one item; y: the item's per-sample values (undiscounted)."""
    y = np.asarray(y, dtype=np.float64)
    ref1 = disc * math.fsum(y.tolist())
    ref2 = disc * disc * math.fsum((y * y).tolist())
    tol1 = REL * disc * float(np.sum(np.abs(y))) + 1e-300
    tol2 = REL * disc * disc * float(np.sum(y * y)) + 1e-300
    assert abs(res["sum"] - ref1) <= tol1, (res["sum"], ref1, tol1)
    assert abs(res["sum2"] - ref2) <= tol2, (res["sum2"], ref2, tol2)


REAL = [core.FP32_EXACT, core.FP64_EXACT, core.CORR_FIXED, core.CORR_FP16, core.CORR_BF16, core.CORR_FP16S,
        core.CORR_BF16S]
CASES = [(v, pay, lev) for v in REAL for pay in (W.EURO, W.DIGITAL, W.ASIAN, W.LOOKBACK) for lev in (0, 1, 3, 6)]


@pytest.mark.parametrize("variant,payoff,level", CASES)
def test_product_kernel_sums_equal_sample_sums(m, variant, payoff, level):
    p = W.params(payoff=payoff, sigma=0.3)
    fmts = [W.default_format(p, lev) for lev in range(level + 1)]
    method = 3 if (level + payoff) % 2 else 1
    P = m.make_params(p, d=10, method=method, formats=fmts, request=2)
    disc = math.exp(-p["r"] * p["T"])
    N = 4097 if level < 6 else 1023
    first, seed = 5, 31 + level
    _, dump = m.mlmc_level_dump(level, N, P, variant, seed, first)
    y = dump["y"]
    assert np.all(np.isfinite(y))
    item = [dict(params=P, level=level, variant=variant, first_sample=first, N=N)]
    for tuning in (dict(threads=32, steps_per_thread=1), dict(threads=96, steps_per_thread=64), None):
        res = m.mlmc_run(item, seed, tuning=tuning)[0]
        assert res["n"] == N
        check_sums(res, y, disc)
    # mlmc_level: the library's default chunking
    check_sums(m.mlmc_level(level, N, P, variant, seed, first), y, disc)


def test_sums_span_many_ctas(m):
    """A correction item of 2^20 samples on level 2 (thousands of CTAs)."""
    p = W.params()
    fmts = [W.default_format(p, lev) for lev in range(3)]
    P = m.make_params(p, d=10, method=1, formats=fmts)
    N = (1 << 20) + 3
    disc = math.exp(-p["r"] * p["T"])
    _, dump = m.mlmc_level_dump(2, N, P, core.CORR_FIXED, 4, 0)
    res = m.mlmc_run([dict(params=P, level=2, variant=core.CORR_FIXED, N=N)], 4)[0]
    check_sums(res, dump["y"], disc)
