"""Method 2 on the GPU against the oracle: the optimised small table, the
interval ranks and the iteration count, the table values in every
representation (bit for bit), per-sample parity of approximate and
correction estimators (fixed point and binary16; the correction's exact path
reads the uniform of interval pi(j)), packed draws, and a nested price; two
fields and n = 3, 4, 6, 7 fields."""
import math

import numpy as np
import pytest

from oracle import core, tables as T
from paper_2502_07123_gb300 import workloads as W
from tests.gpu_helpers import compare_samples
from tests.test_oracle_paths import black_scholes_call

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


@pytest.mark.parametrize("d", [4, 6, 8, 10, 12, 14])
def test_small_table_and_ranks(m, d):
    g = m.mlmc_icdf_method2(d)
    r = T.m2_optimise(d)
    assert g["iterations"] == r["iterations"]
    # two least-squares solvers (normal equations vs SVD): agreement to ~1e-14 of the table scale
    np.testing.assert_allclose(g["x"], r["x"], rtol=1e-11, atol=1e-13)
    np.testing.assert_array_equal(g["pi"], r["pi"])


@pytest.mark.parametrize("d", [6, 10, 12])
def test_table_values(m, d):
    for rep, name, fZ in ((4, "fixed", 12), (4, "fixed", 16), (2, "fp16", 0), (3, "bf16", 0), (1, "fp32", 0)):
        g = m.mlmc_icdf_table(2, d, rep, fZ)
        o = T.table(d, 2, name, fZ)
        np.testing.assert_array_equal(g, o, err_msg="%s fZ=%d" % (name, fZ))
    np.testing.assert_allclose(m.mlmc_icdf_table(2, d, 0), T.table(d, 2, "fp64"), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("variant", [core.FIXED_APPROX, core.CORR_FIXED, core.FP16_APPROX, core.CORR_FP16,
                                     core.BF16_APPROX, core.CORR_BF16])
@pytest.mark.parametrize("level", [0, 1, 4])
@pytest.mark.parametrize("d", [8, 10])
def test_samples_match_oracle(m, variant, level, d):
    p = W.params(payoff=W.EURO)
    fm = [W.default_format(p, lev) for lev in range(level + 1)]
    P = m.make_params(p, d=d, method=2, formats=fm)
    N, first, seed = 300, 5, 606
    _, od = core.level(p, level, first, N, variant, seed, d=d, method=2, fmt=fm[level], dump=True)
    _, gd = m.mlmc_level_dump(level, N, P, variant, seed, first)
    compare_samples(variant, p, gd, od)


def test_packed_draws_and_sums(m):
    p = W.params(payoff=W.DIGITAL)
    lev = 3
    fm = [W.default_format(p, k) for k in range(lev + 1)]
    P = m.make_params(p, d=10, method=2, formats=fm, rng_pack=1)
    N = 30_001
    os_, _ = core.level(p, lev, 0, N, core.FIXED_APPROX, 9, d=10, method=2, fmt=fm[lev], pack=1)
    gs = m.mlmc_level(lev, N, P, core.FIXED_APPROX, 9)
    assert gs["isum"] == os_["isum"] and gs["isum2"] == os_["isum2"]


def test_nested_price_with_method2(m):
    p = W.params()
    P = m.make_params(p, d=10, method=2, formats=[W.default_format(p, k) for k in range(11)], rng_pack=1)
    r = m.mlmc_estimate(0.01, P, m.MODE_NESTED_FIXED_EXACT_LOW, 3, 10)
    ref = black_scholes_call(p["S0"], p["K"], p["r"], p["sigma"], p["T"])
    assert abs(r["price"] - ref) < 4 * r["stderr"] + 0.01 / math.sqrt(2)


def test_noalloc_rejects_method2(m):
    P = m.make_params(W.params(), d=10, method=2)
    with pytest.raises(m.MLMCError) as e:
        m.mlmc_level_noalloc(2, 1000, P, core.FIXED_APPROX, 1)
    assert e.value.status == m.EINVAL


# n fields of d/n bits: (d, n) with 2 to 4 bits per field
FIELDS = [(6, 3), (9, 3), (12, 3), (8, 4), (12, 4), (12, 6), (14, 7)]


@pytest.mark.parametrize("d,n", FIELDS)
def test_n_fields_small_table_and_ranks(m, d, n):
    g = m.mlmc_icdf_method2(d, n)
    r = T.m2_optimise(d, n)
    assert g["iterations"] == r["iterations"]
    np.testing.assert_allclose(g["x"], r["x"], rtol=1e-11, atol=1e-13)
    np.testing.assert_array_equal(g["pi"], r["pi"])


@pytest.mark.parametrize("d,n", FIELDS)
def test_n_fields_table_values(m, d, n):
    for rep, name, fZ in ((4, "fixed", 12), (2, "fp16", 0), (3, "bf16", 0), (1, "fp32", 0)):
        g = m.mlmc_icdf_method2_table(d, n, rep, fZ)
        np.testing.assert_array_equal(g, T.table(d, 2, name, fZ, n), err_msg="%s" % name)
    np.testing.assert_allclose(m.mlmc_icdf_method2_table(d, n, 0), T.table(d, 2, "fp64", 0, n), rtol=1e-11,
                               atol=1e-13)


@pytest.mark.parametrize("variant", [core.FIXED_APPROX, core.CORR_FIXED, core.FP16_APPROX, core.CORR_BF16])
@pytest.mark.parametrize("d,n", [(9, 3), (12, 4)])
@pytest.mark.parametrize("level", [0, 3])
def test_n_fields_samples_match_oracle(m, variant, d, n, level):
    p = W.params(payoff=W.EURO)
    fm = [W.default_format(p, lev) for lev in range(level + 1)]
    P = m.make_params(p, d=d, method=2, formats=fm, fields=n)
    N, first, seed = 300, 5, 607
    _, od = core.level(p, level, first, N, variant, seed, d=d, method=2, fmt=fm[level], dump=True, fields=n)
    _, gd = m.mlmc_level_dump(level, N, P, variant, seed, first)
    compare_samples(variant, p, gd, od)


def test_n_fields_rules(m):
    p = W.params()
    for d, n in ((10, 3), (10, 4), (8, 8), (16, 4)):     # n must divide d with >= 2 bits per field, d <= 14
        with pytest.raises(m.MLMCError) as e:
            m.mlmc_level(2, 100, m.make_params(p, d=d, method=2, fields=n), core.FIXED_APPROX, 1)
        assert e.value.status == m.EINVAL
    with pytest.raises(m.MLMCError):
        m.mlmc_level(2, 100, m.make_params(p, d=10, method=1, fields=2), core.FIXED_APPROX, 1)
    # n = 0 is n = 2
    a = m.mlmc_level(3, 5000, m.make_params(p, d=10, method=2, fields=0), core.CORR_FIXED, 4)
    b = m.mlmc_level(3, 5000, m.make_params(p, d=10, method=2, fields=2), core.CORR_FIXED, 4)
    assert a["sum"] == b["sum"] and a["sum2"] == b["sum2"]
