"""The library's bit-width optimiser (host code behind the C ABI, no GPU
needed) against the oracle's, on the oracle's error-model statistics: the
same real widths, multiplier, integer widths, model variances, costs and
table size."""
import math

import numpy as np
import pytest

from oracle import core, optimiser as O, tables
from paper_2502_07123_gb300 import workloads as W

MSE = [0.0, 0.0] + [float(tables.moments_m1(d)[1]) for d in range(2, 17)]


@pytest.fixture(scope="module")
def m():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2502_07123_gb300 import mlmc
    return mlmc


def test_struct_layouts(m):
    import ctypes
    assert ctypes.sizeof(m.Sensitivity) == 200
    assert ctypes.sizeof(m.OptConfig) == 136
    assert ctypes.sizeof(m.OptResult) == 200


@pytest.mark.parametrize("lev", [0, 1, 3, 5])
def test_optimiser_matches_oracle(m, lev):
    p = W.params()
    N = 3000 if lev < 4 else 800
    r = core.sensitivities(p, lev, 0, N, 5, per_instance=True)
    A = list(r["A"] / N)
    B = list(np.sqrt(r["inst"] / N).sum(axis=1))
    V = r["sum_dp2"] / N - (r["sum_dp"] / N) ** 2
    ref = O.optimise_level(lev, A, B, list(r["maxabs"]), V, mse_of_lut=lambda d: MSE[d])
    got = m.mlmc_optimise_level(lev, dict(A=A, B=B, maxabs=list(r["maxabs"]), var=V), lut_mse=MSE)
    assert got["e"] == ref["e"]
    np.testing.assert_allclose(got["d_real"], ref["d_real"], rtol=0, atol=1e-6)
    assert got["d"] == ref["d"]
    assert got["lambda"] == pytest.approx(ref["lambda"], rel=1e-5)
    for k in ("v_indep", "v_corr", "cost_lp", "cost_exact", "level_cost_ratio"):
        assert got[k] == pytest.approx(ref[k], rel=1e-9), k
    assert got["lut_bits"] == ref["lut_bits"]
    assert got["format"]["e"] == ref["e"]
    assert got["format"]["f"] == [max(0, d - e) for d, e in zip(ref["d"], ref["e"])]


def test_optimiser_custom_cost_and_errors(m):
    """Operand counts and c_rng are inputs; invalid statistics are rejected."""
    A = [1.0, 2e5, 300.0, 5e4, 5e4, 3.0, 3.0]
    B = [10.0] * 7
    mx = [4.0, 0.02, 0.1, 0.4, 0.4, 40.0, 200.0]
    mul = [2.0, 0.0, 2.0, 0.0, 2.0, 0.0, 2.0]
    add = [0.0, 1.0, 0.0, 1.0, 0.0, 1.0, 1.0]
    ref = O.optimise_level(2, A, B, mx, 1.5, c_rng=3e3, M=mul, Mp=add)
    got = m.mlmc_optimise_level(2, dict(A=A, B=B, maxabs=mx, var=1.5), c_rng=3e3, mul=mul, add=add)
    assert got["d"] == ref["d"]
    np.testing.assert_allclose(got["d_real"], ref["d_real"], atol=1e-6)
    with pytest.raises(m.MLMCError):
        m.mlmc_optimise_level(2, dict(A=A, B=B, maxabs=mx, var=0.0))
    with pytest.raises(m.MLMCError):
        m.mlmc_optimise_level(2, dict(A=[-1.0] + A[1:], B=B, maxabs=mx, var=1.0))
