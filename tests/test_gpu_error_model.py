"""GPU error-model statistics (mlmc_sensitivities) against the oracle's
reverse-mode sensitivities on the same samples, and the model check of
Sec. 4.4 on the GPU: the simulated variance of the fixed-point corrections
with the optimised widths respects the pessimistic bound and is of the
order of the optimistic one; S gains about one bit per level (Sec. 6.3)."""
import math

import numpy as np
import pytest

from oracle import core, optimiser as O, tables
from paper_2502_07123_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MSE = [0.0, 0.0] + [float(tables.moments_m1(d)[1]) for d in range(2, 17)]


@pytest.fixture(scope="module")
def m():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2502_07123_gb300 import mlmc
    return mlmc


@pytest.mark.parametrize("lev,N,first", [(0, 5000, 0), (1, 4000, 17), (3, 3000, 0), (6, 700, 1000), (10, 40, 3)])
def test_sensitivities_match_oracle(m, lev, N, first):
    p = W.params()
    P = m.make_params(p, request=2)
    g = m.mlmc_sensitivities(lev, N, P, 31, first_sample=first, per_instance=True)
    r = core.sensitivities(p, lev, first, N, 31, request=2, per_instance=True)
    np.testing.assert_allclose(g["A"], r["A"] / N, rtol=1e-10, atol=1e-300)
    np.testing.assert_allclose(g["inst"], r["inst"] / N, rtol=1e-10, atol=1e-14 * np.max(r["inst"] / N))
    B = np.sqrt(r["inst"] / N).sum(axis=1)
    np.testing.assert_allclose(g["B"], B, rtol=1e-9)
    np.testing.assert_allclose(g["maxabs"], r["maxabs"], rtol=1e-13)
    mean = r["sum_dp"] / N
    var = r["sum_dp2"] / N - mean * mean
    assert g["mean"] == pytest.approx(mean, rel=1e-10, abs=1e-12)
    assert g["var"] == pytest.approx(var, rel=1e-9)
    assert g["n"] == N and g["n_instances"] == core.sens_instances(lev)


def test_sensitivities_reject_unsupported(m):
    for over in (dict(payoff=W.DIGITAL), dict(scheme=W.MILSTEIN)):
        with pytest.raises(m.MLMCError):
            m.mlmc_sensitivities(2, 100, m.make_params(W.params(**over)), 1)
    with pytest.raises(m.MLMCError):
        m.mlmc_sensitivities(11, 100, m.make_params(W.params()), 1)


def test_optimised_widths_bound_the_gpu_corrections(m):
    """10^6 paths per level (the paper's count): optimise, then run the GPU
    fixed-point correction estimator with the optimised widths and table size."""
    p = W.params()
    slope_d = {}
    for lev in (2, 4, 6):
        P = m.make_params(p)
        s = m.mlmc_sensitivities(lev, 1_000_000, P, 77)
        o = m.mlmc_optimise_level(lev, s, lut_mse=MSE)
        slope_d[lev] = o["d_real"][6]
        lut = o["lut_bits"]
        assert 4 <= lut <= 14
        fmts = [W.default_format(p, k) for k in range(lev)] + [o["format"]]
        Pq = m.make_params(p, d=lut, method=1, formats=fmts)
        N = 400_000
        res = m.mlmc_level(lev, N, Pq, W.CORR_FIXED, 5)
        mean = res["sum"] / N
        var = res["sum2"] / N - mean * mean
        v_corr_ext = (math.sqrt(o["v_corr"]) + s["B"][0] * math.sqrt(MSE[lut])) ** 2
        v_indep_ext = o["v_indep"] + s["A"][0] * MSE[lut]
        assert res["saturations"] <= N // 1000
        assert var <= v_corr_ext, (lev, var, v_corr_ext)
        assert 0.1 * v_indep_ext <= var <= 10.0 * v_indep_ext, (lev, var, v_indep_ext)
    slope = (slope_d[6] - slope_d[2]) / 4.0
    assert 0.6 <= slope <= 1.4


def test_table_mse_matches_oracle(m):
    for d in (4, 8, 10, 12, 14):
        assert m.icdf_mse(d) == pytest.approx(MSE[d], rel=1e-9)
