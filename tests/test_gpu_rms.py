"""Accuracy of the adaptive estimators over seeds (the Giles 2008 target MSE
eps^2): for the European call of the test case, the root-mean-square error
of mlmc_estimate against Black-Scholes over 100 seeds stays within eps (up
to the sampling error of 100 seeds), for plain FP32 MLMC and the nested
estimators."""
import math

import numpy as np
import pytest

from paper_2502_07123_gb300 import workloads as W
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


@pytest.mark.parametrize("mode", [1, 2, 5, 6])
def test_rms_error_over_seeds(m, mode):
    p = W.params()
    P = m.make_params(p, d=10, method=1, formats=[W.default_format(p, k) for k in range(11)], rng_pack=1)
    ref = black_scholes_call(p["S0"], p["K"], p["r"], p["sigma"], p["T"])
    eps = 0.02
    err = np.array([m.mlmc_estimate(eps, P, mode, s, 10)["price"] - ref for s in range(1, 101)])
    rms = math.sqrt(float(np.mean(err * err)))
    assert rms <= 1.3 * eps, (mode, rms / eps)
    assert abs(float(np.mean(err))) <= 0.8 * eps     # bias within the target
