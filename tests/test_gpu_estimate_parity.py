"""mlmc_estimate against the oracle's pricer on the GPU's own schedule (the
on-line phase of Sec. 6, with the sample allocation of Sec. 2.1 / 2.2).

The adaptive loop's sample counts depend on the sums it sees, so the oracle
cannot repeat the loop on its own; instead it prices exactly the schedule the
GPU returns (every term's samples [0, N_l), the GPU having taken them in
several pieces), with the same packed draws and, in mode 5, the enumerated
approximate terms of levels 0 and 1.  Integer terms are then identical; the
real-valued terms differ only by the per-sample FP32 path bound, so the price
must agree within the mean of those bounds and the variance within the bound
they imply for sum Y^2, plus FP64 rounding."""
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


@pytest.mark.parametrize("mode,payoff,seed", [(driver.PLAIN_FP32, W.EURO, 3), (driver.NESTED_FIXED, W.EURO, 4),
                                              (driver.NESTED_FIXED_EXACT_LOW, W.EURO, 5),
                                              (driver.NESTED_FIXED, W.ASIAN, 6),
                                              (driver.NESTED_FP16S_EXACT_LOW, W.EURO, 7),
                                              (driver.NESTED_BF16S, W.DIGITAL, 8)])
def test_estimate_equals_oracle_on_the_same_schedule(m, mode, payoff, seed):
    eps = 0.05
    p = W.params(payoff=payoff)
    fmts = [W.default_format(p, lev) for lev in range(11)]
    P = m.make_params(p, d=10, method=1, formats=fmts, rng_pack=1)
    r = m.mlmc_estimate(eps, P, mode, seed, 10)
    o = driver.price_on_schedule(p, seed, mode, r["N"], fmt_of_level=lambda lev: fmts[lev], pack=1, dump=True)
    tol_p, tol_v, terms = schedule_bounds(mode, p, o["dumps"], r["N"])
    var_gpu = r["stderr"] ** 2
    assert abs(r["price"] - o["price"]) <= tol_p + 1e-12 * terms * (abs(o["price"]) + 1.0), \
        (r["price"], o["price"], tol_p)
    assert abs(var_gpu - o["var"]) <= tol_v + 1e-10 * o["var"], (var_gpu, o["var"], tol_v)
    # the schedule met its own variance target: sum V/N <= eps^2 / 2
    assert var_gpu <= 0.5 * eps * eps * (1 + 1e-9)
