"""Every fixed-point datapath of the CUDA library (fast 32-bit S, fast 64-bit S,
general saturating) against the oracle's exact-integer emulation, bit for bit,
including formats that make S saturate."""
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


def _formats(p, kind, level, rng):
    fm = [W.default_format(p, lev) for lev in range(level + 1)]
    f = fm[level]
    if kind == "saturating_S":
        f["e"][6] = 7                      # |S| < 128 while S0 = 100: frequent saturation
        f["e"][5] = 7 + f["e"][4]
    elif kind == "general":
        f["f"][1], f["f"][3] = f["f"][3] - 1, f["f"][3]   # f_con1 < f_mul1: no fast datapath
    elif kind == "wide_S":
        f["f"][6] = 24                     # e_S + f_S > 30: 64-bit S
    elif kind == "random":
        f["f"] = [int(x) for x in rng.integers(8, 20, 7)]
    return fm


@pytest.mark.parametrize("kind", ["default", "saturating_S", "general", "wide_S", "random"])
@pytest.mark.parametrize("variant", [core.FIXED_APPROX, core.CORR_FIXED])
@pytest.mark.parametrize("scheme", [W.EULER, W.MILSTEIN])
@pytest.mark.parametrize("payoff", [W.EURO, W.ASIAN, W.LOOKBACK, W.DIGITAL])
@pytest.mark.parametrize("level", [0, 3, 6])
def test_fixed_datapaths(m, kind, variant, scheme, payoff, level):
    rng = np.random.default_rng(level * 100 + payoff * 10 + scheme)
    p = W.params(payoff=payoff, scheme=scheme, sigma=0.25)
    fm = _formats(p, kind, level, rng)
    P = m.make_params(p, d=10, method=1, formats=fm)
    N, first, seed = 257, 3, 4242
    try:
        os_, od = core.level(p, level, first, N, variant, seed, fmt=fm[level], dump=True)
    except core.OracleError:
        pytest.skip("format rejected by the oracle")
    try:
        gs, gd = m.mlmc_level_dump(level, N, P, variant, seed, first)
    except m.MLMCError as e:
        assert e.status in (m.EINVAL, m.EOVERFLOW) and kind == "random"
        return
    compare_samples(variant, p, gd, od)
    if variant == core.FIXED_APPROX:
        assert gs["isum"] == os_["isum"] and gs["isum2"] == os_["isum2"]
        assert gs["saturations"] == os_["saturations"]
        # without per-sample records (the lazy 32-bit datapath where it applies)
        ls = m.mlmc_level(level, N, P, variant, seed, first)
        assert ls["isum"] == os_["isum"] and ls["isum2"] == os_["isum2"]
        assert ls["saturations"] == os_["saturations"]
    if kind == "saturating_S":
        assert os_["saturations"] > 0
