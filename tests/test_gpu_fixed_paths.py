"""Every fixed-point datapath of the CUDA library (fast 32-bit S, fast 64-bit S,
general saturating) against the oracle's exact-integer emulation, bit for bit,
including formats that make S saturate, formats whose sums align onto the
finer term's grid (mul1 finer than con1, mul2 finer than S: the fast datapath
folds the two roundings into one shift) and one the fast datapath must leave
to the general one (sum1 finer than both of its terms)."""
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
        f["f"][4] = max(f["f"][1], f["f"][3]) + 1          # sum1 finer than con1 and mul1: no fast datapath
    elif kind == "mul1_finer":
        f["f"][1], f["f"][3] = f["f"][3] - 1, f["f"][3]   # f_con1 < f_mul1: con1 aligned onto mul1's grid
    elif kind == "mul2_finer":
        f["f"][6] = 6                                      # f_S < f_mul2 (as the optimiser's widths have)
        f["f"][5] = 9
    elif kind == "wide_S":
        f["f"][6] = 24                     # e_S + f_S > 30: 64-bit S
    elif kind == "random":
        f["f"] = [int(x) for x in rng.integers(8, 20, 7)]
    return fm


FAST_FAMILIES = {8, 9, 10, 11, 15, 16, 17, 24}
GENERAL_FAMILIES = {2, 5, 12}


def _family(m, P, level, variant, N, first):
    plan = m.Plan([dict(params=P, level=level, variant=variant, N=N, first_sample=first)], 1)
    return plan.launch_info(0)[0]


@pytest.mark.parametrize("kind", ["default", "saturating_S", "general", "mul1_finer", "mul2_finer", "wide_S",
                                  "random"])
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
    fam = _family(m, P, level, variant, N, first)
    if kind in ("mul1_finer", "mul2_finer"):
        # the alignment costs nothing: the datapath is the one the default format gets
        P0 = m.make_params(p, d=10, method=1, formats=_formats(p, "default", level, rng))
        fam0 = _family(m, P0, level, variant, N, first)
        assert fam == fam0 and fam in FAST_FAMILIES, (fam, fam0)
    elif kind == "general":
        assert fam in GENERAL_FAMILIES, fam
    if variant == core.FIXED_APPROX:
        assert gs["isum"] == os_["isum"] and gs["isum2"] == os_["isum2"]
        assert gs["saturations"] == os_["saturations"]
        # without per-sample records (the lazy 32-bit datapath where it applies)
        ls = m.mlmc_level(level, N, P, variant, seed, first)
        assert ls["isum"] == os_["isum"] and ls["isum2"] == os_["isum2"]
        assert ls["saturations"] == os_["saturations"]
    if kind == "saturating_S":
        assert os_["saturations"] > 0
