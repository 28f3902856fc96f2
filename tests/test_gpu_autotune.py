"""Launch-shape autotuner: it picks shapes from its candidate set, installs
them for calls without an explicit shape, leaves integer sums unchanged (FP64
sums of real samples change at most in rounding), and mlmc_tuning_reset restores the
default chunking bit for bit."""
import pytest

from paper_2502_07123_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2502_07123_gb300 import mlmc
    yield mlmc
    mlmc.mlmc_tuning_reset()


def _items(m):
    p = W.params()
    pp = m.make_params(p, d=10, method=1, rng_pack=1)
    items = [dict(params=pp, level=lev, variant=W.FIXED_APPROX, N=300_000) for lev in (0, 1, 3, 6, 9)]
    items += [dict(params=pp, level=lev, variant=W.CORR_FIXED, N=30_000) for lev in (0, 3, 6)]
    items += [dict(params=pp, level=4, variant=W.FP32_EXACT, N=50_000)]
    return items


def test_autotune_shapes_and_sums(m):
    m.mlmc_tuning_reset()
    items = _items(m)
    before = m.mlmc_run(items, 9)
    shapes = m.mlmc_autotune(items, 9, reps=3)
    assert len(shapes) == len(items)
    for t, sp in shapes:
        assert t in (64, 96, 128) and sp in (64, 128, 256, 512, 1024, 2048)
    after = m.mlmc_run(items, 9)
    for it, b, a in zip(items, before, after):
        assert a["n"] == b["n"]
        if it["variant"] == W.FIXED_APPROX:
            assert a["isum"] == b["isum"] and a["isum2"] == b["isum2"]
        else:
            # FP64 sums of the same samples: another chunking reorders the additions
            # only (sum |Y| <= sqrt(n sum Y^2))
            assert abs(a["sum"] - b["sum"]) <= 2e-12 * (b["n"] * b["sum2"]) ** 0.5
            assert abs(a["sum2"] - b["sum2"]) <= 2e-12 * b["sum2"]
    m.mlmc_tuning_reset()
    again = m.mlmc_run(items, 9)
    for b, c in zip(before, again):
        assert c["sum"] == b["sum"] and c["sum2"] == b["sum2"]


def test_autotuned_engine_still_equals_estimate(m):
    """Engine admissions and mlmc_estimate read the same shape table."""
    m.mlmc_tuning_reset()
    m.mlmc_autotune(_items(m), 9, reps=2)
    p = W.params(payoff=W.DIGITAL)
    P = m.make_params(p, d=10, method=1, rng_pack=1, request=4,
                      formats=[W.default_format(p, lev) for lev in range(11)])
    ref = m.mlmc_estimate(0.01, P, 5, 77, 10)
    out = m.mlmc_batch_estimate([P], [0.01], 5, 77, max_level=10)
    m.mlmc_tuning_reset()
    assert out["price"][0] == ref["price"] and out["stderr"][0] == ref["stderr"] and out["L"][0] == ref["L"]
