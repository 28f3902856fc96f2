"""Full-size parity of the nested workload in the launch configuration the
benchmark times (one plan over all 36 work items): exact integer sums of every
approximate item equal the oracle's; every sample of each correction item
agrees with the oracle's within the FP32 path bound and the plan's correction
sums are the FP64 sums of those samples; sampled samples of the approximate
items agree one by one."""
import math

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


def test_nested_workload_full_size(m):
    import bench
    items, meta, cfg = bench.build_items(m)
    plan = m.Plan(items, cfg["seed"])
    plan.launch()
    res = plan.results()
    plan.launch()
    res2 = plan.results()
    for a, b in zip(res, res2):         # deterministic across launches
        assert a["sum"] == b["sum"] and a["sum2"] == b["sum2"] and a["isum"] == b["isum"]
    for k, (it, r) in enumerate(zip(meta, res)):
        p = it["params"]
        fmt = W.default_format(p, it["level"])
        assert r["n"] == it["N"]
        if it["variant"] == W.FIXED_APPROX:
            o, _ = core.level(p, it["level"], 0, it["N"], it["variant"], cfg["seed"], request=it["request"],
                              d=cfg["d"], method=cfg["method"], fmt=fmt, pack=cfg["rng_pack"])
            assert r["isum"] == o["isum"] and r["isum2"] == o["isum2"], it
            assert r["saturations"] == o["saturations"]
        else:
            # every sample of the correction item against the oracle, and the
            # plan's sums against the FP64 sums of those samples (1e-12 of sum |Y|)
            _, od = core.level(p, it["level"], 0, it["N"], it["variant"], cfg["seed"], request=it["request"],
                               d=cfg["d"], method=cfg["method"], fmt=fmt, dump=True)
            P = items[k]["params"]
            _, gd = m.mlmc_level_dump(it["level"], it["N"], P, it["variant"], cfg["seed"], 0)
            compare_samples(it["variant"], p, gd, od)
            disc = math.exp(-p["r"] * p["T"])
            y = gd["y"]
            assert abs(r["sum"] - disc * math.fsum(y.tolist())) <= 1e-12 * disc * np.sum(np.abs(y)), it
            assert abs(r["sum2"] - disc * disc * math.fsum((y * y).tolist())) <= 1e-12 * disc * disc * np.sum(y * y)


def test_nested_workload_sampled_samples(m):
    """Per-sample parity on sampled indices of the largest items, at full size."""
    cfg = W.nested_config()
    rng = np.random.default_rng(8)
    for it in cfg["items"]:
        if it["level"] not in (0, 4, 8):
            continue
        p = it["params"]
        fmts = [W.default_format(p, lev) for lev in range(9)]
        P = m.make_params(p, d=cfg["d"], method=cfg["method"], formats=fmts, request=it["request"],
                          rng_pack=cfg["rng_pack"])
        pack = cfg["rng_pack"] if it["variant"] == W.FIXED_APPROX else 0
        _, gd = m.mlmc_level_dump(it["level"], it["N"], P, it["variant"], cfg["seed"], 0)
        idx = np.sort(rng.choice(it["N"], size=64, replace=False))
        for s in idx:
            _, od = core.level(p, it["level"], int(s), 1, it["variant"], cfg["seed"], request=it["request"],
                               d=cfg["d"], method=cfg["method"], fmt=fmts[it["level"]], dump=True, pack=pack)
            compare_samples(it["variant"], p, gd[s:s + 1], od)
