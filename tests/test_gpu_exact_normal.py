"""The FP32 exact Normal the level kernels compute (mlmc_exact_normal_f32):
within its error bound of Phi^{-1} in FP64 (scipy.special.ndtri) over words J
across the whole range, odd under J -> ~J, equal to the host emulation of the
same FP32 steps, and the same Normal the FP32 exact path uses (a level-0
path from it equals the kernel's dump)."""
import numpy as np
import pytest

from oracle import core
from paper_2502_07123_gb300 import workloads as W
from tests import test_phi_inv_table as host

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


def _run(m, J):
    import torch
    Jd = torch.from_numpy(J.astype(np.uint32).view(np.int32)).cuda()
    z = torch.empty(len(J), dtype=torch.float32, device="cuda")
    m.exact_normal_f32(Jd, z)
    return z.cpu().numpy().astype(np.float64)


def test_exact_normal_error_bound_and_symmetry(m):
    ndtri = pytest.importorskip("scipy.special").ndtri
    J = host._words()
    z = _run(m, J)
    Jp = np.where(J >= 2 ** 31, (2 ** 32 - 1) - J, J)
    ref = ndtri((Jp.astype(np.float64) + 0.5) * 2.0 ** -32) * np.where(J >= 2 ** 31, -1.0, 1.0)
    err = np.abs(z - ref)
    assert np.all(err <= 1.5e-7 + 2e-7 * np.abs(ref)), float(np.max(err - 2e-7 * np.abs(ref)))
    zneg = _run(m, (2 ** 32 - 1) - J)
    np.testing.assert_array_equal(zneg, -z)
    # the device steps are the host emulation's (fused multiply-adds aside, which
    # the emulation rounds twice): equal to within one unit in the last place
    ze, _ = host._emulate(J, host._header_table())
    assert np.all(np.abs(z - ze) <= np.spacing(np.abs(ze).astype(np.float32)).astype(np.float64) + 1e-45)


def test_exact_path_uses_the_same_normal(m):
    # level 0, FP32 exact: S_1 = S0 + S0 (c1 + c2 Z) with Z the word's Normal
    p = W.params(payoff=W.EURO)
    P = m.make_params(p, d=10, method=1, formats=[W.default_format(p, lev) for lev in range(11)], request=3)
    _, rec = m.mlmc_level_dump(0, 4096, P, W.FP32_EXACT, 7)
    # the word J of sample s's one fine step (the oracle's Philox, stream 0)
    words = core.draws(7, 3, 0, 0, np.arange(4096), np.zeros(4096))
    z = _run(m, words.astype(np.uint64)).astype(np.float32)
    c1 = np.float32(p["r"] * p["T"])
    c2 = np.float32(p["sigma"] * np.sqrt(p["T"]))
    S0 = np.float32(p["S0"])
    inc = host._fma32(np.full_like(z, c2), z, np.full_like(z, c1))
    S1 = host._fma32(np.full_like(z, S0), inc, np.full_like(z, S0))
    np.testing.assert_allclose(rec["sf"], S1.astype(np.float64), rtol=2.5e-7)
