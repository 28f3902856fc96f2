"""Pins of the oracle's exact inverse Normal CDF (Sec. 3: Z = Phi^{-1}(U), U = 2^-D (J + 1/2),
D = 32) against scipy.special.ndtri."""
import numpy as np
from scipy.special import ndtri

from oracle import core

EDGE = np.array([0, 1, 2, 3, 255, 2**24 - 1, 2**24, 2**31 - 2, 2**31 - 1, 2**31, 2**31 + 1,
                 2**32 - 2**24, 2**32 - 2, 2**32 - 1], dtype=np.uint64).astype(np.uint32)


def test_exact_normal_matches_ndtri():
    rng = np.random.default_rng(2025)
    J = np.concatenate([EDGE, rng.integers(0, 2**32, 100_000, dtype=np.uint64).astype(np.uint32)])
    z = core.exact_normal(J)
    u = (J.astype(np.float64) + 0.5) * 2.0**-32
    ref = ndtri(u)
    err = np.abs(z - ref)
    assert np.all(err <= 2e-14 * np.abs(ref) + 1e-300), float(np.max(err / np.abs(ref)))


def test_exact_normal_symmetry_and_monotonicity():
    rng = np.random.default_rng(7)
    J = np.sort(rng.integers(0, 2**32, 50_000, dtype=np.uint64)).astype(np.uint32)
    z = core.exact_normal(J)
    zm = core.exact_normal(~J)
    assert np.array_equal(z, -zm)
    assert np.all(np.diff(z) >= 0)
    assert core.exact_normal(np.array([2**31 - 1], np.uint32))[0] < 0 < core.exact_normal(np.array([2**31], np.uint32))[0]
