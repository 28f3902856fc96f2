"""Pins of the oracle's binary16 / bfloat16 rounding (round to nearest, ties to even)."""
import numpy as np
import pytest

from oracle import core


def _random_doubles(rng, n, lo, hi):
    mant = rng.uniform(1.0, 2.0, n)
    ex = rng.integers(lo, hi, n)
    sign = rng.choice([-1.0, 1.0], n)
    return sign * np.ldexp(mant, ex)


def test_fp16_rounding_matches_numpy():
    rng = np.random.default_rng(3)
    x = _random_doubles(rng, 100_000, -30, 17)
    # exact ties at several binades, including the subnormal range
    k = rng.integers(0, 2048, 5000)
    e = rng.integers(-24, 5, 5000)
    ties = np.ldexp(k + 0.5, e)
    x = np.concatenate([x, ties, -ties, [0.0, 65504.0, 65519.99, 65520.0, 1e6, 2**-25, 2**-26, 3 * 2**-26]])
    ours = core.round_fp16(x)
    ref = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(ours, ref)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = _random_doubles(rng, 100_000, -130, 120).astype(np.float32).astype(np.float64)
    k = rng.integers(0, 256, 5000)
    e = rng.integers(-120, 100, 5000)
    ties = np.ldexp(k + 0.5, e).astype(np.float32).astype(np.float64)
    x = np.concatenate([x, ties, -ties, [0.0, 1.0, 3.0e38]])
    ours = core.round_bf16(x)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)
