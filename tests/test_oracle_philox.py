"""Pins of the oracle's Philox4x32-10 and counter layout.

The oracle's generator is checked against cuRAND's host-side
PHILOX4_32_10 generator (a library implementation of the same published
algorithm), whose output word 4q + k is word k of Philox4x32-10 applied to
the counter (0, 0, q, 0) under the key (seed_lo, seed_hi).
"""
import ctypes

import numpy as np
import pytest

from oracle import core

MASK = 0xFFFFFFFF
CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def _curand_words(seed, n, offset=0):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        buf = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)),
                                  ctypes.c_size_t(n)) == 0
        return buf
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1234, 0x123456789ABCDEF0, 2**64 - 1, 20250211])
def test_philox_matches_curand_host(seed):
    n = 4 * 4096
    ref = _curand_words(seed, n)
    ctr = np.zeros((n // 4, 4), dtype=np.uint32)
    ctr[:, 2] = np.arange(n // 4, dtype=np.uint32)
    out = core.philox(ctr, [seed & MASK, seed >> 32])
    assert np.array_equal(out.reshape(-1), ref)


def test_philox_matches_curand_host_with_offset():
    seed = 987654321
    q0 = 1000
    ref = _curand_words(seed, 64, offset=4 * q0)
    ctr = np.zeros((16, 4), dtype=np.uint32)
    ctr[:, 2] = q0 + np.arange(16, dtype=np.uint32)
    out = core.philox(ctr, [seed & MASK, seed >> 32])
    assert np.array_equal(out.reshape(-1), ref)


def test_draw_counter_layout():
    """J for (sample s, step i) is word (w mod 4) of the call q = w div 4, w = s 2^l + i,
    with counter (q_lo, q_hi, level | stream << 8, request)."""
    rng = np.random.default_rng(1)
    seed, request = 0xDEADBEEFCAFEF00D, 77
    for level in (0, 1, 2, 5, 10):
        for stream in (0, 1):
            s = rng.integers(0, 2**40, 200, dtype=np.uint64)
            i = rng.integers(0, 2**level, 200, dtype=np.uint64)
            J = core.draws(seed, request, level, stream, s, i.astype(np.uint32))
            w = (s << np.uint64(level)) + i
            q = w >> np.uint64(2)
            ctr = np.stack([(q & np.uint64(MASK)).astype(np.uint32), (q >> np.uint64(32)).astype(np.uint32),
                            np.full(200, level | (stream << 8), np.uint32),
                            np.full(200, request, np.uint32)], axis=1)
            words = core.philox(ctr, [seed & MASK, seed >> 32])
            ref = words[np.arange(200), (w & np.uint64(3)).astype(np.int64)]
            assert np.array_equal(J, ref)


def test_top_bits_uniform():
    """The table index uses the top d bits of J: they must be uniform (chi-square)."""
    from scipy.stats import chisquare
    n = 1 << 18
    s = np.arange(n, dtype=np.uint64)
    J = core.draws(5, 0, 3, 0, s // 8, (s % 8).astype(np.uint32))
    counts = np.bincount(J >> 22, minlength=1024)
    assert chisquare(counts).pvalue > 1e-6
