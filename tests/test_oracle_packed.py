"""Pins of the packed draws of approximate-only estimators: sample s = k P + L
(k = floor(32/d)) reads field L (bits [32-d(L+1), 32-dL)) of the word its pack P
would read at step i.  Checked against the Philox words, for uniformity and
independence of the fields, and for the law of the estimator (same mean and
variance as with one word per draw)."""
import math

import numpy as np
import pytest
from scipy.stats import chisquare

from oracle import core
from paper_2502_07123_gb300 import workloads as W

MASK = 0xFFFFFFFF


@pytest.mark.parametrize("d", [8, 10, 12, 16])
def test_packed_draw_layout(d):
    k = 32 // d
    rng = np.random.default_rng(d)
    seed, request, level, stream = 0xABCDEF0123, 9, 3, 1
    s = rng.integers(0, 2**36, 500, dtype=np.uint64)
    i = rng.integers(0, 2**level, 500, dtype=np.uint64)
    J = core.draws_packed(seed, request, level, stream, s, i.astype(np.uint32), d)
    P, L = s // np.uint64(k), s % np.uint64(k)
    w = (P << np.uint64(level)) + i
    q = w >> np.uint64(2)
    ctr = np.stack([(q & np.uint64(MASK)).astype(np.uint32), (q >> np.uint64(32)).astype(np.uint32),
                    np.full(500, level | (stream << 8), np.uint32), np.full(500, request, np.uint32)], axis=1)
    words = core.philox(ctr, [seed & MASK, seed >> 32])[np.arange(500), (w & np.uint64(3)).astype(np.int64)]
    field = (words.astype(np.uint64) >> (np.uint64(32) - np.uint64(d) * (L + np.uint64(1)))) & np.uint64((1 << d) - 1)
    assert np.array_equal((J >> np.uint32(32 - d)).astype(np.uint64), field)


def test_packed_fields_uniform_and_independent():
    d, level = 10, 2
    n = 3 * (1 << 16)
    s = np.arange(n, dtype=np.uint64)
    J = core.draws_packed(7, 0, level, 1, s, np.zeros(n, np.uint32), d)
    j = (J >> np.uint32(22)).astype(np.int64)
    for lane in range(3):
        assert chisquare(np.bincount(j[lane::3], minlength=1024)).pvalue > 1e-6
    # pairs of lanes from the same word: joint top-5-bit histogram is uniform
    pair = (j[0::3] >> 5) * 32 + (j[1::3] >> 5)
    assert chisquare(np.bincount(pair, minlength=1024)).pvalue > 1e-6


@pytest.mark.parametrize("variant", [core.FIXED_APPROX, core.FP16_APPROX])
def test_packed_estimator_has_the_same_law(variant):
    p = W.params()
    lev, N = 2, 60_000
    fmt = W.default_format(p, lev)
    a, _ = core.level(p, lev, 0, N, variant, 31, fmt=fmt, pack=1)
    b, _ = core.level(p, lev, 0, N, variant, 32, fmt=fmt, pack=0)
    ma, mb = a["sum"] / N, b["sum"] / N
    va, vb = a["sum2"] / N - ma * ma, b["sum2"] / N - mb * mb
    assert abs(ma - mb) < 4 * math.sqrt((va + vb) / N)
    assert abs(va / vb - 1) < 0.05


def test_packing_is_rejected_for_coupled_estimators():
    p = W.params()
    with pytest.raises(core.OracleError):
        core.level(p, 2, 0, 10, core.CORR_FIXED, 1, fmt=W.default_format(p, 2), pack=1)
    with pytest.raises(core.OracleError):
        core.level(p, 2, 0, 10, core.FP32_EXACT, 1, pack=1)
