"""mlmc_level_noalloc: the single-level estimator for callers that must not
allocate device memory while they run (their device memory belongs to another
allocator, or a cudaMalloc would stall a latency-critical loop).  Its scratch
lives in a fixed device array inside the library, so it can only handle up to
16384 CTAs per call.  This file is collected last on purpose: it checks the
entry point through the C ABI against mlmc_level, twice in a row (the array
keeps the previous call's contents), in a fresh process or after every other
test."""
import ctypes

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
    return mlmc


CASES = [
    # (variant, level, N, first, payoff, scheme, method)
    (W.FIXED_APPROX, 0, 200_000, 3, W.EURO, W.EULER, 1),
    (W.FIXED_APPROX, 6, 5_000, 0, W.DIGITAL, W.MILSTEIN, 3),
    (W.FP32_EXACT, 3, 20_000, 11, W.ASIAN, W.MILSTEIN, 1),
    (W.CORR_FIXED, 5, 3_000, 0, W.EURO, W.EULER, 1),
    (W.FP16_APPROX, 2, 50_000, 7, W.LOOKBACK, W.EULER, 3),
    (W.FP64_EXACT, 1, 4_000, 0, W.DIGITAL, W.EULER, 1),
    (W.CORR_BF16, 4, 2_000, 1, W.ASIAN, W.EULER, 1),
]


def _call_c_abi(m, level, N, P, variant, seed, first):
    """Call the entry point directly through the C ABI (ctypes), legacy default stream."""
    lib = ctypes.CDLL(m.LIB_PATH)
    fn = lib.mlmc_level_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(m.Params), ctypes.c_int, ctypes.c_uint64,
                   ctypes.c_uint64, ctypes.POINTER(m.Sums), ctypes.c_void_p]
    s = m.Sums()
    st = fn(level, N, ctypes.byref(P), variant, seed, first, ctypes.byref(s), None)
    assert st == 0, m.mlmc_strerror(st)
    d = {k: getattr(s, k) for k, _ in m.Sums._fields_}
    d["isum2"] = (int(s.isum2_hi) << 64) | int(s.isum2_lo)
    return d


@pytest.mark.parametrize("variant,level,N,first,payoff,scheme,method", CASES)
def test_noalloc_matches_mlmc_level(m, variant, level, N, first, payoff, scheme, method):
    p = W.params(payoff=payoff, scheme=scheme)
    P = m.make_params(p, d=10, method=method, formats=[W.default_format(p, lev) for lev in range(level + 1)])
    ref = m.mlmc_level(level, N, P, variant, 99, first)
    for _ in range(2):  # the second call reuses the array the first one left behind
        got = _call_c_abi(m, level, N, P, variant, 99, first)
        assert got["n"] == ref["n"] and got["saturations"] == ref["saturations"]
        assert got["exact_int"] == ref["exact_int"] and got["unit"] == ref["unit"]
        if ref["exact_int"]:
            assert got["isum"] == ref["isum"] and got["isum2"] == ref["isum2"]
            assert got["sum"] == ref["sum"]
        else:
            # same kernels and chunking as mlmc_level; the real-valued sums use the
            # FP32 per-path bound of the parity tests as their tolerance
            assert abs(got["sum"] - ref["sum"]) <= 1e-5 * (abs(ref["sum"]) + N * 1e-3)
            assert abs(got["sum2"] - ref["sum2"]) <= 1e-5 * abs(ref["sum2"]) + 1e-12


def test_noalloc_rejects_sizes_beyond_its_array(m):
    p = W.params()
    P = m.make_params(p, d=10, method=1)
    with pytest.raises(m.MLMCError) as e:
        m.mlmc_level_noalloc(10, 1 << 22, P, m.FP32_EXACT, 1)   # 32768 CTAs > 16384
    assert e.value.status == m.EINVAL
