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
    # (variant, level, N, first, payoff, scheme, method, d, rng_pack)
    (W.FIXED_APPROX, 0, 200_000, 3, W.EURO, W.EULER, 1, 10, 0),
    (W.FIXED_APPROX, 6, 5_000, 0, W.DIGITAL, W.MILSTEIN, 3, 10, 0),
    (W.FP32_EXACT, 3, 20_000, 11, W.ASIAN, W.MILSTEIN, 1, 10, 0),
    (W.CORR_FIXED, 5, 3_000, 0, W.EURO, W.EULER, 1, 10, 0),
    (W.FP16_APPROX, 2, 50_000, 7, W.LOOKBACK, W.EULER, 3, 10, 0),
    (W.FP64_EXACT, 1, 4_000, 0, W.DIGITAL, W.EULER, 1, 10, 0),
    (W.CORR_BF16, 4, 2_000, 1, W.ASIAN, W.EULER, 1, 10, 0),
    # packed draws: three samples per pack on level 0, and one sample per
    # thread for a deep item smaller than one wave (the lane-split layout)
    (W.FIXED_APPROX, 0, 300_001, 5, W.EURO, W.EULER, 1, 10, 1),
    (W.FIXED_APPROX, 3, 5_000, 0, W.EURO, W.EULER, 1, 10, 1),
    (W.BF16_APPROX, 4, 7_001, 2, W.ASIAN, W.EULER, 3, 9, 1),
    # the largest table the scratch array holds (d = 14: a 64 KiB fixed-point table)
    (W.FIXED_APPROX, 0, 100_000, 0, W.EURO, W.EULER, 1, 14, 0),
    (W.CORR_FIXED, 2, 10_000, 0, W.DIGITAL, W.EULER, 1, 14, 0),
]


def _fn(m):
    lib = ctypes.CDLL(m.LIB_PATH)
    fn = lib.mlmc_level_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(m.Params), ctypes.c_int, ctypes.c_uint64,
                   ctypes.c_uint64, ctypes.POINTER(m.Sums), ctypes.c_void_p]
    return fn


def _call_c_abi(m, level, N, P, variant, seed, first, stream=None):
    """Call the entry point directly through the C ABI (ctypes); stream None is
    the legacy default stream, else a cudaStream_t handle (int)."""
    s = m.Sums()
    st = _fn(m)(level, N, ctypes.byref(P), variant, seed, first, ctypes.byref(s), stream)
    assert st == 0, m.mlmc_strerror(st)
    d = {k: getattr(s, k) for k, _ in m.Sums._fields_}
    d["isum2"] = (int(s.isum2_hi) << 64) | int(s.isum2_lo)
    return d


def _params(m, payoff, scheme, level, method, d, rng_pack):
    p = W.params(payoff=payoff, scheme=scheme)
    return m.make_params(p, d=d, method=method, formats=[W.default_format(p, lev) for lev in range(level + 1)],
                         rng_pack=rng_pack)


def _same(got, ref):
    """The same work item, chunking, kernels and chunk-ordered reduction as
    mlmc_level: every field of the result is identical, real sums included."""
    for k in ("n", "saturations", "exact_int", "unit", "isum", "isum2", "sum", "sum2"):
        assert got[k] == ref[k], (k, got[k], ref[k])


@pytest.mark.parametrize("variant,level,N,first,payoff,scheme,method,d,rng_pack", CASES)
def test_noalloc_matches_mlmc_level(m, variant, level, N, first, payoff, scheme, method, d, rng_pack):
    P = _params(m, payoff, scheme, level, method, d, rng_pack)
    ref = m.mlmc_level(level, N, P, variant, 99, first)
    for _ in range(2):  # the second call reuses the array the first one left behind
        _same(_call_c_abi(m, level, N, P, variant, 99, first), ref)


def test_noalloc_on_a_caller_stream(m):
    """On a non-blocking stream the caller created, results as on the default stream."""
    import torch
    P = _params(m, W.EURO, W.EULER, 4, 1, 10, 0)
    ref = m.mlmc_level(4, 30_000, P, W.CORR_FIXED, 5, 0)
    st = torch.cuda.Stream()
    for _ in range(2):
        _same(_call_c_abi(m, 4, 30_000, P, W.CORR_FIXED, 5, 0, stream=st.cuda_stream), ref)


def test_noalloc_leaves_device_memory_unchanged(m):
    """After one call of each kind (which may load kernel code once), further
    calls take no device memory: the free bytes stay the same over 50 calls."""
    import torch
    kinds = [(W.FIXED_APPROX, 0, 100_000, 1, 10, 1), (W.CORR_FIXED, 5, 3_000, 3, 10, 0),
             (W.FP32_EXACT, 3, 20_000, 1, 12, 0)]
    calls = []
    for v, lev, N, method, d, pack in kinds:
        P = _params(m, W.EURO, W.EULER, lev, method, d, pack)
        calls.append((lev, N, P, v))
        _call_c_abi(m, lev, N, P, v, 1, 0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(50):
        lev, N, P, v = calls[k % len(calls)]
        _call_c_abi(m, lev, N, P, v, 7 + k, 0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_sizes_beyond_its_array(m):
    p = W.params()
    P = m.make_params(p, d=10, method=1)
    with pytest.raises(m.MLMCError) as e:
        m.mlmc_level_noalloc(10, 1 << 22, P, m.FP32_EXACT, 1)   # 32768 CTAs > 16384
    assert e.value.status == m.EINVAL
    # sample ranges whose word indices would pass 2^62 (no wrap-around in the check)
    with pytest.raises(m.MLMCError) as e:
        m.mlmc_level_noalloc(3, (1 << 57) + 1, P, m.FIXED_APPROX, 1)
    assert e.value.status == m.EINVAL
    with pytest.raises(m.MLMCError) as e:
        m.mlmc_level_noalloc(2, 10, P, m.FIXED_APPROX, 1, first_sample=(1 << 58) - 5)
    assert e.value.status == m.EINVAL
