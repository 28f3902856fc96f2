"""ctypes wrapper of the C oracle (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline /
reference arm may import this module.  The record layouts below mirror the
structs of ``oracle/mlmc_oracle.c``; nothing here is shared with the CUDA
library.
"""
import ctypes

import numpy as np

from . import build as _build

EURO, DIGITAL, ASIAN, LOOKBACK = 0, 1, 2, 3
EULER, MILSTEIN = 0, 1
FP64_EXACT, FP32_EXACT, FP16_APPROX, BF16_APPROX, FIXED_APPROX, CORR_FIXED, CORR_FP16, CORR_BF16 = range(8)
# half-precision increments with S in FP32
FP16S_APPROX, BF16S_APPROX, CORR_FP16S, CORR_BF16S = range(8, 12)
VARIANT_NAMES = ["fp64_exact", "fp32_exact", "fp16_approx", "bf16_approx", "fixed_approx",
                 "corr_fixed", "corr_fp16", "corr_bf16", "fp16s_approx", "bf16s_approx", "corr_fp16s", "corr_bf16s"]
CORR_VARIANTS = (CORR_FIXED, CORR_FP16, CORR_BF16, CORR_FP16S, CORR_BF16S)
APPROX_ONLY_VARIANTS = (FP16_APPROX, BF16_APPROX, FIXED_APPROX, FP16S_APPROX, BF16S_APPROX)


def has_exact(v):
    return v in (FP64_EXACT, FP32_EXACT) + CORR_VARIANTS


def has_approx(v):
    return v not in (FP64_EXACT, FP32_EXACT)


def approx_rep(v):
    if v in (FIXED_APPROX, CORR_FIXED):
        return "fixed"
    if v in (FP16_APPROX, CORR_FP16, FP16S_APPROX, CORR_FP16S):
        return "fp16"
    if v in (BF16_APPROX, CORR_BF16, BF16S_APPROX, CORR_BF16S):
        return "bf16"
    return None


def default_stream(v):
    """Approximate-only estimators draw from stream 1, all others from stream 0."""
    return 1 if v in APPROX_ONLY_VARIANTS else 0


class Params(ctypes.Structure):
    _fields_ = [("S0", ctypes.c_double), ("K", ctypes.c_double), ("r", ctypes.c_double),
                ("sigma", ctypes.c_double), ("T", ctypes.c_double),
                ("payoff", ctypes.c_int32), ("scheme", ctypes.c_int32)]


class Format(ctypes.Structure):
    _fields_ = [("e", ctypes.c_int32 * 7), ("f", ctypes.c_int32 * 7)]


class Sample(ctypes.Structure):
    _fields_ = [("pf", ctypes.c_double), ("pc", ctypes.c_double),
                ("sf", ctypes.c_double), ("sc", ctypes.c_double),
                ("af", ctypes.c_double), ("ac", ctypes.c_double),
                ("qf", ctypes.c_int64), ("qc", ctypes.c_int64),
                ("y", ctypes.c_double), ("sat", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


SAMPLE_DTYPE = np.dtype([("pf", "<f8"), ("pc", "<f8"), ("sf", "<f8"), ("sc", "<f8"),
                         ("af", "<f8"), ("ac", "<f8"), ("qf", "<i8"), ("qc", "<i8"),
                         ("y", "<f8"), ("sat", "<u4"), ("pad", "<u4")])
assert SAMPLE_DTYPE.itemsize == ctypes.sizeof(Sample)


class Sums(ctypes.Structure):
    _fields_ = [("sum", ctypes.c_double), ("sum2", ctypes.c_double),
                ("isum", ctypes.c_int64), ("isum2_lo", ctypes.c_uint64), ("isum2_hi", ctypes.c_uint64),
                ("n", ctypes.c_uint64), ("saturations", ctypes.c_uint64),
                ("unit", ctypes.c_int32), ("exact_int", ctypes.c_int32)]


class Sens(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double * 7), ("maxabs", ctypes.c_double * 7), ("sum_dp", ctypes.c_double),
                ("sum_dp2", ctypes.c_double), ("n", ctypes.c_uint64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        L.or_philox_array.argtypes = [u32p, u32p, ctypes.c_uint64, u32p]
        L.or_draw_array.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                    u64p, u32p, ctypes.c_uint64, u32p]
        L.or_draw_packed_array.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                           u64p, u32p, ctypes.c_uint64, ctypes.c_int, u32p]
        L.or_exact_normal_array.argtypes = [u32p, ctypes.c_uint64, f64p]
        L.or_round_fp16_array.argtypes = [f64p, ctypes.c_uint64, f64p]
        L.or_round_bf16_array.argtypes = [f64p, ctypes.c_uint64, f64p]
        L.or_approx_normal_array.argtypes = [u32p, ctypes.c_uint64, ctypes.c_int, f64p, f64p]
        L.or_norminv_lower.argtypes = [ctypes.c_double]
        L.or_norminv_lower.restype = ctypes.c_double
        L.or_level.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                               ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                               ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(Format), ctypes.c_int,
                               ctypes.c_int, ctypes.POINTER(Sums), ctypes.c_void_p, ctypes.c_void_p]
        L.or_level.restype = ctypes.c_int
        L.or_sens_instances.argtypes = [ctypes.c_int]
        L.or_sens_instances.restype = ctypes.c_int
        L.or_sensitivities.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(Sens), ctypes.c_void_p]
        L.or_sensitivities.restype = ctypes.c_int
        L.or_sens_probe.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                    ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
        L.or_sens_probe.restype = ctypes.c_double
        _lib = L
    return _lib


def philox(ctr: np.ndarray, key) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    lib().or_philox_array(ctr.reshape(-1), k, ctr.shape[0], out.reshape(-1))
    return out


def draws(seed, request, level, stream, samples, steps) -> np.ndarray:
    s = np.ascontiguousarray(samples, dtype=np.uint64)
    t = np.ascontiguousarray(steps, dtype=np.uint32)
    out = np.empty(s.shape[0], dtype=np.uint32)
    lib().or_draw_array(seed, request, level, stream, s, t, s.shape[0], out)
    return out


def draws_packed(seed, request, level, stream, samples, steps, d) -> np.ndarray:
    s = np.ascontiguousarray(samples, dtype=np.uint64)
    t = np.ascontiguousarray(steps, dtype=np.uint32)
    out = np.empty(s.shape[0], dtype=np.uint32)
    lib().or_draw_packed_array(seed, request, level, stream, s, t, s.shape[0], int(d), out)
    return out


def exact_normal(J) -> np.ndarray:
    J = np.ascontiguousarray(J, dtype=np.uint32)
    out = np.empty(J.shape[0], dtype=np.float64)
    lib().or_exact_normal_array(J, J.shape[0], out)
    return out


def approx_normal(J, d, ztab) -> np.ndarray:
    J = np.ascontiguousarray(J, dtype=np.uint32)
    z = np.ascontiguousarray(ztab, dtype=np.float64)
    out = np.empty(J.shape[0], dtype=np.float64)
    lib().or_approx_normal_array(J, J.shape[0], int(d), z, out)
    return out


def round_fp16(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    out = np.empty_like(x)
    lib().or_round_fp16_array(x, x.shape[0], out)
    return out


def round_bf16(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    out = np.empty_like(x)
    lib().or_round_bf16_array(x, x.shape[0], out)
    return out


def make_format(fmt):
    """fmt: dict {'e': [7 ints], 'f': [7 ints]} in the order Z, con1, con2, mul1, sum1, mul2, S."""
    F = Format()
    for i in range(7):
        F.e[i] = int(fmt["e"][i])
        F.f[i] = int(fmt["f"][i])
    return F


class OracleError(RuntimeError):
    pass


def level(p, lev, first, N, variant, seed, request=0, stream=None, d=10, method=1,
          fmt=None, dump=False, pack=0, enumerate=0, fields=2):
    """Simulate samples [first, first+N) of one level; return (sums dict, dump array or None).

    p: dict with S0, K, r, sigma, T, payoff, scheme; fields: n of Method 2.
    """
    from . import tables
    if stream is None:
        stream = default_stream(variant)
    P = Params(p["S0"], p["K"], p["r"], p["sigma"], p["T"], int(p["payoff"]), int(p["scheme"]))
    ztab = None
    F = None
    rep = approx_rep(variant)
    if rep is not None:
        fZ = int(fmt["f"][0]) if rep == "fixed" else 0
        ztab = np.ascontiguousarray(tables.table(d, method, rep, fZ, fields), dtype=np.float64)
    if rep == "fixed":
        F = make_format(fmt)
    S = Sums()
    out = np.zeros(N, dtype=SAMPLE_DTYPE) if dump else None
    perm = None
    if method == 2 and variant in CORR_VARIANTS:
        perm = np.ascontiguousarray(tables.m2_optimise(d, fields)["pi"], dtype=np.uint32)
    st = lib().or_level(ctypes.byref(P), int(lev), int(first), int(N), int(variant), int(seed),
                        int(request), int(stream), int(d),
                        ztab.ctypes.data if ztab is not None else None,
                        ctypes.byref(F) if F is not None else None, int(pack), int(enumerate),
                        ctypes.byref(S), out.ctypes.data if dump else None,
                        perm.ctypes.data if perm is not None else None)
    if st != 0:
        raise OracleError("or_level returned %d" % st)
    sums = {k: getattr(S, k) for k, _ in Sums._fields_}
    sums["isum2"] = (int(S.isum2_hi) << 64) | int(S.isum2_lo)
    return sums, out


# ---------------------------------------------------------------------------
# Error-model statistics (Sec. 4.2-4.3), European call, Euler-Maruyama
# ---------------------------------------------------------------------------
SENS_VARS = ("Z", "con1", "con2", "mul1", "sum1", "mul2", "S")


def sens_instances(lev):
    return int(lib().or_sens_instances(int(lev)))


def sensitivities(p, lev, first, N, seed, request=0, per_instance=True):
    """Sums over samples [first, first+N) of the per-type squared sensitivities
    of DeltaP_l, maxima of |x| per type, sums of DeltaP and DeltaP^2, and (if
    per_instance) the per-instance sums of squared sensitivities (7 x n_inst)."""
    P = Params(p["S0"], p["K"], p["r"], p["sigma"], p["T"], int(p["payoff"]), int(p["scheme"]))
    S = Sens()
    ni = sens_instances(lev)
    inst = np.zeros((7, ni), dtype=np.float64) if per_instance else None
    st = lib().or_sensitivities(ctypes.byref(P), int(lev), int(first), int(N), int(seed), int(request),
                                ctypes.byref(S), inst.ctypes.data if per_instance else None)
    if st != 0:
        raise OracleError("or_sensitivities returned %d" % st)
    return {"A": np.array(S.A[:]), "maxabs": np.array(S.maxabs[:]), "sum_dp": S.sum_dp, "sum_dp2": S.sum_dp2,
            "n": S.n, "inst": inst}


def sens_probe(p, lev, seed, request, s, vtype, inst, delta, want_xbar=False):
    """DeltaP of sample s with delta added to one instance; with want_xbar also the
    adjoint sensitivities of every instance of the unperturbed sample (7 x n_inst)."""
    P = Params(p["S0"], p["K"], p["r"], p["sigma"], p["T"], int(p["payoff"]), int(p["scheme"]))
    xb = np.zeros((7, sens_instances(lev)), dtype=np.float64) if want_xbar else None
    dp = lib().or_sens_probe(ctypes.byref(P), int(lev), int(seed), int(request), int(s), int(vtype), int(inst),
                             float(delta), xb.ctypes.data if want_xbar else None)
    return (dp, xb) if want_xbar else dp
