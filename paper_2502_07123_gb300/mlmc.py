"""Python binding of libmlmc_gb300.so (the C ABI of include/mlmc.h).

Argument marshalling only: every step of the level simulation runs in the
CUDA library.  PyTorch is used for device memory (per-sample dumps) and for
the current CUDA stream.  There is no fallback: if the library has not been
built, or no CUDA device is usable, the calls raise MLMCError.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmlmc_gb300.so")

# enums (include/mlmc.h)
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EOVERFLOW, ENOTREADY = range(7)
EULER, MILSTEIN = 0, 1
EURO, DIGITAL, ASIAN, LOOKBACK = 0, 1, 2, 3
FP64_EXACT, FP32_EXACT, FP16_APPROX, BF16_APPROX, FIXED_APPROX, NESTED_CORR_FIXED, NESTED_CORR_FP16, \
    NESTED_CORR_BF16 = range(8)
# binary16 / bfloat16 increments with S in FP32
FP16S_APPROX, BF16S_APPROX, NESTED_CORR_FP16S, NESTED_CORR_BF16S = range(8, 12)
MODE_PLAIN_FP64, MODE_PLAIN_FP32, MODE_NESTED_FIXED, MODE_NESTED_FP16, MODE_NESTED_BF16, \
    MODE_NESTED_FIXED_EXACT_LOW, MODE_NESTED_FP16_EXACT_LOW = range(7)
MODE_NESTED_FP16S, MODE_NESTED_BF16S, MODE_NESTED_FP16S_EXACT_LOW, MODE_NESTED_BF16S_EXACT_LOW = range(7, 11)
WORK_ENUMERATE = 1
REP_FP64, REP_FP32, REP_FP16, REP_BF16, REP_FIXED = range(5)


class MLMCError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.mlmc_strerror(status).decode() if _lib is not None else str(status)
        super().__init__("%s: %s (status %d)" % (where, msg, status))


class Format(ctypes.Structure):
    _fields_ = [("e", ctypes.c_int8 * 7), ("f", ctypes.c_int8 * 7)]


class Params(ctypes.Structure):
    _fields_ = [("S0", ctypes.c_double), ("K", ctypes.c_double), ("r", ctypes.c_double),
                ("sigma", ctypes.c_double), ("T", ctypes.c_double),
                ("payoff", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("icdf_method", ctypes.c_int32), ("icdf_bits", ctypes.c_int32),
                ("formats", ctypes.POINTER(Format)), ("n_formats", ctypes.c_int32),
                ("request_id", ctypes.c_uint32), ("rng_pack", ctypes.c_int32), ("icdf_fields", ctypes.c_int32)]


class Sums(ctypes.Structure):
    _fields_ = [("sum", ctypes.c_double), ("sum2", ctypes.c_double), ("n", ctypes.c_uint64),
                ("seconds", ctypes.c_double), ("saturations", ctypes.c_uint64),
                ("isum", ctypes.c_int64), ("isum2_lo", ctypes.c_uint64), ("isum2_hi", ctypes.c_uint64),
                ("unit", ctypes.c_int32), ("exact_int", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("steps_per_thread", ctypes.c_int32)]


class EngineConfig(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("max_level", ctypes.c_int32),
                ("device_bytes_budget", ctypes.c_uint64), ("iters_per_launch", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Sensitivity(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double * 7), ("B", ctypes.c_double * 7), ("maxabs", ctypes.c_double * 7),
                ("mean", ctypes.c_double), ("var", ctypes.c_double), ("n", ctypes.c_uint64),
                ("n_instances", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class OptConfig(ctypes.Structure):
    _fields_ = [("c_rng", ctypes.c_double), ("mul", ctypes.c_double * 7), ("add", ctypes.c_double * 7),
                ("lut_mse", ctypes.POINTER(ctypes.c_double)), ("lut_max_bits", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class OptResult(ctypes.Structure):
    _fields_ = [("e", ctypes.c_int32 * 7), ("d", ctypes.c_int32 * 7), ("d_real", ctypes.c_double * 7),
                ("lambda_", ctypes.c_double), ("v_indep", ctypes.c_double), ("v_indep_real", ctypes.c_double),
                ("v_corr", ctypes.c_double), ("cost_lp", ctypes.c_double), ("cost_exact", ctypes.c_double),
                ("level_cost_ratio", ctypes.c_double), ("mse_term", ctypes.c_double),
                ("lut_bits", ctypes.c_int32), ("reserved", ctypes.c_int32), ("format", Format)]


class Work(ctypes.Structure):
    _fields_ = [("params", ctypes.POINTER(Params)), ("level", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("first_sample", ctypes.c_uint64), ("N", ctypes.c_uint64),
                ("stream", ctypes.c_int32), ("flags", ctypes.c_int32)]


SAMPLE_DTYPE = np.dtype([("pf", "<f8"), ("pc", "<f8"), ("sf", "<f8"), ("sc", "<f8"),
                         ("af", "<f8"), ("ac", "<f8"), ("qf", "<i8"), ("qc", "<i8"),
                         ("y", "<f8"), ("sat", "<u4"), ("pad", "<u4")])
SAMPLE_BYTES = SAMPLE_DTYPE.itemsize

_lib = None


def load():
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmlmc_gb300.so is not built (run paper_2502_07123_gb300/build.py or "
                          "__graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    st = ctypes.c_int
    sig = {
        "mlmc_level": (st, [ctypes.c_int, ctypes.c_uint64, P(Params), ctypes.c_int, ctypes.c_uint64,
                            ctypes.c_uint64, P(Sums)]),
        "mlmc_level_dump": (st, [ctypes.c_int, ctypes.c_uint64, P(Params), ctypes.c_int, ctypes.c_uint64,
                                 ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p, P(Sums)]),
        "mlmc_level_noalloc": (st, [ctypes.c_int, ctypes.c_uint64, P(Params), ctypes.c_int, ctypes.c_uint64,
                                    ctypes.c_uint64, P(Sums), ctypes.c_void_p]),
        "mlmc_plan_create": (st, [P(ctypes.c_void_p), P(Work), ctypes.c_int, ctypes.c_uint64, P(Tuning)]),
        "mlmc_plan_launch": (st, [ctypes.c_void_p, ctypes.c_void_p]),
        "mlmc_plan_results": (st, [ctypes.c_void_p, P(Sums)]),
        "mlmc_plan_info": (st, [ctypes.c_void_p, P(ctypes.c_int), P(ctypes.c_uint64), P(ctypes.c_uint64),
                                P(ctypes.c_uint64), P(ctypes.c_uint64)]),
        "mlmc_plan_kernel_time": (st, [ctypes.c_void_p, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_double)]),
        "mlmc_plan_elapsed": (st, [ctypes.c_void_p, P(ctypes.c_double)]),
        "mlmc_plan_launch_info": (st, [ctypes.c_void_p, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int),
                                       P(ctypes.c_uint64), P(ctypes.c_uint64)]),
        "mlmc_plan_launch_items": (st, [ctypes.c_void_p, ctypes.c_int, P(ctypes.c_int32), ctypes.c_int,
                                        P(ctypes.c_int)]),
        "mlmc_plan_destroy": (None, [ctypes.c_void_p]),
        "mlmc_run": (st, [P(Work), ctypes.c_int, ctypes.c_uint64, P(Tuning), P(Sums), ctypes.c_void_p]),
        "mlmc_estimate": (st, [ctypes.c_double, P(Params), ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                               P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_uint64),
                               ctypes.c_int]),
        "mlmc_cost_model": (st, [ctypes.c_int, ctypes.c_double]),
        "mlmc_engine_create": (st, [P(ctypes.c_void_p), P(EngineConfig)]),
        "mlmc_engine_submit": (st, [ctypes.c_void_p, P(Params), ctypes.c_double, ctypes.c_int, ctypes.c_uint64,
                                    P(ctypes.c_uint64)]),
        "mlmc_engine_step": (st, [ctypes.c_void_p, ctypes.c_void_p, P(ctypes.c_int), P(ctypes.c_int)]),
        "mlmc_engine_poll": (st, [ctypes.c_void_p, ctypes.c_uint64, P(ctypes.c_double), P(ctypes.c_double),
                                  P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_double)]),
        "mlmc_engine_completed": (st, [ctypes.c_void_p, P(ctypes.c_uint64), ctypes.c_int, P(ctypes.c_int)]),
        "mlmc_engine_request_info": (st, [ctypes.c_void_p, ctypes.c_uint64, P(ctypes.c_uint64), ctypes.c_int,
                                          P(ctypes.c_double)]),
        "mlmc_engine_stats": (st, [ctypes.c_void_p, P(ctypes.c_uint64), P(ctypes.c_uint64), P(ctypes.c_uint64),
                                   P(ctypes.c_int)]),
        "mlmc_engine_graph_info": (st, [ctypes.c_void_p, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int),
                                        P(ctypes.c_uint64)]),
        "mlmc_engine_destroy": (None, [ctypes.c_void_p]),
        "mlmc_batch_estimate": (st, [P(Params), P(ctypes.c_double), ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.c_int, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double),
                                     P(ctypes.c_int), P(ctypes.c_int), ctypes.c_void_p]),
        "mlmc_autotune": (st, [P(Work), ctypes.c_int, ctypes.c_uint64, ctypes.c_int, P(Tuning)]),
        "mlmc_tuning_reset": (None, []),
        "mlmc_sensitivities": (st, [ctypes.c_int, ctypes.c_uint64, P(Params), ctypes.c_uint64, ctypes.c_uint64,
                                    P(Sensitivity), ctypes.c_void_p]),
        "mlmc_optimise_level": (st, [ctypes.c_int, P(Sensitivity), P(OptConfig), P(OptResult)]),
        "mlmc_icdf_method2": (st, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, P(ctypes.c_int)]),
        "mlmc_icdf_method2_table": (st, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_double)]),
        "mlmc_default_format": (st, [P(Params), ctypes.c_int, P(Format)]),
        "mlmc_icdf_table": (st, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_double)]),
        "mlmc_icdf_mse": (st, [ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_double)]),
        "mlmc_exact_normal_f32": (st, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
        "mlmc_philox": (st, [P(ctypes.c_uint32), ctypes.c_uint64, ctypes.c_uint64, P(ctypes.c_uint32)]),
        "mlmc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "mlmc_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status, where):
    if status != OK:
        raise MLMCError(status, where)


def _sums_dict(s):
    d = {k: getattr(s, k) for k, _ in Sums._fields_}
    d["isum2"] = (int(s.isum2_hi) << 64) | int(s.isum2_lo)
    return d


SUMS_DTYPE = np.dtype([(k, {ctypes.c_double: "<f8", ctypes.c_uint64: "<u8", ctypes.c_int64: "<i8",
                            ctypes.c_int32: "<i4"}[t]) for k, t in Sums._fields_])


def _sums_list(out, raw=False):
    """Results of an mlmc_sums array: a structured array (raw) or one dict per item."""
    a = np.frombuffer(out, dtype=SUMS_DTYPE)   # a view that keeps `out` alive
    if raw:
        return a
    names = SUMS_DTYPE.names
    res = []
    for row in a.tolist():
        d = dict(zip(names, row))
        d["isum2"] = (d["isum2_hi"] << 64) | d["isum2_lo"]
        res.append(d)
    return res


def make_params(p, d=10, method=1, formats=None, request=0, rng_pack=0, fields=0):
    """Build an mlmc_params from a dict (S0, K, r, sigma, T, payoff, scheme).

    formats: None (library default schedule) or a list, indexed by level, of
    {'e': [7], 'f': [7]}.  Returns the ctypes struct; the format array is kept
    alive as an attribute of the struct."""
    P = Params()
    P.S0, P.K, P.r, P.sigma, P.T = (float(p[k]) for k in ("S0", "K", "r", "sigma", "T"))
    P.payoff, P.scheme = int(p["payoff"]), int(p["scheme"])
    P.icdf_method, P.icdf_bits = int(method), int(d)
    P.request_id = int(request)
    P.rng_pack = int(rng_pack)
    P.icdf_fields = int(fields)
    if formats is not None:
        arr = (Format * len(formats))()
        for i, fm in enumerate(formats):
            for j in range(7):
                arr[i].e[j] = int(fm["e"][j])
                arr[i].f[j] = int(fm["f"][j])
        P.formats = ctypes.cast(arr, ctypes.POINTER(Format))
        P.n_formats = len(formats)
        P._keep = arr
    else:
        P.formats = None
        P.n_formats = 0
    return P


def mlmc_level(level, N, params, variant, seed, first_sample=0):
    L = load()
    s = Sums()
    _check(L.mlmc_level(level, N, ctypes.byref(params), variant, seed, first_sample, ctypes.byref(s)),
           "mlmc_level")
    return _sums_dict(s)


def mlmc_level_dump(level, N, params, variant, seed, first_sample=0, stream=-1):
    """Returns (sums dict, numpy structured array of the N samples)."""
    import torch
    L = load()
    buf = torch.empty(max(1, N) * SAMPLE_BYTES, dtype=torch.uint8, device="cuda")
    s = Sums()
    torch.cuda.synchronize()
    _check(L.mlmc_level_dump(level, N, ctypes.byref(params), variant, seed, first_sample, stream,
                             ctypes.c_void_p(buf.data_ptr()), ctypes.byref(s)), "mlmc_level_dump")
    host = buf[: N * SAMPLE_BYTES].cpu().numpy()
    return _sums_dict(s), host.view(SAMPLE_DTYPE)


def mlmc_level_noalloc(level, N, params, variant, seed, first_sample=0, stream=None):
    """mlmc_level without device allocation (scratch in a fixed device array of the
    library); `stream` is a cudaStream_t handle as int, a torch stream, or None for
    the legacy default stream."""
    L = load()
    s = Sums()
    h = ctypes.c_void_p(None) if stream is None else _stream_handle(stream)
    _check(L.mlmc_level_noalloc(level, N, ctypes.byref(params), variant, seed, first_sample, ctypes.byref(s), h),
           "mlmc_level_noalloc")
    return _sums_dict(s)


class WorkList:
    """A work list marshalled once (the mlmc_work array and the params it points
    to), for repeated mlmc_run / Plan calls on the same items."""

    def __init__(self, items):
        items = list(items)
        self.arr = (Work * len(items))()
        self.keep = [it["params"] for it in items]
        P = ctypes.POINTER(Params)
        for i, it in enumerate(items):
            self.arr[i] = Work(P(it["params"]), int(it["level"]), int(it["variant"]), int(it.get("first_sample", 0)),
                               int(it["N"]), int(it.get("stream", -1)), int(it.get("flags", 0)))

    def __len__(self):
        return len(self.arr)


def _works(items):
    """items: a WorkList, or a list of dict(params=Params, level, variant, first_sample=0, N, stream=-1)."""
    wl = items if isinstance(items, WorkList) else WorkList(items)
    return wl.arr, wl.keep


def _tuning(tuning):
    if tuning is None:
        return None
    t = Tuning()
    t.threads, t.steps_per_thread = int(tuning.get("threads", 0)), int(tuning.get("steps_per_thread", 0))
    return ctypes.byref(t)


_raw_stream = None


def _current_raw_stream():
    """torch's current stream on the current device as a raw cudaStream_t
    (without building a torch.cuda.Stream object on every call)."""
    global _raw_stream
    if _raw_stream is None:
        import torch
        get = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        if get is None:
            _raw_stream = lambda: torch.cuda.current_stream().cuda_stream
        else:
            _raw_stream = lambda: get(torch.cuda.current_device())
    return _raw_stream()


def _stream_handle(stream):
    if stream is None:
        return ctypes.c_void_p(_current_raw_stream())
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A device-resident work list (mlmc_plan_create / _launch / _results)."""

    def __init__(self, items, seed, tuning=None):
        L = load()
        self._arr, self._keep = _works(items)
        self.n = len(self._arr)
        self._h = ctypes.c_void_p()
        _check(L.mlmc_plan_create(ctypes.byref(self._h), self._arr, self.n, seed, _tuning(tuning)),
               "mlmc_plan_create")

    def launch(self, stream=None):
        _check(load().mlmc_plan_launch(self._h, _stream_handle(stream)), "mlmc_plan_launch")

    def results(self, raw=False):
        out = (Sums * self.n)()
        _check(load().mlmc_plan_results(self._h, out), "mlmc_plan_results")
        return _sums_list(out, raw)

    def info(self):
        k = ctypes.c_int()
        c, ps, hb, db = (ctypes.c_uint64() for _ in range(4))
        _check(load().mlmc_plan_info(self._h, ctypes.byref(k), ctypes.byref(c), ctypes.byref(ps),
                                     ctypes.byref(hb), ctypes.byref(db)), "mlmc_plan_info")
        return dict(kernels=k.value, ctas=c.value, path_steps=ps.value, h2d_bytes=hb.value, d2h_bytes=db.value)

    def launch_info(self, k):
        """(family, items, ctas, path_steps) of level-kernel launch k."""
        fam, items = ctypes.c_int(), ctypes.c_int()
        ctas, ps = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().mlmc_plan_launch_info(self._h, k, ctypes.byref(fam), ctypes.byref(items), ctypes.byref(ctas),
                                            ctypes.byref(ps)), "mlmc_plan_launch_info")
        return fam.value, items.value, ctas.value, ps.value

    def launch_items(self, k):
        """Work-list positions of the items of level-kernel launch k, in launch order."""
        n = ctypes.c_int()
        _check(load().mlmc_plan_launch_items(self._h, k, None, 0, ctypes.byref(n)), "mlmc_plan_launch_items")
        buf = (ctypes.c_int32 * max(1, n.value))()
        _check(load().mlmc_plan_launch_items(self._h, k, buf, n.value, ctypes.byref(n)), "mlmc_plan_launch_items")
        return [int(buf[i]) for i in range(n.value)]

    def kernel_time(self, k):
        """(family, ms) of level kernel k of the last launch (CUDA events on its stream)."""
        fam = ctypes.c_int()
        ms = ctypes.c_double()
        _check(load().mlmc_plan_kernel_time(self._h, k, ctypes.byref(fam), ctypes.byref(ms)),
               "mlmc_plan_kernel_time")
        return fam.value, ms.value

    def elapsed_ms(self):
        """Device time (ms) of the whole last launch (mlmc_plan_elapsed)."""
        ms = ctypes.c_double()
        _check(load().mlmc_plan_elapsed(self._h, ctypes.byref(ms)), "mlmc_plan_elapsed")
        return ms.value

    def close(self):
        if self._h:
            load().mlmc_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlmc_run(items, seed, tuning=None, stream=None, raw=False):
    """Plan, launch, read and release (mlmc_run); items a list of dicts or a WorkList.
    Returns one dict per item, or with raw a structured array (SUMS_DTYPE)."""
    L = load()
    arr, keep = _works(items)
    out = (Sums * len(arr))()
    _check(L.mlmc_run(arr, len(arr), seed, _tuning(tuning), out, _stream_handle(stream)), "mlmc_run")
    return _sums_list(out, raw)


def mlmc_sensitivities(level, N, params, seed, first_sample=0, per_instance=False):
    """Error-model statistics of DeltaP_l (mlmc_sensitivities): per-type A, B, maxima,
    mean and variance; with per_instance the 7 x n_instances array of E[xbar^2]."""
    L = load()
    out = Sensitivity()
    ni = (1 << level) + ((1 << level) // 2 if level > 0 else 0) + 1
    inst = np.zeros((7, ni), dtype=np.float64) if per_instance else None
    _check(L.mlmc_sensitivities(level, N, ctypes.byref(params), seed, first_sample, ctypes.byref(out),
                                inst.ctypes.data if per_instance else None), "mlmc_sensitivities")
    d = dict(A=list(out.A), B=list(out.B), maxabs=list(out.maxabs), mean=out.mean, var=out.var, n=out.n,
             n_instances=out.n_instances, struct=out)
    if per_instance:
        d["inst"] = inst
    return d


def mlmc_optimise_level(level, sens, c_rng=0.0, lut_mse=None, lut_max_bits=0, mul=None, add=None):
    """Optimal bit-widths of one level (mlmc_optimise_level, host only).  sens: a dict
    with A, B, maxabs, var (for example from mlmc_sensitivities); lut_mse: sequence
    indexed by table bits (MSE of the approximate Normal) or None."""
    L = load()
    S = Sensitivity()
    for t in range(7):
        S.A[t], S.B[t], S.maxabs[t] = sens["A"][t], sens["B"][t], sens["maxabs"][t]
    S.var = sens["var"]
    S.mean = sens.get("mean", 0.0)
    cfg = OptConfig()
    cfg.c_rng = c_rng
    if mul is not None:
        for t in range(7):
            cfg.mul[t], cfg.add[t] = mul[t], add[t]
    keep = None
    if lut_mse is not None:
        keep = (ctypes.c_double * len(lut_mse))(*[float(x) for x in lut_mse])
        cfg.lut_mse = keep
    cfg.lut_max_bits = lut_max_bits
    out = OptResult()
    _check(L.mlmc_optimise_level(level, ctypes.byref(S), ctypes.byref(cfg), ctypes.byref(out)),
           "mlmc_optimise_level")
    return dict(e=list(out.e), d=list(out.d), d_real=list(out.d_real), **{"lambda": out.lambda_},
                v_indep=out.v_indep, v_indep_real=out.v_indep_real, v_corr=out.v_corr, cost_lp=out.cost_lp,
                cost_exact=out.cost_exact, level_cost_ratio=out.level_cost_ratio, mse_term=out.mse_term,
                lut_bits=out.lut_bits, format={"e": list(out.format.e), "f": list(out.format.f)})


def mlmc_autotune(items, seed, reps=5):
    """Time the launch shapes of each kernel class in `items` and install the fastest
    (mlmc_autotune); returns the chosen (threads, steps_per_thread) per item."""
    L = load()
    arr, keep = _works(items)
    out = (Tuning * len(arr))()
    _check(L.mlmc_autotune(arr, len(arr), seed, reps, out), "mlmc_autotune")
    return [(t.threads, t.steps_per_thread) for t in out]


def mlmc_tuning_reset():
    load().mlmc_tuning_reset()


def mlmc_batch_estimate(params_list, eps, mode, seed, max_level=10, iters_per_launch=1, stream=None):
    """Batched adaptive MLMC through one engine (mlmc_batch_estimate).  params_list: Params
    structures (distinct request ids); eps: one accuracy per request."""
    L = load()
    n = len(params_list)
    P = (Params * n)(*params_list)
    E = (ctypes.c_double * n)(*[float(x) for x in eps])
    pr, se = (ctypes.c_double * n)(), (ctypes.c_double * n)()
    lv = (ctypes.c_int * n)()
    launches = ctypes.c_int()
    h = ctypes.c_void_p(None) if stream is None else _stream_handle(stream)
    _check(L.mlmc_batch_estimate(P, E, n, mode, seed, max_level, iters_per_launch, pr, se, lv,
                                 ctypes.byref(launches), h), "mlmc_batch_estimate")
    return dict(price=list(pr), stderr=list(se), L=list(lv), launches=launches.value)


def mlmc_estimate(eps, params, mode, seed, max_level=10):
    L = load()
    cap = max_level + 1
    price, se = ctypes.c_double(), ctypes.c_double()
    lev = ctypes.c_int()
    Nl = (ctypes.c_uint64 * (2 * cap))()
    _check(L.mlmc_estimate(eps, ctypes.byref(params), mode, seed, max_level, ctypes.byref(price),
                           ctypes.byref(se), ctypes.byref(lev), Nl, cap), "mlmc_estimate")
    N = [[int(Nl[2 * l]), int(Nl[2 * l + 1])] for l in range(lev.value + 1)]
    return dict(price=price.value, stderr=se.value, L=lev.value, N=N)


class Engine:
    """Continuous-batching engine (mlmc_engine_*): submit requests, step, poll."""

    def __init__(self, max_slots=256, max_level=10, device_bytes_budget=0, iters_per_launch=1):
        L = load()
        cfg = EngineConfig(max_slots, max_level, device_bytes_budget, iters_per_launch, 0)
        self._h = ctypes.c_void_p()
        _check(L.mlmc_engine_create(ctypes.byref(self._h), ctypes.byref(cfg)), "mlmc_engine_create")
        self._keep = {}

    def submit(self, params, eps, mode, seed):
        rid = ctypes.c_uint64()
        _check(load().mlmc_engine_submit(self._h, ctypes.byref(params), eps, mode, seed, ctypes.byref(rid)),
               "mlmc_engine_submit")
        return rid.value

    def step(self, stream=None):
        a, q = ctypes.c_int(), ctypes.c_int()
        h = ctypes.c_void_p(None) if stream is None else _stream_handle(stream)
        _check(load().mlmc_engine_step(self._h, h, ctypes.byref(a), ctypes.byref(q)), "mlmc_engine_step")
        return a.value, q.value

    def poll(self, rid):
        pr, se, lat = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        lev, done = ctypes.c_int(), ctypes.c_int()
        _check(load().mlmc_engine_poll(self._h, rid, ctypes.byref(pr), ctypes.byref(se), ctypes.byref(lev),
                                       ctypes.byref(done), ctypes.byref(lat)), "mlmc_engine_poll")
        if not done.value:
            return None
        return dict(price=pr.value, stderr=se.value, L=lev.value, latency_s=lat.value)

    def completed(self, cap=4096):
        """Ids of the requests that completed since the last call, in completion
        order (mlmc_engine_completed); at most cap per call."""
        ids = (ctypes.c_uint64 * max(1, cap))()
        n = ctypes.c_int()
        _check(load().mlmc_engine_completed(self._h, ids, cap, ctypes.byref(n)), "mlmc_engine_completed")
        return [int(ids[i]) for i in range(n.value)]

    def request_info(self, rid, cap_levels=21):
        """Schedule N[l] = [N_approx_or_plain, N_corr] per level and the final
        remaining-bias estimate of a completed request (mlmc_engine_request_info)."""
        Nl = (ctypes.c_uint64 * (2 * cap_levels))()
        rem = ctypes.c_double()
        _check(load().mlmc_engine_request_info(self._h, rid, Nl, cap_levels, ctypes.byref(rem)),
               "mlmc_engine_request_info")
        N = [[int(Nl[2 * l]), int(Nl[2 * l + 1])] for l in range(cap_levels)]
        while N and N[-1] == [0, 0]:
            N.pop()
        return dict(N=N, bias_estimate=rem.value)

    def stats(self):
        a, b, c = (ctypes.c_uint64() for _ in range(3))
        sl = ctypes.c_int()
        _check(load().mlmc_engine_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                        ctypes.byref(sl)), "mlmc_engine_stats")
        return dict(steps=a.value, launches=b.value, path_steps=c.value, slots=sl.value)

    def graph_info(self):
        g, c, it = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        cap = ctypes.c_uint64()
        _check(load().mlmc_engine_graph_info(self._h, ctypes.byref(g), ctypes.byref(c), ctypes.byref(it),
                                             ctypes.byref(cap)), "mlmc_engine_graph_info")
        return dict(groups=g.value, captures=c.value, iters_per_launch=it.value, partial_capacity=cap.value)

    def close(self):
        if self._h:
            load().mlmc_engine_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlmc_cost_model(kind, cost_per_step):
    _check(load().mlmc_cost_model(kind, cost_per_step), "mlmc_cost_model")


def mlmc_default_format(params, level):
    F = Format()
    _check(load().mlmc_default_format(ctypes.byref(params), level, ctypes.byref(F)), "mlmc_default_format")
    return {"e": [F.e[i] for i in range(7)], "f": [F.f[i] for i in range(7)]}


def mlmc_icdf_table(method, d, rep, fZ=0):
    out = (ctypes.c_double * (1 << (d - 1)))()
    _check(load().mlmc_icdf_table(method, d, rep, fZ, out), "mlmc_icdf_table")
    return np.frombuffer(out, dtype=np.float64).copy()


def mlmc_icdf_method2(d, n=2):
    """Method-2 small table, interval ranks pi and least-squares fits of n fields (mlmc_icdf_method2)."""
    n = n or 2
    x = np.zeros(1 << max(0, d // n - 1), dtype=np.float64)
    pi = np.zeros(1 << d, dtype=np.uint32)
    it = ctypes.c_int()
    _check(load().mlmc_icdf_method2(d, n, x.ctypes.data, pi.ctypes.data, ctypes.byref(it)), "mlmc_icdf_method2")
    return dict(x=x, pi=pi, iterations=it.value)


def mlmc_icdf_method2_table(d, n, rep, fZ=0):
    """Method-2 values of the indices k < 2^(d-1) in a representation (mlmc_icdf_method2_table)."""
    out = (ctypes.c_double * (1 << (d - 1)))()
    _check(load().mlmc_icdf_method2_table(d, n, rep, fZ, out), "mlmc_icdf_method2_table")
    return np.frombuffer(out, dtype=np.float64).copy()


def exact_normal_f32(J, z, stream=None):
    """z = the FP32 exact Normal of the uint32 words J (device tensors of equal
    length, z float32), as the level kernels compute it (mlmc_exact_normal_f32)."""
    if J.numel() != z.numel():
        raise ValueError("J and z differ in length")
    h = ctypes.c_void_p(None) if stream is None else _stream_handle(stream)
    _check(load().mlmc_exact_normal_f32(ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                        J.numel(), h), "mlmc_exact_normal_f32")
    return z


def icdf_mse(d, method=1, fields=0):
    """Mean square error E[(Z - Z~)^2] of the approximate Normal with d table bits
    (mlmc_icdf_mse)."""
    out = ctypes.c_double()
    _check(load().mlmc_icdf_mse(int(method), int(d), int(fields), ctypes.byref(out)), "mlmc_icdf_mse")
    return out.value


def mlmc_philox(ctr, seed):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    P = ctypes.POINTER(ctypes.c_uint32)
    _check(load().mlmc_philox(ctr.ctypes.data_as(P), ctr.shape[0], seed, out.ctypes.data_as(P)), "mlmc_philox")
    return out


def mlmc_strerror(status):
    return load().mlmc_strerror(status).decode()


def mlmc_version():
    return load().mlmc_version().decode()
