"""The C ABI library builds for sm_103a, loads without a GPU and exports every
function include/mlmc.h declares; host-only helpers agree with their stated rules."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mlmc.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mlmc_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists(
            os.path.join(ROOT, "paper_2502_07123_gb300", "_build", "libmlmc_gb300.so")):
        pytest.skip("nvcc not available")
    from paper_2502_07123_gb300 import build
    build.build()
    from paper_2502_07123_gb300 import mlmc
    return mlmc


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("mlmc_level", "mlmc_estimate", "mlmc_level_dump", "mlmc_plan_create", "mlmc_plan_launch",
                     "mlmc_plan_results", "mlmc_run", "mlmc_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    L = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_struct_layouts(lib):
    assert ctypes.sizeof(lib.Params) == 80
    assert ctypes.sizeof(lib.Sums) == 72
    assert ctypes.sizeof(lib.Work) == 40
    assert lib.SAMPLE_BYTES == 80


def test_default_format_matches_input_schedule(lib):
    from paper_2502_07123_gb300 import workloads as W
    wide = 0
    for over in ({}, {"sigma": 0.4}, {"sigma": 0.1, "r": 0.0}, {"S0": 80.0, "K": 120.0, "T": 2.0},
                 {"scheme": W.MILSTEIN, "sigma": 0.5, "T": 0.25},
                 {"S0": 120.0, "K": 80.0, "sigma": 0.5, "T": 2.0}, {"S0": 5000.0, "K": 5000.0, "sigma": 0.3}):
        p = W.params(**over)
        P = lib.make_params(p)
        for lev in range(0, 21):
            f = W.default_format(p, lev)
            assert lib.mlmc_default_format(P, lev) == f, (over, lev)
            # S keeps to 30 bits (32-bit datapath) unless that would leave fewer than 10 fractional bits
            assert f["e"][6] + f["f"][6] <= 30 or f["f"][6] == 10
            wide += f["f"][6] < min(21, 14 + lev)
    assert wide > 0     # the cases above include options whose S gives up fractional bits


def test_strerror_and_version(lib):
    assert lib.mlmc_strerror(lib.EINVAL) == "invalid argument"
    assert "sm_103a" in lib.mlmc_version()


def test_host_argument_checks(lib):
    from paper_2502_07123_gb300 import workloads as W
    P = lib.make_params(W.params())
    with pytest.raises(lib.MLMCError) as e:
        lib.mlmc_default_format(P, 21)
    assert e.value.status == lib.EINVAL
    with pytest.raises(lib.MLMCError):
        lib.mlmc_cost_model(7, 1.0)
    lib.mlmc_cost_model(2, 0.0)  # restores the default


def test_no_cpu_fallback(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2502_07123_gb300 import workloads as W
    P = lib.make_params(W.params())
    with pytest.raises(lib.MLMCError) as e:
        lib.mlmc_level(2, 100, P, lib.FP32_EXACT, 1)
    assert e.value.status == lib.ECUDA


def test_null_handle_and_pointer_checks(lib):
    # argument checks that come before any CUDA call (no GPU needed)
    import ctypes
    L = ctypes.CDLL(lib.LIB_PATH)
    L.mlmc_engine_completed.restype = ctypes.c_int
    L.mlmc_engine_completed.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    n = ctypes.c_int(-1)
    ids = (ctypes.c_uint64 * 4)()
    assert L.mlmc_engine_completed(None, ids, 4, ctypes.byref(n)) == lib.EINVAL
    L.mlmc_plan_elapsed.restype = ctypes.c_int
    L.mlmc_plan_elapsed.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    ms = ctypes.c_double()
    assert L.mlmc_plan_elapsed(None, ctypes.byref(ms)) == lib.EINVAL
    L.mlmc_exact_normal_f32.restype = ctypes.c_int
    L.mlmc_exact_normal_f32.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
    assert L.mlmc_exact_normal_f32(None, None, 0, None) == lib.OK          # nothing to do
    assert L.mlmc_exact_normal_f32(None, None, 16, None) == lib.EINVAL
