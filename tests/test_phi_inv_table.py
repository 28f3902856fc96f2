"""The FP32 exact path's inverse-Normal cubics (csrc/phi_inv_table.h): the
committed header is its generator's output, and the FP32 evaluation the
kernels perform (emulated here on the host) stays within its error bound of
Phi^{-1} in FP64 (scipy.special.ndtri) for words J across the whole range."""
import importlib.util
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_07123_gb300", "csrc")


def _header_table():
    txt = open(os.path.join(CSRC, "phi_inv_table.h")).read()
    rows = re.findall(r"\{([-0-9.e+f, ]+)\},", txt)
    return np.array([[float(v.strip().rstrip("f")) for v in r.split(",")] for r in rows], dtype=np.float32)


def _generator():
    spec = importlib.util.spec_from_file_location("gen_phi_inv_table", os.path.join(CSRC, "gen_phi_inv_table.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_header_is_the_generator_output():
    pytest.importorskip("scipy")
    c = _generator().coefficients().astype(np.float32)
    assert c.shape == (512, 4)
    h = _header_table()
    assert h.shape == (513, 4)
    np.testing.assert_array_equal(h[:512], c)
    np.testing.assert_array_equal(h[512], 0.0)   # u = 1/2


def _fma32(a, b, c):
    # a b + c of float32 operands: the product is exact in FP64, one rounding
    # of the FP64 sum, then to FP32 (a double rounding: within the test's margin)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _emulate(J, C):
    """exact_normal_f32 of device_common.cuh, step by step on the host."""
    J = J.astype(np.uint64)
    upper = J >= 2 ** 31
    Jp = np.where(upper, (2 ** 32 - 1) - J, J)
    # J' rounded to nearest as a float
    q = Jp.astype(np.float32)
    u = _fma32(q, np.float32(2.0 ** -32), np.float32(2.0 ** -33))
    b = u.view(np.uint32).astype(np.uint64)
    idx = (b >> 19).astype(np.int64) - (94 << 4)
    assert idx.min() >= 0 and idx.max() <= 512
    t = ((((b << 4) & 0x7FFFF0) | 0x3F800000).astype(np.uint32).view(np.float32) - np.float32(1.0)).astype(np.float32)
    c = C[idx]
    z = _fma32(_fma32(_fma32(c[:, 3], t, c[:, 2]), t, c[:, 1]), t, c[:, 0])
    return np.where(upper, -z, z).astype(np.float64), Jp


def _words():
    rng = np.random.default_rng(20250211)
    edge = [0, 1, 2, 3, 255, 256, 2 ** 24 - 1, 2 ** 24, 2 ** 24 + 1, 2 ** 31 - 129, 2 ** 31 - 128, 2 ** 31 - 65,
            2 ** 31 - 64, 2 ** 31 - 1]
    edge = edge + [2 ** 32 - 1 - j for j in edge]
    tails = np.floor(2.0 ** rng.uniform(0, 31, 100_000)).astype(np.uint64)   # every octave of u
    return np.concatenate([np.array(edge, dtype=np.uint64), tails, 2 ** 32 - 1 - tails,
                           rng.integers(0, 2 ** 32, 1_000_000, dtype=np.uint64)])


def test_fp32_evaluation_error_bound():
    ndtri = pytest.importorskip("scipy.special").ndtri
    J = _words()
    z, Jp = _emulate(J, _header_table())
    ref = ndtri((Jp.astype(np.float64) + 0.5) * 2.0 ** -32) * np.where(J >= 2 ** 31, -1.0, 1.0)
    err = np.abs(z - ref)
    # the float's rounding of u alone moves Phi^{-1} by up to ~8e-8 near u = 1/2
    assert np.all(err <= 1.5e-7 + 2e-7 * np.abs(ref)), float(np.max(err - 2e-7 * np.abs(ref)))
    # the cubics' own (FP64) interpolation error, over every part, is far below that
    c64 = _generator().coefficients()
    tt = np.linspace(0.0, 1.0, 65)
    parts = np.arange(512)
    E, m = parts // 16 - 33, parts % 16
    u = (2.0 ** E)[:, None] * (1.0 + (m[:, None] + tt[None, :]) / 16)
    fit = c64[:, :1] + tt * (c64[:, 1:2] + tt * (c64[:, 2:3] + tt * c64[:, 3:4]))
    assert np.max(np.abs(fit - ndtri(u))) < 2e-8
