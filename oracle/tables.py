"""Approximate inverse-CDF tables for the CPU oracle (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline /
reference arm may import this module.  It shares nothing with the CUDA path,
which builds its own tables on the device.

Method 1 (Sec. 3.1): on [0, 1/2] the inverse Normal CDF is replaced by its
mean over each uniform interval [k 2^-d, (k+1) 2^-d], k < 2^(d-1):

    Z_k = 2^d * integral_{u_k}^{u_{k+1}} Phi^{-1}(u) du
        = 2^d * (phi(Phi^{-1}(u_k)) - phi(Phi^{-1}(u_{k+1}))),   phi(Phi^{-1}(0)) = 0,

(the second line is the antiderivative of z phi(z) after u = Phi(z)).  It is
evaluated here in mpmath at 40 significant digits and rounded once.

Method 3 (Sec. 3.3): Z_k is replaced by a + b k on each dyadic index class.
Reading of the classes: {0, 1}, {2, 3}, {4..7}, ..., {2^(d-2) .. 2^(d-1)-1},
i.e. d-1 classes (the table size stated in Sec. 3.3), with index 0 merged into
the first class so that the first two classes hold two points each, as stated
in Sec. 3.4.  (a, b) is the equal-weight least-squares line through (k, Z_k)
over the class (eq. mse_dyadic and the minimisation that follows it).

Representations handed to the C oracle (each rounded once from the stated
source value):
  fp64  : Z_k rounded to double
  fp32  : fp32(fp64 value)
  fp16  : binary16(fp64 value), round to nearest even
  bf16  : bfloat16(fp64 value), round to nearest even
  fixed : floor(fp64 value * 2^fZ + 1/2)   (ties toward +infinity)
Method 3 evaluates a + b k in the path's arithmetic:
  fp32/fp16/bf16 : fp32(a32 + b32 k) (one rounding, as a fused multiply-add
                   gives), then rounded to binary16/bfloat16 when needed;
  fixed          : A = rd_30(a), B = rd_30(b), value = rd_{30-fZ}(A + B k).
"""
import functools

import mpmath as mp
import numpy as np

M3_COEF_FRAC_BITS = 30


@functools.lru_cache(maxsize=None)
def m1_exact(d: int, dps: int = 40):
    """Method-1 table Z_k (k < 2^(d-1)) as mpmath numbers, closed form."""
    if not 2 <= d <= 16:
        raise ValueError("d must be in [2, 16]")
    with mp.workdps(dps):
        half = 1 << (d - 1)
        scale = mp.mpf(2) ** d

        def pdf_at_quantile(k):
            if k == 0:
                return mp.mpf(0)
            u = mp.mpf(k) / scale
            z = mp.sqrt(2) * mp.erfinv(2 * u - 1)
            return mp.exp(-z * z / 2) / mp.sqrt(2 * mp.pi)

        g = [pdf_at_quantile(k) for k in range(half + 1)]
        return tuple(scale * (g[k] - g[k + 1]) for k in range(half))


def m1_fp64(d: int) -> np.ndarray:
    return np.array([float(z) for z in m1_exact(d)], dtype=np.float64)


def _classes(d: int):
    """Dyadic index classes of Method 3 (see module docstring)."""
    out = [(0, 1)]
    for c in range(1, d - 1):
        out.append((1 << c, (1 << (c + 1)) - 1))
    return out


@functools.lru_cache(maxsize=None)
def m3_exact(d: int, dps: int = 40):
    """Least-squares (a, b) per class, as mpmath numbers."""
    Z = m1_exact(d)
    coef = []
    with mp.workdps(dps):
        for lo, hi in _classes(d):
            ks = list(range(lo, hi + 1))
            n = len(ks)
            kbar = mp.mpf(sum(ks)) / n
            zbar = mp.fsum(Z[k] for k in ks) / n
            sxx = mp.fsum((k - kbar) ** 2 for k in ks)
            sxy = mp.fsum((k - kbar) * (Z[k] - zbar) for k in ks)
            b = sxy / sxx
            a = zbar - b * kbar
            coef.append((a, b))
    return tuple(coef)


def m3_class_of(k: int) -> int:
    return 0 if k < 2 else k.bit_length() - 1


def m3_coefficients_fp64(d: int):
    return [(float(a), float(b)) for a, b in m3_exact(d)]


def round_fixed(x: float, f: int) -> int:
    """rd of a double to f fractional bits: floor(x 2^f + 1/2)."""
    import math
    return int(math.floor(math.ldexp(x, f) + 0.5))


def _round_fp16(x: np.ndarray) -> np.ndarray:
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def _round_bf16(x: np.ndarray) -> np.ndarray:
    from . import core
    return core.round_bf16(np.asarray(x, dtype=np.float64))


def table(d: int, method: int, rep: str, fZ: int = 0) -> np.ndarray:
    """Approximate-Normal value for every table index k < 2^(d-1), as float64.

    rep is one of 'fp64', 'fp32', 'fp16', 'bf16', 'fixed' (fixed values are
    n 2^-fZ, exactly representable as doubles).
    """
    half = 1 << (d - 1)
    if method == 1:
        z64 = m1_fp64(d)
        if rep == "fp64":
            return z64
        if rep == "fp32":
            return z64.astype(np.float32).astype(np.float64)
        if rep == "fp16":
            return _round_fp16(z64)
        if rep == "bf16":
            return _round_bf16(z64)
        if rep == "fixed":
            import math
            return np.array([math.ldexp(round_fixed(v, fZ), -fZ) for v in z64])
        raise ValueError(rep)
    if method != 3:
        raise ValueError("method must be 1 or 3")
    coef = m3_coefficients_fp64(d)
    if rep == "fixed":
        import math
        F = M3_COEF_FRAC_BITS
        out = []
        for k in range(half):
            a, b = coef[m3_class_of(k)]
            A, B = round_fixed(a, F), round_fixed(b, F)
            v = A + B * k
            sh = F - fZ
            q = (v + (1 << (sh - 1))) >> sh if sh > 0 else v << (-sh)
            out.append(math.ldexp(q, -fZ))
        return np.array(out)
    if rep == "fp64":
        return np.array([coef[m3_class_of(k)][0] + coef[m3_class_of(k)][1] * k for k in range(half)])
    vals = []
    for k in range(half):
        a, b = coef[m3_class_of(k)]
        a32, b32 = float(np.float32(a)), float(np.float32(b))
        exact = a32 + b32 * k          # exact in double (spans < 53 bits)
        vals.append(float(np.float32(exact)))
    v32 = np.array(vals)
    if rep == "fp32":
        return v32
    if rep == "fp16":
        return _round_fp16(v32)
    if rep == "bf16":
        return _round_bf16(v32)
    raise ValueError(rep)


def moments_m1(d: int, dps: int = 40):
    """E[Z~^2] and MSE = E[(Z - Z~)^2] = 1 - E[Z~^2] for Method 1 (exact)."""
    Z = m1_exact(d)
    with mp.workdps(dps):
        ez2 = 2 * mp.fsum(z * z for z in Z) / mp.mpf(2) ** d
        return ez2, 1 - ez2


def mse_m3(d: int, dps: int = 40):
    """MSE of Method 3 from eq. mse_dyadic: MSE_M1 + 2^-d sum (Zbar_k - Z_k)^2 (both halves)."""
    Z = m1_exact(d)
    coef = m3_exact(d)
    _, mse1 = moments_m1(d, dps)
    with mp.workdps(dps):
        extra = mp.fsum((coef[m3_class_of(k)][0] + coef[m3_class_of(k)][1] * k - Z[k]) ** 2
                        for k in range(len(Z)))
        return mse1 + 2 * extra / mp.mpf(2) ** d
