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

Method 2 (Sec. 3.2): the d-bit index j is split into n fields of b = d/n bits
(the first field is the top bits); each field gives X = +-x_k from a small
table of 2^(b-1) values with the Method-1 sign rule, and the approximate
Normal is the sum of the n values.  Reading (summation order): the sum is
formed as sum_k c_k x_k over the small-table indices k in ascending order,
c_k the net count of +x_k minus -x_k among the fields (terms with c_k = 0
left out), so that indices whose fields hold the same values in another
order, or a cancelling pair, get the identical FP64 sum (exactly tied and
ranked by j), as the mathematical sum does; for n = 2 this is the plain sum.  The small table starts as the b-bit
Method-1 table divided by sqrt(n); then, repeatedly, the 2^d sums are sorted
ascending (ties by j), which defines the permutation pi (pi(j) = rank of
Z~_j), and the small table is refitted by least squares to the d-bit
Method-1 values of the intervals the sums are ranked at, Z_{pi(j)}, until pi
no longer changes.  Reading (cycles): for n > 2 the iteration can alternate
between permutations for ever (period 2 at (d, n) = (8, 4) and (12, 3)); it
stops when the new permutation equals any earlier one, convergence being the
case of the last one, and keeps the last fit with its own ranking.  The exact path uses the uniform in interval pi(j) with
J's low bits: U = 2^-d pi(j) + 2^-32 ((J mod 2^(32-d)) + 1/2).

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


def m1_full(d: int) -> np.ndarray:
    """The d-bit Method-1 values of every interval j < 2^d in ascending order
    (lower half Z_j, upper half -Z_{2^d - 1 - j})."""
    half = m1_fp64(d)
    return np.concatenate([half, -half[::-1]])


def _m2_fields(d: int, n: int):
    """Per field i (top bits first): (index into the small table, sign) for every j < 2^d."""
    b = d // n
    full, half = 1 << b, 1 << (b - 1)
    j = np.arange(1 << d)
    out = []
    for i in range(n):
        f = (j >> (b * (n - 1 - i))) & (full - 1)
        low = f < half
        out.append((np.where(low, f, full - 1 - f), np.where(low, 1.0, -1.0)))
    return out


def m2_design(d: int, n: int) -> np.ndarray:
    """Matrix A (2^d x 2^(b-1)) with Z~ = A x: field value f < 2^(b-1) adds +x_f,
    otherwise -x_{2^b - 1 - f} (the Method-1 sign rule per field)."""
    b = d // n
    A = np.zeros((1 << d, 1 << (b - 1)))
    rows = np.arange(1 << d)
    for idx, sgn in _m2_fields(d, n):
        np.add.at(A, (rows, idx), sgn)
    return A


def m2_sums(x: np.ndarray, d: int, n: int) -> np.ndarray:
    """Z~_j = X^(1) + ... + X^(n) in FP64 as sum_k c_k x_k: the nonzero net counts
    c_k (row j of the design matrix) in ascending k, each product and each
    addition rounded once, from +0."""
    A = m2_design(d, n)
    acc = np.zeros(1 << d)
    for k in range(A.shape[1]):
        c = A[:, k]
        nz = c != 0
        acc[nz] = acc[nz] + c[nz] * x[k]
    return acc


def m2_rank(values: np.ndarray) -> np.ndarray:
    """pi(j) = position of values[j] in the ascending order (ties by j)."""
    order = np.argsort(values, kind="stable")
    pi = np.empty(len(values), dtype=np.int64)
    pi[order] = np.arange(len(values))
    return pi


def m2_mse(values: np.ndarray, pi: np.ndarray, d: int) -> float:
    """E[(Phi^{-1}(U) - Z~)^2] with U in interval pi(j): the Method-1 MSE plus
    2^-d sum_j (Z_{pi(j)} - Z~_j)^2 (the decomposition of eq. mse_dyadic)."""
    _, mse1 = moments_m1(d)
    return float(mse1) + float(np.sum((m1_full(d)[pi] - values) ** 2)) / (1 << d)


@functools.lru_cache(maxsize=None)
def m2_optimise(d: int, n: int = 2, max_iter: int = 1000):
    """Method 2 small table after the iterative least-squares stage; returns
    dict(x, values, pi, iterations, x0, mse0, mse).  The iteration stops when the
    permutation no longer changes (or after max_iter least-squares solves)."""
    if d % n or d // n < 2:
        raise ValueError("n must divide d with at least 2 bits per field")
    b = d // n
    A = m2_design(d, n)
    T = m1_full(d)
    x0 = m1_fp64(b) / np.sqrt(n)
    v0 = m2_sums(x0, d, n)
    pi0 = m2_rank(v0)
    x, pi, it = x0, pi0, 0
    seen = {pi0.tobytes()}
    while it < max_iter:
        x = np.linalg.lstsq(A, T[pi], rcond=None)[0]
        it += 1
        v = m2_sums(x, d, n)
        new = m2_rank(v)
        key = new.tobytes()
        pi = new
        if key in seen:          # converged, or back in an earlier state
            break
        seen.add(key)
    v = m2_sums(x, d, n)
    return {"x": x, "values": v, "pi": pi, "iterations": it, "x0": x0, "mse0": m2_mse(v0, pi0, d),
            "mse": m2_mse(v, pi, d)}


def m2_table(d: int, rep: str, fZ: int = 0, n: int = 2) -> np.ndarray:
    """Method-2 values of every j < 2^d in a representation: each small-table value
    rounded once (fixed: to fZ bits; fp16 / bf16; fp32), then sum_k c_k x_k over
    the nonzero net counts in ascending k, exactly in fixed point and otherwise
    with one rounding per product c_k x_k and per addition."""
    import math
    res = m2_optimise(d, n)
    x = res["x"]
    A = m2_design(d, n).astype(np.int64)
    if rep == "fp64":
        return res["values"]
    if rep == "fixed":
        xq = [round_fixed(v, fZ) for v in x]
    elif rep == "fp16":
        xq = list(_round_fp16(x))
    elif rep == "bf16":
        xq = list(_round_bf16(x))
    elif rep == "fp32":
        xq = [float(np.float32(v)) for v in x]
    else:
        raise ValueError(rep)
    def rnd(v):
        if rep == "fp16":
            return float(_round_fp16(np.array([v]))[0])
        if rep == "bf16":
            return float(_round_bf16(np.array([v]))[0])
        if rep == "fp32":
            return float(np.float32(v))
        return v                           # fixed: integers, exact

    out = np.empty(1 << d)
    for j in range(1 << d):
        acc = 0
        for k in np.nonzero(A[j])[0]:
            acc = rnd(acc + rnd(int(A[j, k]) * xq[k]))
        out[j] = math.ldexp(acc, -fZ) if rep == "fixed" else acc
    return out


def table(d: int, method: int, rep: str, fZ: int = 0, fields: int = 2) -> np.ndarray:
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
    if method == 2:
        return m2_table(d, rep, fZ, fields)[:half]
    if method != 3:
        raise ValueError("method must be 1, 2 or 3")
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
