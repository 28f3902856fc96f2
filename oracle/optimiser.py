"""Bit-width optimisation of the low-precision path (oracle side).

TEST INFRASTRUCTURE ONLY (tests/ and bench.py's reporting may import it).

Follows Sec. 4-6 of the paper for one level l:

* error model (Sec. 4.2): V_indep(d) = 1/12 sum_t A_t 4^(e_t - d_t)
  (eq. optimistic) and V_corr(d) = (sum_t B_t 2^(e_t - d_t - 1))^2
  (eq. pessimistic), with A_t = E[sum over instances of xbar^2] and
  B_t = sum over instances of sqrt(E[xbar^2]) for the variable types
  t = Z, con1, con2, mul1, sum1, mul2, S of Algorithm 1, e_t the exponents
  and d_t the bit-widths (fractional bits f_t = d_t - e_t);
* cost model (Sec. 5, eq. cost_sq): C~(d) = steps (1/2 sum_t M_t d_t^2 +
  sum_t M'_t d_t), M_t / M'_t the multiplications / additions per time step
  variable t takes part in, steps = fine + coarse steps of one sample; the
  exact sample costs C = 2^l c_rng (Sec. 5);
* level cost (eq. level_cost2): F(d) = sqrt(V C~(d)) + sqrt(V_indep(d) C);
* Lagrange solve (Sec. 6.1, eq. Lagr): for a multiplier lambda each d_t
  solves (ln 4 / 12) A_t 4^(e_t - d_t) = lambda steps (M_t d_t + M'_t);
  golden-section search over log(lambda) minimises F(d(lambda));
* integer rounding (Sec. 6.2): round every d_t down, then add one bit at a
  time to the variable with the largest variance decrease per unit cost
  (eq. ratio_lagr) until V_indep is back at or below the real solution's;
* extended model (Sec. 4.3, eq. extended): the approximate Normals add
  A_Z MSE to V_indep; the table size is the smallest d_lut whose term does
  not exceed V_indep of the chosen widths.  Reading: the printed 1/12 in
  front of the MSE term belongs to the uniform rounding model only (MSE is
  already a mean square, and V'_corr carries no such factor), so the term is
  A_Z MSE.
"""
import math

VARS = ("Z", "con1", "con2", "mul1", "sum1", "mul2", "S")
# operands per time step of Algorithm 1: mul1 = con2 Z, sum1 = con1 + mul1,
# mul2 = S sum1, S = S + mul2
M_MUL = (1.0, 0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
M_ADD = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0, 1.0)
LN4 = math.log(4.0)
D_MIN, D_MAX = 1.0, 60.0


def exponent(maxabs):
    """Smallest integer e with |x| < 2^e (Sec. 4.1 exponents from the maximum)."""
    if maxabs <= 0.0:
        return 0
    return int(math.floor(math.log2(maxabs))) + 1


def steps_of(level):
    n = 1 << level
    return n + (n // 2 if level > 0 else 0)


def v_indep(A, e, d):
    return sum(a * 4.0 ** (ei - di) for a, ei, di in zip(A, e, d)) / 12.0


def v_corr(B, e, d):
    return sum(b * 2.0 ** (ei - di - 1) for b, ei, di in zip(B, e, d)) ** 2


def cost_lp(d, level, M=M_MUL, Mp=M_ADD):
    return steps_of(level) * (0.5 * sum(m * x * x for m, x in zip(M, d)) + sum(m * x for m, x in zip(Mp, d)))


def level_cost(V, C, A, e, d, level, M=M_MUL, Mp=M_ADD):
    return math.sqrt(V * cost_lp(d, level, M, Mp)) + math.sqrt(v_indep(A, e, d) * C)


def solve_widths(lam, A, e, level, M=M_MUL, Mp=M_ADD):
    """d_t(lambda): root of (ln4/12) A_t 4^(e_t - d) - lambda steps (M_t d + M'_t) by bisection."""
    st = steps_of(level)
    out = []
    for a, ei, m, mp in zip(A, e, M, Mp):
        def g(x):
            return LN4 / 12.0 * a * 4.0 ** (ei - x) - lam * st * (m * x + mp)
        lo, hi = D_MIN, D_MAX
        if g(lo) <= 0.0:
            out.append(lo)
            continue
        if g(hi) >= 0.0:
            out.append(hi)
            continue
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if g(mid) > 0.0:
                lo = mid
            else:
                hi = mid
        out.append(0.5 * (lo + hi))
    return out


def golden(f, a, b, iters=200):
    """Golden-section search for the minimum of a unimodal f on [a, b]."""
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    c, dd = b - gr * (b - a), a + gr * (b - a)
    fc, fd = f(c), f(dd)
    for _ in range(iters):
        if fc <= fd:
            b, dd, fd = dd, c, fc
            c = b - gr * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, dd, fd
            dd = a + gr * (b - a)
            fd = f(dd)
    return 0.5 * (a + b)


def round_widths(A, e, d_real, level, M=M_MUL, Mp=M_ADD):
    """Greedy integer rounding (Sec. 6.2)."""
    target = v_indep(A, e, d_real)
    d = [float(math.floor(x)) for x in d_real]
    while v_indep(A, e, d) > target:
        best, bt = -1.0, 0
        v0, c0 = v_indep(A, e, d), cost_lp(d, level, M, Mp)
        for t in range(len(d)):
            dn = list(d)
            dn[t] += 1.0
            r = (v0 - v_indep(A, e, dn)) / (cost_lp(dn, level, M, Mp) - c0)
            if r > best:
                best, bt = r, t
        d[bt] += 1.0
    return [int(x) for x in d]


def optimise_level(level, A, B, maxabs, V, c_rng=1e4, M=M_MUL, Mp=M_ADD, mse_of_lut=None):
    """Optimal bit-widths of one level; returns a dict with the real and integer
    solutions, the multiplier, the model variances and costs, and the table size."""
    e = [exponent(x) for x in maxabs]
    C = (1 << level) * c_rng

    def F_of_loglam(x):
        return level_cost(V, C, A, e, solve_widths(math.exp(x), A, e, level, M, Mp), level, M, Mp)

    x = golden(F_of_loglam, math.log(1e-40), math.log(1e10))
    lam = math.exp(x)
    d_real = solve_widths(lam, A, e, level, M, Mp)
    d_int = round_widths(A, e, d_real, level, M, Mp)
    out = {"e": e, "lambda": lam, "d_real": d_real, "d": d_int,
           "v_indep_real": v_indep(A, e, d_real), "v_indep": v_indep(A, e, d_int),
           "v_corr": v_corr(B, e, d_int), "cost_lp": cost_lp(d_int, level, M, Mp), "cost_exact": C,
           "level_cost_ratio": math.sqrt(cost_lp(d_int, level, M, Mp) / C) + math.sqrt(v_indep(A, e, d_int) / V)}
    if mse_of_lut is not None:
        lut = None
        for dl in range(2, 17):
            if A[0] * mse_of_lut(dl) <= out["v_indep"]:
                lut = dl
                break
        out["lut_bits"] = lut
        out["mse_term"] = A[0] * mse_of_lut(lut) if lut else None
    return out
