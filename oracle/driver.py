"""MLMC sample-size formulas and the adaptive MLMC driver (oracle side).

TEST INFRASTRUCTURE ONLY (tests/, __graft_entry__.smoke(), bench.py's
CPU-baseline / reference arm).

Sec. 2.1: with per-level variance V_l and cost C_l, minimising
sum N_l C_l subject to sum V_l / N_l = eps^2 gives N_l = lambda sqrt(V_l / C_l)
with lambda = eps^-2 sum_k sqrt(V_k C_k), and total cost
eps^-2 (sum_l sqrt(V_l C_l))^2 (eq. total_cost_MLMC).
Sec. 2.2: the nested estimator has two terms per level (the approximate
level difference and the exact-minus-approximate correction) and the same
formula applies over all 2(L+1) terms with one multiplier lambda_M.

The adaptive loop is the one of Giles (2008), which Sec. 6 says the on-line
phase follows, in the form Giles (2015) gives it: each round evaluates every
pending sample and recomputes the optimal counts; the bias test (and with it
a new level) waits only until every remaining top-up is at most
ALMOST_DONE = 1% of its term's samples, so a new level's first samples run in
the same round as those small top-ups; the run ends when nothing is pending
and the test passed (or L = L_max).  Stated constants (the paper gives none):
variance target (1 - theta) eps^2 with theta = 1/2, bias target sqrt(theta)
eps, weak order alpha = 1 (Euler-Maruyama), extrapolated variance decay beta
(1 for Euler-Maruyama, 2 for Milstein) for a newly added level, L_min = 2,
N_init = 10^4, L_max = 10.  Costs follow the model C = 2^l c_kind, so the
sample counts are deterministic functions of the sums.
"""
import math

from . import core


def optimal_n(V, C, var_target):
    """Real-valued optimal sample counts N_k = lambda sqrt(V_k / C_k)."""
    lam = sum(math.sqrt(v * c) for v, c in zip(V, C)) / var_target
    return [lam * math.sqrt(v / c) if v > 0 else 0.0 for v, c in zip(V, C)]


def total_cost(V, C, eps2):
    """eps^-2 (sum sqrt(V C))^2, eq. total_cost_MLMC (and its nested analogue)."""
    return (sum(math.sqrt(v * c) for v, c in zip(V, C))) ** 2 / eps2


def floor_levels(values, factor):
    """Giles' safeguard against levels whose few samples show almost nothing:
    from level 2 on, x_l >= x_{l-1} / (2 factor), applied in level order."""
    out = list(values)
    for l in range(2, len(out)):
        out[l] = max(out[l], 0.5 * out[l - 1] / factor)
    return out


def bias_estimate(means, alpha=1.0):
    """Giles (2008) remaining-bias estimate from the last two (floored) level means."""
    m = floor_levels([abs(x) for x in means], 2.0 ** alpha)
    L = len(m) - 1
    r = m[L] / (2.0 ** alpha - 1.0)
    if L >= 1:
        r = max(r, m[L - 1] / 2.0 ** alpha / (2.0 ** alpha - 1.0))
    return r


PLAIN_FP64, PLAIN_FP32, NESTED_FIXED, NESTED_FP16, NESTED_BF16, NESTED_FIXED_EXACT_LOW, NESTED_FP16_EXACT_LOW = range(7)
# half-precision increments with S in FP32
NESTED_FP16S, NESTED_BF16S, NESTED_FP16S_EXACT_LOW, NESTED_BF16S_EXACT_LOW = range(7, 11)

# The bias test runs once every pending top-up is at most this fraction of its
# term's samples.
ALMOST_DONE = 0.01

# Levels whose approximate level difference is computed exactly, by enumerating
# the 2^(d 2^l) combinations of table cells (d 2^l <= EXACT_MAX_BITS).
EXACT_MAX_BITS = 20


def exact_levels(mode, d):
    if mode not in (NESTED_FIXED_EXACT_LOW, NESTED_FP16_EXACT_LOW, NESTED_FP16S_EXACT_LOW, NESTED_BF16S_EXACT_LOW):
        return set()
    return {lev for lev in (0, 1) if (d << lev) <= EXACT_MAX_BITS}


def estimator_plan(mode):
    """Per-level estimator variants for a driver mode."""
    return {
        PLAIN_FP64: [core.FP64_EXACT],
        PLAIN_FP32: [core.FP32_EXACT],
        NESTED_FIXED: [core.FIXED_APPROX, core.CORR_FIXED],
        NESTED_FP16: [core.FP16_APPROX, core.CORR_FP16],
        NESTED_BF16: [core.BF16_APPROX, core.CORR_BF16],
        NESTED_FIXED_EXACT_LOW: [core.FIXED_APPROX, core.CORR_FIXED],
        NESTED_FP16_EXACT_LOW: [core.FP16_APPROX, core.CORR_FP16],
        NESTED_FP16S: [core.FP16S_APPROX, core.CORR_FP16S],
        NESTED_BF16S: [core.BF16S_APPROX, core.CORR_BF16S],
        NESTED_FP16S_EXACT_LOW: [core.FP16S_APPROX, core.CORR_FP16S],
        NESTED_BF16S_EXACT_LOW: [core.BF16S_APPROX, core.CORR_BF16S],
    }[mode]


def mlmc(eps, p, seed, mode=PLAIN_FP64, cost=None, fmt_of_level=None, d=10, method=1,
         request=0, L_min=2, L_max=10, N_init=10_000, theta=0.5):
    """Adaptive (nested) MLMC; returns dict(price, var, L, N=[[N per estimator] per level])."""
    plan = estimator_plan(mode)
    ne = len(plan)
    if cost is None:
        cost = {v: 1.0 for v in plan}
    beta = 2.0 if p["scheme"] == core.MILSTEIN else 1.0
    disc = math.exp(-p["r"] * p["T"])
    L = L_min
    N = [[0] * ne for _ in range(L + 1)]
    S1 = [[0.0] * ne for _ in range(L + 1)]
    S2 = [[0.0] * ne for _ in range(L + 1)]
    dN = [[N_init] * ne for _ in range(L + 1)]
    extrap = [[None] * ne for _ in range(L + 1)]
    exact = exact_levels(mode, d)
    for lev in exact:
        dN[lev][0] = 1 << (d << lev)   # every combination of table cells once

    def is_exact(lev, k):
        return k == 0 and lev in exact

    def _vc():
        """Floored level variances and costs of every (level, estimator), level-major."""
        cols = []
        for k in range(ne):
            col = []
            for lev in range(L + 1):
                if is_exact(lev, k):
                    col.append(0.0)          # an exact mean has no variance
                elif N[lev][k] > 0:
                    m = S1[lev][k] / N[lev][k]
                    col.append(max(S2[lev][k] / N[lev][k] - m * m, 0.0))
                else:
                    col.append(extrap[lev][k])
            cols.append(floor_levels(col, 2.0 ** beta))
        V = [max(cols[k][lev], 1e-300) for lev in range(L + 1) for k in range(ne)]
        C = [cost[plan[k]] * 2.0 ** lev for lev in range(L + 1) for k in range(ne)]
        return V, C

    def run(lev, k, count):
        v = plan[k]
        fmt = fmt_of_level(lev) if fmt_of_level else None
        s, _ = core.level(p, lev, N[lev][k], count, v, seed, request=request, d=d,
                          method=method, fmt=fmt, enumerate=1 if is_exact(lev, k) else 0)
        S1[lev][k] += disc * s["sum"]
        S2[lev][k] += disc * disc * s["sum2"]
        N[lev][k] += count

    while True:
        # one round: every pending sample, then the optimal counts again
        for lev in range(L + 1):
            for k in range(ne):
                if dN[lev][k] > 0:
                    run(lev, k, dN[lev][k])
        Nopt = optimal_n(*_vc(), (1.0 - theta) * eps * eps)
        for lev in range(L + 1):
            for k in range(ne):
                want = int(math.ceil(Nopt[lev * ne + k]))
                dN[lev][k] = max(0, want - N[lev][k])
        # the bias test waits until every remaining top-up is small
        if any(dN[lev][k] > ALMOST_DONE * N[lev][k] for lev in range(L + 1) for k in range(ne)):
            continue
        means = [sum(S1[lev][k] / N[lev][k] for k in range(ne)) for lev in range(L + 1)]
        if bias_estimate(means) <= math.sqrt(theta) * eps or L >= L_max:
            if all(x == 0 for row in dN for x in row):
                break
            continue
        # add a level with extrapolated variances; its first samples run in the
        # same round as the remaining top-ups
        L += 1
        N.append([0] * ne)
        S1.append([0.0] * ne)
        S2.append([0.0] * ne)
        prev_var = []
        for k in range(ne):
            m = S1[L - 1][k] / N[L - 1][k]
            prev_var.append(max(S2[L - 1][k] / N[L - 1][k] - m * m, 1e-300) / 2.0 ** beta)
        extrap.append(prev_var)
        Nopt = optimal_n(*_vc(), (1.0 - theta) * eps * eps)
        dN = [[max(0, int(math.ceil(Nopt[lev * ne + k])) - N[lev][k]) for k in range(ne)]
              for lev in range(L + 1)]
    price = sum(S1[lev][k] / N[lev][k] for lev in range(L + 1) for k in range(ne))
    var = 0.0
    for lev in range(L + 1):
        for k in range(ne):
            if is_exact(lev, k):
                continue
            m = S1[lev][k] / N[lev][k]
            var += max(S2[lev][k] / N[lev][k] - m * m, 0.0) / N[lev][k]
    return dict(price=price, var=var, L=L, N=N)


def price_on_schedule(p, seed, mode, N, fmt_of_level=None, d=10, method=1, request=0, pack=0, dump=False):
    """Price and variance from fixed per-(level, estimator) sample counts N[l][k]
    (samples [0, N) of each term; entries beyond the mode's estimators are
    ignored).  Approximate-only terms read packed draws when pack is set.  In the
    modes with exact low levels, the approximate term of such a level is the mean
    over every combination of table cells (N[l][0] = 2^(d 2^l)) and adds no
    variance.  With dump, also returns every term's per-sample records."""
    plan = estimator_plan(mode)
    exact = exact_levels(mode, d)
    disc = math.exp(-p["r"] * p["T"])
    price, var = 0.0, 0.0
    sums, dumps = [], []
    for lev, row in enumerate(N):
        srow, drow = [], []
        for k, n in enumerate(row[:len(plan)]):
            v = plan[k]
            is_exact = k == 0 and lev in exact
            approx_only = v in core.APPROX_ONLY_VARIANTS
            fmt = fmt_of_level(lev) if fmt_of_level else None
            s, dm = core.level(p, lev, 0, n, v, seed, request=request, d=d, method=method, fmt=fmt,
                               dump=dump, pack=pack if approx_only and not is_exact else 0,
                               enumerate=1 if is_exact else 0)
            m = disc * s["sum"] / n
            price += m
            if not is_exact:
                var += max(disc * disc * s["sum2"] / n - m * m, 0.0) / n
            srow.append(s)
            drow.append(dm)
        sums.append(srow)
        dumps.append(drow)
    out = dict(price=price, var=var, sums=sums)
    if dump:
        out["dumps"] = dumps
    return out
