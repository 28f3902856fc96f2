"""Pins of the sample-size formulas of Sec. 2 (eqs. total_cost_MLMC, cost_nested, var_nested)."""
import math

import numpy as np

from oracle import driver


def test_optimal_n_meets_variance_target_and_cost():
    rng = np.random.default_rng(0)
    for _ in range(20):
        n = int(rng.integers(2, 12))
        V = list(rng.uniform(1e-6, 10, n))
        C = list(rng.uniform(1, 1000, n))
        eps2 = float(rng.uniform(1e-6, 1e-2))
        N = driver.optimal_n(V, C, eps2)
        assert abs(sum(v / x for v, x in zip(V, N)) - eps2) <= 1e-12 * eps2
        assert abs(sum(x * c for x, c in zip(N, C)) - driver.total_cost(V, C, eps2)) <= 1e-9 * driver.total_cost(V, C, eps2)
        # Lagrange optimality: any feasible perturbation costs more
        N2 = [x * (1 + 0.01 * rng.standard_normal()) for x in N]
        scale = sum(v / x for v, x in zip(V, N2)) / eps2
        N2 = [x * scale for x in N2]
        assert sum(x * c for x, c in zip(N2, C)) >= sum(x * c for x, c in zip(N, C)) * (1 - 1e-12)


def test_nested_saving_factor():
    """Sec. 2.2: if V^D/V~ << C~/C^D << 1 the nested cost is about max C~/C^D of the plain cost."""
    V = [1.0, 0.5, 0.25]
    C = [1.0, 2.0, 4.0]
    ratio = 0.1
    Vt, Ct = V, [c * ratio for c in C]
    Vd, Cd = [v * 1e-6 for v in V], [c * (1 + ratio) for c in C]
    plain = driver.total_cost(V, C, 1.0)
    nested = driver.total_cost(Vt + Vd, Ct + Cd, 1.0)
    assert abs(nested / plain - ratio) < 0.02


def test_bias_estimate():
    assert driver.bias_estimate([1.0, 0.5, 0.25]) == max(0.25, 0.5 / 2)
