"""Pins of the oracle's MC / MLMC estimators (Section 4) against the paper's
printed tables and exponents and closed forms."""
import os

import numpy as np
import pytest

from oracle import mlmc

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _tables():
    rows = {}
    for line in open(os.path.join(GOLD, "mlmc_allocation_tables.txt")):
        if line.startswith("#") or not line.strip():
            continue
        p = line.split()
        rows[(p[0], float(p[1]))] = [int(x) for x in p[2:]]
    return rows


@pytest.mark.parametrize("problem", ["type2", "type1"])
def test_allocation_tables_floor(problem):
    """Tables of Sections 6.2/6.3: V_l, C_l chosen so that Eq. sample_allocation
    gives N_l(10 N) + 1/2 at eps_s = 10 N; floor then reproduces the printed rows
    at 50 and 100 N, ceil and rounding do not."""
    t = _tables()
    n10 = np.array(t[(problem, 10.0)][:5], np.float64)
    C = 4.0 ** np.arange(5)               # gamma = 1, M_l = 4^l M_0
    target = n10 + 0.5
    eps = 10.0
    V = target ** 2 * C * eps ** 2 / (target * C).sum()
    assert np.array_equal(mlmc.allocation(V, C, 10.0), n10.astype(np.int64))
    for e in (50.0, 100.0):
        got = mlmc.allocation(V, C, e)
        assert list(got) == t[(problem, e)][:5]
        exact = mlmc.allocation(V, C, e).astype(float)
        ceil = np.ceil(target * (10.0 / e) ** 2)
        assert not np.array_equal(ceil, t[(problem, e)][:5])
    # standard MC: N = floor(V[Q_L]/eps^2)
    nmc10 = t[(problem, 10.0)][5]
    Vmc = (nmc10 + 0.5) * 100.0
    for e in (50.0, 100.0):
        assert mlmc.mc_samples(Vmc, e) == t[(problem, e)][5]


def test_cost_exponents():
    for line in open(os.path.join(GOLD, "mlmc_rates.txt")):
        if line.startswith("#") or not line.strip():
            continue
        _, a, b, g, e_ml, e_mc = line.split()
        a, b, g, e_ml, e_mc = map(float, (a, b, g, e_ml, e_mc))
        assert round(mlmc.cost_exponent(a, b, g), 2) == e_ml
        assert round(mlmc.mc_cost_exponent(a, g), 2) == e_mc


def test_allocation_meets_sampling_tolerance_at_min_cost():
    """Eq. sample_allocation (before flooring) satisfies sum V/N = eps^2 and is
    the Lagrange minimiser of sum N C: perturbations that keep the constraint cost more."""
    V = np.array([4.0, 1.0, 0.3, 0.05])
    C = np.array([1.0, 4.0, 16.0, 64.0])
    eps = 0.01
    S = np.sqrt(V * C).sum()
    N = S * np.sqrt(V / C) / eps ** 2
    assert abs((V / N).sum() - eps ** 2) < 1e-12 * eps ** 2
    cost = (N * C).sum()
    assert abs(cost - S ** 2 / eps ** 2) < 1e-9 * cost
    rng = np.random.default_rng(1)
    for _ in range(20):
        p = N * np.exp(0.1 * rng.standard_normal(4))
        p *= (V / p).sum() / eps ** 2       # rescale onto the constraint
        assert (p * C).sum() >= cost * (1 - 1e-12)


def test_estimators_and_variance():
    y = np.array([1.0, 2.0, 4.0, 7.0])
    mean, vb, vu = mlmc.level_stats(y)
    assert mean == 3.5 and abs(vb - np.var(y)) < 1e-15 and abs(vu - np.var(y, ddof=1)) < 1e-14
    q, v = mlmc.mlmc_estimate([10.0, -1.0, 0.25], [4.0, 1.0, 0.5], [100, 10, 5])
    assert q == 9.25 and abs(v - (0.04 + 0.1 + 0.1)) < 1e-15
    assert abs(mlmc.bias(0.2, 4.0, 0.5) - 0.2) < 1e-15     # 1/(4^0.5 - 1) = 1


def test_fit_rate_recovers_exponent():
    M = 350.0 * 4.0 ** np.arange(5)
    y = 3.0 * M ** -0.528
    assert abs(mlmc.fit_rate(M, y) + 0.528) < 1e-12


def test_multilevel_inverse_cdf():
    rng = np.random.default_rng(2)
    q0 = rng.standard_normal(1000)
    # one level: the empirical quantile with index ceil(N u)
    assert mlmc.ml_inverse_cdf([q0], 0.5) == np.sort(q0)[499]
    # a level whose fine and coarse members coincide adds nothing
    f = rng.standard_normal(50)
    assert mlmc.ml_inverse_cdf([q0, (f, f)], 0.3) == mlmc.ml_inverse_cdf([q0], 0.3)
    # a constant shift on the fine members shifts every quantile
    assert abs(mlmc.ml_inverse_cdf([q0, (f + 2.0, f)], 0.7) - (mlmc.ml_inverse_cdf([q0], 0.7) + 2.0)) < 1e-12
    F = mlmc.ml_cdf([q0], [0.0], n_u=2000)
    assert abs(F[0] - 0.5) < 0.05


def test_adaptive_algorithm_adds_levels():
    """Algorithm MLMC on a synthetic hierarchy: Y_l has mean 2^-l, variance 4^-l."""
    rng = np.random.default_rng(4)

    def sampler(l, n):
        return 2.0 ** -l + 2.0 ** -l * rng.standard_normal(n), 4.0 ** l

    out = mlmc.adaptive(sampler, eps_s=0.02, eps_b=0.1, m_dof=4.0, alpha=0.5, n_star=100, L_max=6)
    assert out["L"] >= 2
    assert all(n >= 100 for n in out["N"])
    assert abs(out["Q"] - sum(2.0 ** -l for l in range(out["L"] + 1))) < 0.1
