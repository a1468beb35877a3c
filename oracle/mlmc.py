"""Monte Carlo and multilevel Monte Carlo estimators in FP64 (Sections 4 and 7).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``mc_estimate``: Q_hat = (1/N) sum Q_j (Eq. MC_estimator).
* ``level_stats``: Y_hat and the paper's sample variance
  s^2 = (1/N) sum Y^2 - Y_hat^2 (Eq. sample_variance); the unbiased N/(N-1)
  form is returned beside it.
* ``allocation``: N_l = floor(eps_s^-2 (sum_k sqrt(V_k C_k)) sqrt(V_l / C_l))
  (Eq. sample_allocation). Reading: floor. Pinned by the paper's two sample
  allocation tables (every entry at eps_s = 50 and 100 N follows from the
  eps_s = 10 N row by floor, none by ceiling or rounding).
* ``mc_samples``: N = floor(V / eps_s^2) (Eq. MC_num_samples).
* ``mlmc_estimate``: Q_hat^ML = sum_l Y_hat_l (Eq. MLMC_estimator) and its
  variance sum_l V_l / N_l (Eq. MLMC_error).
* ``bias``: |Y_hat_L| / (r m^alpha - 1) with r = 1 (Eq. bias_error); m is the
  ratio of degrees of freedom between levels.
* ``cost_exponent``: 2 + max(0, (gamma - beta)/alpha) (Eq.
  MLMC_computational_cost); plain MC: 2 + gamma/alpha. Pinned by the printed
  exponents 2.35 / 3.89 and 2.94 / 4.97 (Section 6).
* ``fit_rate``: least-squares slope of log|y| against log M (the alpha, beta,
  gamma fits of Section 6).
* ``ml_inverse_cdf``: F_L^-1(u) = R_0^[N_0 u] + sum_l (R_l^[N_l u] - R~_{l-1}^[N_l u]),
  where R~_{l-1} are the coarse members of the level-l pairs (Section 7).
  Reading: the index [N u] is ceil(N u), 1-based, clamped to [1, N]; the
  printed N_{l-1} on the coarse term is read as N_l (with N_{l-1} the sum
  would telescope to the finest level alone).
* ``adaptive``: Algorithm MLMC (warm-up N* samples on each new level,
  re-allocate, bias test, add a level).
"""
from __future__ import annotations

import math

import numpy as np


def mc_estimate(Q) -> float:
    Q = np.asarray(Q, np.float64)
    return float(Q.sum() / Q.size)


def level_stats(Y):
    Y = np.asarray(Y, np.float64)
    N = Y.size
    mean = Y.sum() / N
    var_b = (Y * Y).sum() / N - mean * mean
    var_u = var_b * N / (N - 1) if N > 1 else 0.0
    return float(mean), float(var_b), float(var_u)


def allocation(V, C, eps_s: float):
    V = np.asarray(V, np.float64)
    C = np.asarray(C, np.float64)
    S = np.sqrt(V * C).sum()
    return np.floor(S * np.sqrt(V / C) / (eps_s * eps_s)).astype(np.int64)


def mc_samples(V: float, eps_s: float) -> int:
    return int(math.floor(V / (eps_s * eps_s)))


def mlmc_estimate(Yhat, V, N):
    Yhat = np.asarray(Yhat, np.float64)
    V = np.asarray(V, np.float64)
    N = np.asarray(N, np.float64)
    return float(Yhat.sum()), float((V / N).sum())


def bias(Yhat_L: float, m_dof: float, alpha: float, r: float = 1.0) -> float:
    return abs(Yhat_L) / (r * m_dof ** alpha - 1.0)


def cost_exponent(alpha: float, beta: float, gamma: float) -> float:
    return 2.0 + max(0.0, (gamma - beta) / alpha)


def mc_cost_exponent(alpha: float, gamma: float) -> float:
    return 2.0 + gamma / alpha


def fit_rate(M, y) -> float:
    """Slope p of |y| ~ M^p by least squares in log-log space."""
    x = np.log(np.asarray(M, np.float64))
    z = np.log(np.abs(np.asarray(y, np.float64)))
    A = np.stack([x, np.ones_like(x)], 1)
    p, _ = np.linalg.lstsq(A, z, rcond=None)[0]
    return float(p)


def _order_stat(x_sorted, u):
    N = x_sorted.size
    idx = min(max(int(math.ceil(N * u)), 1), N)
    return x_sorted[idx - 1]


def ml_inverse_cdf(levels, u):
    """levels[0] = Q_0 samples; levels[l>0] = (Q_l fine, Q_{l-1} coarse) pair arrays."""
    q0 = np.sort(np.asarray(levels[0], np.float64))
    out = _order_stat(q0, u)
    for fine, coarse in levels[1:]:
        f = np.sort(np.asarray(fine, np.float64))
        c = np.sort(np.asarray(coarse, np.float64))
        out += _order_stat(f, u) - _order_stat(c, u)
    return float(out)


def ml_cdf(levels, x, n_u: int = 1000):
    """F(x) = (1/n) sum 1{X_i <= x} over X_i = F_L^-1(u_i), u_i = (i - 1/2)/n."""
    X = np.array([ml_inverse_cdf(levels, (i + 0.5) / n_u) for i in range(n_u)])
    x = np.atleast_1d(np.asarray(x, np.float64))
    return (X[None, :] <= x[:, None]).mean(axis=1)


def adaptive(sampler, eps_s: float, eps_b: float, m_dof: float, alpha: float,
             n_star: int = 100, L_max: int = 4):
    """Algorithm MLMC. ``sampler(l, n)`` returns (Y [n], cost per sample)."""
    Ys, C = [], []
    L = 0
    while True:
        y, c = sampler(L, n_star)
        Ys.append(np.asarray(y, np.float64))
        C.append(float(c))
        V = [level_stats(y)[1] for y in Ys]
        N_hat = allocation(V, C, eps_s)
        for l in range(L + 1):
            extra = int(N_hat[l]) - Ys[l].size
            if extra > 0:
                y, _ = sampler(l, extra)
                Ys[l] = np.concatenate([Ys[l], np.asarray(y, np.float64)])
        Yhat = [level_stats(y)[0] for y in Ys]
        eb = bias(Yhat[L], m_dof, alpha)
        if eb < eps_b or L >= L_max:
            break
        L += 1
    stats = [level_stats(y) for y in Ys]
    return dict(L=L, N=[y.size for y in Ys], Yhat=[s[0] for s in stats],
                V=[s[1] for s in stats], Q=float(sum(s[0] for s in stats)), bias=eb)
