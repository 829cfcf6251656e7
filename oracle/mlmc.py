"""Monte Carlo and Multi-Level Monte Carlo estimators (oracle), Sec. II-B.

Eq. 8:  E_MC[Q]   = (1/N) sum_k Q^(k)
Eq. 9:  E_MLMC[Q] = sum_{l=0}^{L} (1/N_l) sum_{k=1}^{N_l} [Q_l^(k,l) - Q_{l-1}^(k,l)],
        Q_{-1} = 0, both solves of a pair on the same sample xi^(k,l).

The level variance is the unbiased sample variance of Y = Q_l - Q_{l-1}
(two-pass, exactly rounded sums via math.fsum); the statistical RMSE of the
estimate is sqrt(sum_l V_l / N_l).
"""
from __future__ import annotations

import math

import numpy as np


def mc_estimate(Q) -> float:
    Q = [float(q) for q in Q]
    return math.fsum(Q) / len(Q)


def level_moments(Y):
    """(N, mean, unbiased variance) of one level's differences."""
    Y = [float(y) for y in Y]
    n = len(Y)
    mean = math.fsum(Y) / n
    var = math.fsum((y - mean) ** 2 for y in Y) / (n - 1) if n > 1 else 0.0
    return n, mean, var


def mlmc_estimate(pairs):
    """pairs[l] = (Q_l samples, Q_{l-1} samples); level 0's second entry is ignored.

    Returns dict(estimate, rmse, levels=[(N_l, mean_l, var_l)]).
    """
    levels = []
    for l, (q_fine, q_coarse) in enumerate(pairs):
        q_fine = np.asarray(q_fine, dtype=np.float64)
        y = q_fine if l == 0 else q_fine - np.asarray(q_coarse, dtype=np.float64)
        levels.append(level_moments(y))
    estimate = math.fsum(m for _, m, _ in levels)
    rmse = math.sqrt(math.fsum(v / n for n, _, v in levels))
    return dict(estimate=estimate, rmse=rmse, levels=levels)


def level_pair(mesh, params, level: int, dt_of_level, steps_of_level, qoi: int,
               freq_hz: float = 50.0):
    """(Q_l, Q_{l-1}) for one sample: both solves use the same parameters."""
    from .stepper import solve_sample
    qf, _, _ = solve_sample(mesh, params, dt_of_level(level), steps_of_level(level), qoi,
                            freq_hz=freq_hz)
    if level == 0:
        return qf, 0.0
    qc, _, _ = solve_sample(mesh, params, dt_of_level(level - 1), steps_of_level(level - 1),
                            qoi, freq_hz=freq_hz)
    return qf, qc
