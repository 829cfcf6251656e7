"""Pins for the oracle's MC / MLMC estimators (Eq. 8-9)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import mlmc, stepper
from workloads import configs, meshes, params


def test_moments_match_exact_rational_arithmetic():
    rng = np.random.default_rng(5)
    y = 1e3 + rng.normal(size=257) * 1e-4          # large mean, tiny spread
    n, mean, var = mlmc.level_moments(y)
    fy = [Fraction(v) for v in y]
    fm = sum(fy) / len(fy)
    fv = sum((v - fm) ** 2 for v in fy) / (len(fy) - 1)
    assert n == 257
    assert mean == pytest.approx(float(fm), rel=1e-15)
    assert var == pytest.approx(float(fv), rel=1e-9)


def test_single_level_is_plain_monte_carlo():
    q = np.random.default_rng(3).random(100)
    est = mlmc.mlmc_estimate([(q, None)])
    assert est["estimate"] == pytest.approx(mlmc.mc_estimate(q), rel=1e-15)
    assert est["rmse"] == pytest.approx(math.sqrt(np.var(q, ddof=1) / 100), rel=1e-12)


def test_telescoping_identity_on_common_samples():
    """With every level evaluated on the same samples the MLMC sum of level
    means equals the plain mean of the finest level (Eq. 9 telescopes)."""
    m = meshes.unit_square(8)
    ps = params.square_samples(6, seed=11)
    L = 2
    Q = np.zeros((L + 1, len(ps)))
    for l in range(L + 1):
        for k, p in enumerate(ps):
            Q[l, k], _, _ = stepper.solve_sample(m, p, configs.level_dt(l, base=16),
                                                 configs.level_steps(1, l, base=16),
                                                 stepper.QOI_ENERGY)
    pairs = [(Q[0], None)] + [(Q[l], Q[l - 1]) for l in range(1, L + 1)]
    est = mlmc.mlmc_estimate(pairs)
    assert est["estimate"] == pytest.approx(Q[L].mean(), rel=1e-13)
    # level differences shrink with dt (first-order scheme): |Y_2| < |Y_1|
    assert abs(est["levels"][2][1]) < abs(est["levels"][1][1])


def test_level_pair_uses_the_same_sample():
    m = meshes.unit_square(8)
    p = params.square_samples(1, seed=4)[0]
    qf, qc = mlmc.level_pair(m, p, 1, lambda l: configs.level_dt(l, base=16),
                             lambda l: configs.level_steps(1, l, base=16), stepper.QOI_JOULE)
    q0, _, _ = stepper.solve_sample(m, p, configs.level_dt(0, base=16), 16, stepper.QOI_JOULE)
    assert qc == q0 and qf != qc
