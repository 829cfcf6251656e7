"""Product planner (Eq. 11, 13-25) against the oracle's planner and the
paper's printed numbers."""
import json
import os

import numpy as np
import pytest

from oracle import planner as ref
from paper_2507_19246_gb300 import planner as P

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


@pytest.mark.parametrize("K,M", [(1, 16), (3, 16), (5, 32), (64, 64)])
def test_parareal_model_matches_oracle(K, M):
    tf, tc = 3.3, 0.21
    assert P.parareal_time(K, M, tf, tc) == pytest.approx(ref.tau_para(K, M, tf, tc), rel=1e-14)
    assert P.parareal_effort(K, M, tf, tc) == pytest.approx(ref.effort_para(K, M, tf, tc), rel=1e-14)
    for k in range(1, K + 1):
        assert P.parareal_iteration_time(k, M, tf, tc) == pytest.approx(
            ref.tau_para_iter(k, M, tf, tc), rel=1e-14)
        assert P.parareal_iteration_effort(k, M, tf, tc) == pytest.approx(
            ref.effort_para_iter(k, M, tf, tc), rel=1e-14)


@pytest.mark.parametrize("r,n", [(10, 16), (10, 180), (2, 32), (4, 1000)])
def test_bounds_match_oracle(r, n):
    assert P.iteration_bound(r, n) == ref.kappa(r, n)
    assert P.speedup_bound(r, 2) == pytest.approx(ref.speedup_inf(r, 2), rel=1e-15)


def test_paper_numbers():
    fe = GOLD["fe_example"]
    N, nc = fe["N_l"], fe["n_c"]
    C = P.exponential_costs(1.0, 10, 2)
    assert P.parareal_cores(nc, N[2], C[2], C[1]) == fe["n_c_para"]
    assert P.level_batches(N[0], C[0], 0.0, nc) == 58
    assert P.finite_core_speedup(N, 10, 2, nc) == pytest.approx(ref.speedup_nc(N, 10, 2, nc), rel=1e-14)
    assert P.effort_ratio(N, C, 2, 16) == pytest.approx(ref.effort_increase_inf(N, C, 2, 16), rel=1e-14)


def test_allocation_meets_the_target_and_follows_eq11():
    V = np.array([167.0, 2.5e-4, 8.8e-5, 4.1e-5])
    C = np.array([256.0, 768.0, 1536.0, 3072.0])
    eps = 0.05
    N = P.allocate_samples(V, C, eps)
    assert np.sum(V / N) <= eps ** 2 * (1 + 1e-12)
    # N_l proportional to sqrt(V_l / C_l) up to the rounding up
    ratio = N / np.sqrt(V / C)
    assert ratio.max() / ratio.min() < 1.0 + 1.0 / N.min() + 1e-9 or N.min() == 2
    # halving eps quadruples the samples
    N2 = P.allocate_samples(V, C, eps / 2)
    assert np.all(N2 >= 4 * N - 4)
