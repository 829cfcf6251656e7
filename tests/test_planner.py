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


def test_figure_curves_tend_to_the_unlimited_core_limits():
    """Fig. 1-2 of Sec. II-D from the model (r = 10, L = 2, V_l ~ 10^-2l, N_l
    by Eq. 11).  With unlimited cores every level is one batch and the
    Parareal time K/M (r^L + (M - (K+1)/2) r^{L-2}) tends to K r^{L-2}; with
    K = r that is C_{L-1} and the speedup tends to Eq. 21's bound.  The effort
    ratio tends to (sum_{l<L} N_l C_l + N_L K (C_L + C_{L-2})) / sum N_l C_l
    (Eq. 16 with M -> infinity)."""
    r, L = 10, 2
    V = [10.0 ** (-2 * l) for l in range(L + 1)]
    C = P.exponential_costs(1.0, r, L)
    N = [int(n) for n in P.allocate_samples(V, C, 1e-2)]
    big = 10 ** 12
    curves = P.figure_curves(N, r, [1, 2, r], [180, 10 ** 4, big])
    s_big = curves[r][0][-1]
    assert s_big == pytest.approx(P.speedup_bound(r, L), rel=1e-6)
    for K in (1, 2, r):
        eps_lim = (sum(n * c for n, c in zip(N[:-1], C[:-1])) + N[-1] * K * (C[L] + C[L - 2])) \
            / sum(n * c for n, c in zip(N, C))
        assert curves[K][1][-1] == pytest.approx(eps_lim, rel=1e-6)
        # more iterations cost more effort at every core count
    for i in range(3):
        e = [curves[K][1][i] for K in (1, 2, r) if curves[K][1][i] is not None]
        assert e == sorted(e)
    # too few cores for two slices per finest-level sample: no point on the curve
    tiny = P.figure_curves(N, r, [2], [N[-1]])
    assert tiny[2] == ([None], [None])


def test_plan_finest_level_follows_eq25():
    # 608 lane slots, 8 finest samples, C_{L-1}/C_L = 1/2: floor(608 / 12) = 50
    # slots each; 128 steps with coarse factor 4 allow 32 slices of one coarse step
    assert P.plan_finest_level(8, 128.0, 64.0, 608, 128, 4) == (50, 32)
    # many samples: fewer than two slots each -> sequential
    assert P.plan_finest_level(500, 128.0, 64.0, 608, 128, 4) == (0, 1)
    # the slice count must divide the steps in whole coarse steps
    assert P.plan_finest_level(2, 128.0, 64.0, 608, 96, 4) == (202, 8)
    assert P.plan_finest_level(2, 128.0, 64.0, 608, 4096, 64, max_slices=64) == (202, 64)
