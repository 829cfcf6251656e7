"""Pins for the oracle's cost model (Eq. 13-25) against closed forms and the
numbers the paper prints."""
import json
import os

import pytest

from oracle import planner

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


@pytest.mark.parametrize("M,K", [(16, 3), (32, 5), (64, 64), (10, 1)])
def test_iteration_sums_give_eq15_and_eq16(M, K):
    tf, tc = 7.0, 0.3
    assert sum(planner.tau_para_iter(k, M, tf, tc) for k in range(1, K + 1)) == \
        pytest.approx(planner.tau_para(K, M, tf, tc), rel=1e-14)
    assert sum(planner.effort_para_iter(k, M, tf, tc) for k in range(1, K + 1)) == \
        pytest.approx(planner.effort_para(K, M, tf, tc), rel=1e-14)


def test_speedup_bound_fig1_setup():
    r, L = GOLD["fig1_setup"]["r"], GOLD["fig1_setup"]["L"]
    # Eq. 21's closed form equals its defining ratio of level costs
    C = [planner.level_cost(1.0, r, l) for l in range(L + 1)]
    ratio = sum(C) / (sum(C[:-1]) + C[L - 1])
    assert planner.speedup_inf(r, L) == pytest.approx(ratio, rel=1e-15)
    assert planner.speedup_inf(r, L) == pytest.approx(999.0 / 189.0, rel=1e-15)


@pytest.mark.parametrize("r,n", [(10, 16), (10, 180), (2, 32), (10, 10 ** 6)])
def test_kappa_is_the_largest_K_meeting_tau_para_le_C_Lminus1(r, n):
    L = 3
    C = [float(r) ** l for l in range(L + 1)]
    kap = planner.kappa(r, n)
    ok = [K for K in range(1, 10 * r) if planner.tau_para(K, n, C[L], C[L - 2]) <= C[L - 1] * (1 + 1e-12)]
    assert kap == (max(k for k in ok if k <= r) if ok else 0)
    assert kap <= r


def test_kappa_examples():
    assert planner.kappa(10, 16) == 1
    assert planner.kappa(10, 180) == 6
    # the smaller root tends to r from below as n grows: kappa <= r always
    assert planner.kappa(10, 10 ** 9) == 9
    assert planner.kappa(10, 10 ** 3) == 9 and planner.kappa(10, 100) == 5   # (399 - sqrt(151201))/2 = 5.08


def test_fe_example_numbers():
    fe = GOLD["fe_example"]
    N, dt, nc = fe["N_l"], fe["dt"], fe["n_c"]
    r = dt[0] / dt[1]
    assert r == pytest.approx(10.0)
    C = [r ** l for l in range(3)]
    # Eq. 25 with Table II's N_L and r = 10 reproduces the printed n_c,para = 16
    assert planner.cores_per_parareal_sample(nc, N[2], C[2], C[1]) == fe["n_c_para"]
    # Table II runtimes give the printed Parareal speedup 2.69
    rt = fe["runtime_s"]
    assert rt["seq_L2"] / rt["para_L2"] == pytest.approx(fe["parareal_speedup"], abs=0.005)
    # steps per level over T = 0.16 s
    assert [round(fe["T"] / d) for d in dt] == [80, 800, 8000]
    # Eq. 24: level 0 needs ceil(10303 / 180) batches
    assert planner.batches(N[0], C[0], 0.0, nc) == 58
    assert planner.batches(N[1], C[1], C[0], nc) == 1


def test_finite_core_speedup_limits():
    """With one batch per level and K = 1 on n_c,para -> infinity slices,
    tau_para -> C_{L-2} and s_nc -> sum_l C_l / (sum_{l<L} C_l + C_{L-2});
    with tau_para held at C_{L-1} instead, Eq. 21's ratio results."""
    s_big = planner.speedup_nc([100, 10, 1], 10, 1, 10 ** 7)
    assert s_big == pytest.approx(111.0 / 12.0, rel=1e-5)
    # few cores: level 0 needs many batches and the speedup collapses towards 1
    s_small = planner.speedup_nc([10303, 85, 10], 10, 2, 180)
    assert 1.0 < s_small < planner.speedup_inf(10, 2)


def test_effort_increase_is_one_without_finest_samples():
    """Eq. 18-19, 23: with N_L = 0 the combined and the plain MLMC effort are
    the same sum over the coarser levels, so eps_inf = 1 whatever K and M."""
    N, C = [40, 7, 0], [1.0, 10.0, 100.0]
    for K, M in ((1, 4), (3, 16), (16, 16)):
        assert planner.effort_increase_inf(N, C, K, M) == pytest.approx(1.0, rel=1e-15)


def test_effort_increase_is_one_for_one_iteration_and_free_coarse_propagator():
    """Eq. 16 with K = 1 and tau_C = 0 leaves E_para = (M-1)/M tau_F + tau_F/M
    = tau_F, the sequential cost: one fine sweep over all slices.  With
    tau_C = C_{L-2} = C_0 = 0, eps_inf = 1."""
    N, C = [5, 3, 2], [0.0, 7.0, 50.0]
    for M in (2, 8, 64):
        assert planner.effort_para(1, M, 50.0, 0.0) == pytest.approx(50.0, rel=1e-15)
        assert planner.effort_increase_inf(N, C, 1, M) == pytest.approx(1.0, rel=1e-15)


def test_effort_increase_worked_case():
    """r = 10, L = 2: C = (1, 10, 100), N = (100, 10, 2), K = 2, M = 16,
    tau_F = C_2 = 100, tau_C = C_0 = 1.  By hand, from Eq. 14 per iteration:
      k = 1: 16/16 * 100 + 15/16 * 1 = 100.9375
      k = 2: 15/16 * 100 + 14/16 * 1 =  94.625      -> E_para = 195.5625
    E_comb = 100*1 + 10*10 + 2*195.5625 = 591.125 (Eq. 19)
    E_ref  = 100*1 + 10*10 + 2*100      = 400     (Eq. 17)
    eps_inf = 591.125 / 400 = 4729/3200."""
    N, C = [100, 10, 2], [1.0, 10.0, 100.0]
    assert planner.effort_para(2, 16, 100.0, 1.0) == 195.5625
    assert planner.effort_comb_inf(N, C, 195.5625) == 591.125
    assert planner.effort_ref_inf(N, C) == 400.0
    assert planner.effort_increase_inf(N, C, 2, 16) == pytest.approx(4729.0 / 3200.0, rel=1e-15)


def test_combined_time_worked_case():
    """Eq. 15 and 18, by hand: C = (1, 10, 100), K = 1, M = 16:
    tau_para = 1/16 (100 + 15 * 1) = 7.1875 and tau_comb = 1 + 10 + 7.1875.
    K = M = 16: tau_para = 100 + 7.5 * 1 (the serial fine cost plus the
    coarse sweeps that Parareal adds when it does not converge early)."""
    C = [1.0, 10.0, 100.0]
    assert planner.tau_para(1, 16, 100.0, 1.0) == 7.1875
    assert planner.tau_comb_inf(C, 7.1875) == 18.1875
    assert planner.tau_para(16, 16, 100.0, 1.0) == 107.5
    assert planner.tau_ref_inf(C) == 111.0
