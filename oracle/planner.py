"""Time-to-solution and effort model of MLMC + Parareal (oracle), Sec. II-C/D.

Costs are in arbitrary units; tau_F, tau_C are the sequential costs of the
fine and coarse propagators over the whole interval, M the number of slices,
K the Parareal iterations, C_l the cost of one level-l solve, N_l the
samples of level l.
"""
from __future__ import annotations

import math


def tau_para_iter(k, M, tau_f, tau_c):
    """Eq. 13: time of Parareal iteration k."""
    return tau_f / M + (M - k) / M * tau_c


def effort_para_iter(k, M, tau_f, tau_c):
    """Eq. 14: effort of Parareal iteration k."""
    return (M - k + 1) / M * tau_f + (M - k) / M * tau_c


def tau_para(K, M, tau_f, tau_c):
    """Eq. 15: Parareal time-to-solution after K iterations."""
    return K / M * (tau_f + (M - (K + 1) / 2.0) * tau_c)


def effort_para(K, M, tau_f, tau_c):
    """Eq. 16: Parareal effort after K iterations."""
    return K / M * (M - (K + 1) / 2.0) * (tau_f + tau_c) + K / M * tau_f


def tau_ref_inf(C):
    """Eq. 17: MLMC time with unlimited cores, sum_l C_l."""
    return math.fsum(C)


def effort_ref_inf(N, C):
    """Eq. 17: MLMC effort, sum_l N_l C_l."""
    return math.fsum(n * c for n, c in zip(N, C))


def tau_comb_inf(C, tau_p):
    """Eq. 18: combined time, Parareal on the finest level."""
    return math.fsum(C[:-1]) + tau_p


def effort_comb_inf(N, C, effort_p):
    """Eq. 19: combined effort."""
    return math.fsum(n * c for n, c in zip(N[:-1], C[:-1])) + N[-1] * effort_p


def level_cost(c0, r, l):
    """Eq. 20: exponential cost model C_l = C_0 r^l."""
    return c0 * r ** l


def speedup_inf(r, L):
    """Eq. 21: best speedup with unlimited cores, (r^{L+1}-1)/(2 r^L - r^{L-1} - 1)."""
    return (r ** (L + 1) - 1) / (2 * r ** L - r ** (L - 1) - 1)


def kappa(r, n_para):
    """Largest K with tau_para <= C_{L-1} when tau_F = C_L, tau_C = C_{L-2}
    (the bound under Eq. 22): the floor of the smaller root of
    K^2 - (2 r^2 + 2 n - 1) K + 2 n r = 0."""
    a = 2.0 * r * r + 2.0 * n_para - 1.0
    return int(math.floor((a - math.sqrt(a * a - 8.0 * n_para * r)) / 2.0))


def effort_increase_inf(N, C, K, M):
    """Eq. 23: eps_inf = E_comb,inf / E_ref,inf with tau_F = C_L, tau_C = C_{L-2}."""
    e_p = effort_para(K, M, C[-1], C[-3])
    return effort_comb_inf(N, C, e_p) / effort_ref_inf(N, C)


def batches(N_l, C_l, C_prev, n_cores):
    """Eq. 24: b_l = ceil(N_l (1 + C_{l-1}/C_l) / n_c); C_prev = 0 on level 0."""
    return int(math.ceil(N_l * (1.0 + C_prev / C_l) / n_cores))


def cores_per_parareal_sample(n_cores, N_L, C_L, C_prev):
    """Eq. 25: n_c,para = floor(n_c / (N_L (1 + C_{L-1}/C_L)))."""
    return int(math.floor(n_cores / (N_L * (1.0 + C_prev / C_L))))


def speedup_nc(N, r, K, n_cores):
    """Finite-core speedup s_nc (unnumbered, after Eq. 25), in units of C_0.

    Levels l < L run in b_l batches of cost C_l = r^l; level L runs one batch
    of Parareal on n_c,para slices with tau_F = r^L, tau_C = r^{L-2}.
    """
    L = len(N) - 1
    C = [float(r) ** l for l in range(L + 1)]
    b = [batches(N[l], C[l], C[l - 1] if l else 0.0, n_cores) for l in range(L + 1)]
    ncp = cores_per_parareal_sample(n_cores, N[L], C[L], C[L - 1])
    num = math.fsum(bl * cl for bl, cl in zip(b, C))
    den = math.fsum(bl * cl for bl, cl in zip(b[:-1], C[:-1])) + \
        K / ncp * (r ** L + (ncp - (K + 1) / 2.0) * r ** (L - 2))
    return num / den
