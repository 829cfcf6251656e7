"""MLMC + Parareal scheduling: the paper's cost model and sample allocation.

Host-side planning around the GPU path (Sec. II-B to II-D):

* ``allocate_samples`` -- Eq. 11, N_l proportional to sqrt(V_l / C_l),
  scaled so that the statistical error sqrt(sum_l V_l / N_l) meets a target
  (the standard Lagrange-multiplier solution of that allocation problem).
* time/effort model of Parareal and of MLMC with and without Parareal on the
  finest level: Eq. 13-19, the exponential cost law Eq. 20, the unlimited-
  core speedup bound Eq. 21, the iteration bound kappa under Eq. 22, the
  effort ratio Eq. 23, batching Eq. 24 and the cores per Parareal sample
  Eq. 25, and the finite-core speedup s_nc.
* ``run_adaptive_mlmc`` -- levels treated sequentially as the paper
  prescribes: pilot samples estimate V_l, Eq. 11 sizes each level, the
  remaining samples run, and the estimator of Eq. 9 is read out; with
  parareal=True the finest level runs Parareal on as many slices as Eq. 25
  gives each of its samples from the GPU's lane slots.
* ``figure_curves`` -- the speedup and effort curves of Fig. 1-2 from the
  model (finite cores, one curve per iteration count).

On one GPU the "cores" of the model are the lane slots the library runs at
once; the model is unit-free, so costs may be seconds or solve-steps.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------- Eq. 11
def allocate_samples(V, C, rmse_target, n_min=2):
    """N_l = ceil(eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k)) (Eq. 11's
    proportionality with the constant that makes sum_l V_l / N_l = eps^2)."""
    V = np.asarray(V, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    if rmse_target <= 0.0:
        raise ValueError("rmse_target must be positive")
    total = float(np.sum(np.sqrt(V * C)))
    N = np.ceil(np.sqrt(V / C) * total / rmse_target ** 2)
    return np.maximum(N, n_min).astype(np.int64)


# ---------------------------------------------------------------- Eq. 13-16
def parareal_iteration_time(k, M, tau_f, tau_c):
    """Eq. 13: fine run of one slice plus the coarse sweep over M - k slices."""
    return tau_f / M + (M - k) * tau_c / M


def parareal_iteration_effort(k, M, tau_f, tau_c):
    """Eq. 14: M - k + 1 fine slices and M - k coarse slices."""
    return (M - k + 1) * tau_f / M + (M - k) * tau_c / M


def parareal_time(K, M, tau_f, tau_c):
    """Eq. 15, the sum of Eq. 13 over k = 1..K."""
    return K * (tau_f + (M - 0.5 * (K + 1)) * tau_c) / M


def parareal_effort(K, M, tau_f, tau_c):
    """Eq. 16, the sum of Eq. 14 over k = 1..K."""
    return K * ((M - 0.5 * (K + 1)) * (tau_f + tau_c) + tau_f) / M


# ---------------------------------------------------------------- Eq. 17-25
def mlmc_time_unlimited(C):
    """Eq. 17 (time): every level's samples at once, levels one after another."""
    return float(sum(C))


def mlmc_effort(N, C):
    """Eq. 17 (effort)."""
    return float(sum(n * c for n, c in zip(N, C)))


def combined_time_unlimited(C, tau_para):
    """Eq. 18: levels below L as in MLMC, level L by Parareal."""
    return float(sum(C[:-1])) + tau_para


def combined_effort(N, C, effort_para):
    """Eq. 19."""
    return float(sum(n * c for n, c in zip(N[:-1], C[:-1]))) + N[-1] * effort_para


def exponential_costs(c0, r, L):
    """Eq. 20 for l = 0..L."""
    return [c0 * float(r) ** l for l in range(L + 1)]


def speedup_bound(r, L):
    """Eq. 21: best speedup of the combined method with unlimited cores."""
    return (float(r) ** (L + 1) - 1.0) / (2.0 * float(r) ** L - float(r) ** (L - 1) - 1.0)


def iteration_bound(r, n_para):
    """kappa (under Eq. 22): the largest K with tau_para <= C_{L-1} when the
    fine and coarse propagators cost C_L and C_{L-2}; smaller root of
    K^2 - (2 r^2 + 2 n - 1) K + 2 n r = 0."""
    a = 2.0 * r * r + 2.0 * n_para - 1.0
    return int(math.floor(0.5 * (a - math.sqrt(a * a - 8.0 * n_para * r))))


def effort_ratio(N, C, K, M):
    """Eq. 23: effort of the combined method over plain MLMC (coarse
    propagator = level L-2)."""
    e_para = parareal_effort(K, M, C[-1], C[-3])
    return combined_effort(N, C, e_para) / mlmc_effort(N, C)


def level_batches(N_l, C_l, C_prev, n_cores):
    """Eq. 24: batches of level l when its two solves per sample share n_cores."""
    return int(math.ceil(N_l * (1.0 + C_prev / C_l) / n_cores))


def parareal_cores(n_cores, N_L, C_L, C_prev):
    """Eq. 25: cores (lane slots) per finest-level sample for Parareal."""
    return int(math.floor(n_cores / (N_L * (1.0 + C_prev / C_L))))


def finite_core_speedup(N, r, K, n_cores):
    """s_nc (after Eq. 25), costs in units of C_0 with one Parareal batch."""
    L = len(N) - 1
    C = exponential_costs(1.0, r, L)
    b = [level_batches(N[l], C[l], C[l - 1] if l else 0.0, n_cores) for l in range(L + 1)]
    m = parareal_cores(n_cores, N[L], C[L], C[L - 1])
    num = sum(bl * cl for bl, cl in zip(b, C))
    den = sum(bl * cl for bl, cl in zip(b[:-1], C[:-1])) + \
        K / m * (float(r) ** L + (m - 0.5 * (K + 1)) * float(r) ** (L - 2))
    return num / den


def finite_core_effort_ratio(N, r, K, n_cores):
    """Effort increase of the combined method with n_cores cores (the model
    behind Fig. 2): the finest level's N_L samples each run Parareal on
    n_c,para = Eq. 25 slices with fine cost C_L and coarse cost C_{L-2}
    (Eq. 16 with M = n_c,para), the other levels as in plain MLMC; divided by
    the plain MLMC effort sum_l N_l C_l.  Costs in units of C_0 (Eq. 20)."""
    L = len(N) - 1
    C = exponential_costs(1.0, r, L)
    m = parareal_cores(n_cores, N[L], C[L], C[L - 1])
    e_para = parareal_effort(K, m, C[L], C[L - 2])
    return combined_effort(N, C, e_para) / mlmc_effort(N, C)


def figure_curves(N, r, K_values, core_counts):
    """Speedup (Fig. 1) and effort increase (Fig. 2) of the combined method
    against the number of cores, one curve per iteration count K: returns
    {K: (s_nc list, effort-ratio list)} over core_counts (counts that leave
    fewer than two cores per finest-level sample are skipped: None)."""
    L = len(N) - 1
    C = exponential_costs(1.0, r, L)
    out = {}
    for K in K_values:
        s, e = [], []
        for nc in core_counts:
            m = parareal_cores(nc, N[L], C[L], C[L - 1])
            ok = m >= max(2, K)
            s.append(finite_core_speedup(N, r, K, nc) if ok else None)
            e.append(finite_core_effort_ratio(N, r, K, nc) if ok else None)
        out[K] = (s, e)
    return out


def plan_finest_level(N_L, C_L, C_prev, slots, n_steps, coarse_factor, max_slices=64):
    """Parareal on the finest level (Sec. II-D): Eq. 25 gives the lane slots
    per sample, n = floor(slots / (N_L (1 + C_{L-1}/C_L))).  The slice count
    is the largest power of two M <= min(n, max_slices) whose slices hold a
    whole number of coarse steps (n_steps divisible by M * coarse_factor).
    Returns (n, M); M = 1 means the level runs sequentially."""
    n = parareal_cores(slots, N_L, C_L, C_prev) if N_L > 0 else 0
    M = 1
    while 2 * M <= min(n, max_slices) and n_steps % (2 * M * coarse_factor) == 0:
        M *= 2
    return n, (M if M >= 2 else 1)


# ---------------------------------------------------------------- adaptive MLMC
def run_adaptive_mlmc(ctx, mesh_id, sampler, dts, t_end, rmse_target, n_pilot=16,
                      qoi_kind=1, solver=None, chunk=1024, max_per_level=1 << 20,
                      parareal=False, par_tol=1e-8, lane_slots=None, plan_out=None,
                      n_min_per_level=None, **prop):
    """Sequential-level MLMC with run-time variance estimates (Sec. II-B).

    sampler(level, first, n) -> [n, n_params] parameters of samples
    first..first+n-1 of `level`; dts[l] the step of level l.  Each level first
    runs n_pilot samples, Eq. 11 (with the pilot variances of the levels run
    so far and C_l proportional to the step count) sets its size, and the
    remaining samples run.

    parareal=True applies the combined method of Sec. II-D: once the finest
    level L >= 2 is sized, plan_finest_level decides from the library's lane
    slots (mqs_lane_slots, the "cores" of Eq. 24-25, or `lane_slots`) how many
    slices each of its remaining samples gets; with two or more they run
    Parareal (coarse propagator = level L-2, tolerance par_tol), else
    sequentially.  plan_out (a dict) receives the decision: slots, n_c,para,
    slices, the coarse factor and the Parareal iterations of each batch.
    n_min_per_level: optional lower bounds on N_l (e.g. to keep a minimum of
    finest-level samples for a bias estimate).

    Returns (estimate, rmse, N_l, levels [N, mean, var]).  All solves run
    through the library's C ABI.
    """
    L = len(dts)
    steps = [round(t_end / dt) for dt in dts]
    cost = [steps[l] + (steps[l - 1] if l else 0) for l in range(L)]
    ctx.mlmc_reset(L)
    done = [0] * L
    plan = {"slices": 1, "iters": []}

    def run(level, first, n, slices=1, cf=1):
        for s0 in range(first, first + n, chunk):
            m = min(chunk, first + n - s0)
            b = ctx.set_samples(mesh_id, sampler(level, s0, m))
            if solver is not None:
                ctx.set_solver(b, solver)
            ctx.set_time(b, 0.0, t_end, 50.0, qoi_kind)
            if slices > 1:
                k = ctx.propagate(b, level, dts[level], dt_prev=dts[level - 1] if level else 0.0,
                                  n_slices=slices, coarse_factor=cf, max_par_iters=slices,
                                  par_tol=par_tol, **prop)
                plan["iters"].append((s0, m, k))
            else:
                ctx.propagate(b, level, dts[level], dt_prev=dts[level - 1] if level else 0.0, **prop)
            ctx.mlmc_accumulate(b, level)
            ctx.free_batch(b)

    variances = []
    for l in range(L):
        run(l, 0, n_pilot)
        done[l] = n_pilot
        lv, _, _ = ctx.mlmc_readout()
        variances.append(max(float(lv[l, 2]), 1e-300))
        # size the levels seen so far; only this level can still grow
        N = allocate_samples(variances, cost[:l + 1], rmse_target, n_min=n_pilot)
        floor_l = n_min_per_level[l] if n_min_per_level is not None else 0
        target = int(min(max(N[l], n_pilot, floor_l), max_per_level))
        slices, cf = 1, 1
        if parareal and l == L - 1 and L >= 3 and target > done[l]:
            slots = lane_slots if lane_slots is not None else ctx.lane_slots(
                prop.get("precision", 0))
            cf = int(round(dts[l - 2] / dts[l]))
            n_para, slices = plan_finest_level(target - done[l], steps[l], steps[l - 1], slots,
                                               steps[l], cf)
            plan.update(slots=slots, n_c_para=n_para, slices=slices, coarse_factor=cf,
                        first_parareal_sample=done[l])
        if target > done[l]:
            run(l, done[l], target - done[l], slices, cf)
            done[l] = target
    if plan_out is not None:
        plan_out.update(plan)
    lv, est, rmse = ctx.mlmc_readout()
    return est, rmse, list(done), lv
