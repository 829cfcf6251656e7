"""Adaptive MLMC (pilot variances -> Eq. 11 sample counts) on the GPU, checked
against the oracle's estimator on exactly the samples the run used."""
import numpy as np
import pytest

from oracle import mlmc, stepper
from workloads import configs, meshes, params

pytestmark = pytest.mark.gpu


def test_adaptive_mlmc_matches_oracle_on_its_samples():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from paper_2507_19246_gb300 import mqs, planner

    mesh = meshes.annulus("5k")
    base = 32
    dts = [configs.level_dt(l, base) for l in range(3)]
    T = configs.PERIOD

    def sampler(level, first, n):
        return params.annulus_samples(n, level, seed=77, first=first)

    with mqs.Context(0) as ctx:
        mid = ctx.upload_mesh(mesh)
        est, rmse, N, lv = planner.run_adaptive_mlmc(
            ctx, mid, sampler, dts, T, rmse_target=0.5, n_pilot=6,
            solver=mqs.MQS_SOLVER_BANDED, precision=mqs.MQS_FP64)
    assert len(N) == 3 and all(n >= 6 for n in N)
    assert N[0] > N[1]                      # the coarse level carries the variance
    pairs = []
    for l, n in enumerate(N):
        p = sampler(l, 0, n)
        qf, qc = [], []
        for s in range(n):
            a, c = mlmc.level_pair(mesh, p[s], l, lambda k: dts[k],
                                   lambda k: round(T / dts[k]), stepper.QOI_JOULE)
            qf.append(a)
            qc.append(c)
        pairs.append((qf, qc if l else None))
    ref = mlmc.mlmc_estimate(pairs)
    assert est == pytest.approx(ref["estimate"], rel=1e-9)
    assert rmse == pytest.approx(ref["rmse"], rel=1e-6)
    assert lv[:, 0].tolist() == [float(n) for n in N]


def test_adaptive_mlmc_with_parareal_on_the_finest_level():
    """The combined method of Sec. II-D: after the finest level (L = 2) is
    sized by Eq. 11, Eq. 25 gives each of its remaining samples
    floor(slots / (N_L (1 + C_{L-1}/C_L))) lane slots, and those samples run
    Parareal on the largest power-of-two slice count that fits (coarse
    propagator = level L-2).  The decision is returned; every level-2 sample
    is checked against the oracle (sequential pilot samples against the serial
    solve, Parareal samples against the oracle's Parareal with the batch's
    iteration count), and the estimate against the oracle's estimator.  The
    finest level's variance is small enough that Eq. 11 keeps it at the pilot
    size, so a lower bound of 10 samples gives it samples to plan for."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from oracle import fem, parareal
    from paper_2507_19246_gb300 import mqs, planner

    mesh = meshes.annulus("5k")
    base = 32
    dts = [configs.level_dt(l, base) for l in range(3)]
    T = configs.PERIOD
    steps = [round(T / dt) for dt in dts]

    def sampler(level, first, n):
        return params.annulus_samples(n, level, seed=91, first=first)

    plan = {}
    with mqs.Context(0) as ctx:
        slots = ctx.lane_slots()
        assert slots >= 152
        mid = ctx.upload_mesh(mesh)
        est, rmse, N, lv = planner.run_adaptive_mlmc(
            ctx, mid, sampler, dts, T, rmse_target=0.5, n_pilot=4, parareal=True,
            par_tol=1e-9, plan_out=plan, n_min_per_level=[0, 0, 10],
            solver=mqs.MQS_SOLVER_BANDED, precision=mqs.MQS_FP64)
    assert plan["slots"] == slots and plan["coarse_factor"] == 4
    n_par = N[2] - plan["first_parareal_sample"]
    assert n_par > 0 and plan["slices"] >= 2
    assert plan["n_c_para"] == int(np.floor(slots / (n_par * 1.5)))
    assert plan["slices"] == planner.plan_finest_level(n_par, steps[2], steps[1], slots, steps[2],
                                                       4)[1]
    assert plan["iters"] and all(k >= 1 for _, _, k in plan["iters"])
    pairs = []
    for l, n in enumerate(N):
        p = sampler(l, 0, n)
        qf, qc = [], []
        for s in range(n):
            if l == 2 and s >= plan["first_parareal_sample"]:
                K = [k for s0, m, k in plan["iters"] if s0 <= s < s0 + m][0]
                d = fem.Discretisation(mesh, p[s])
                ref = parareal.parareal_sample(d, dts[2], steps[2], plan["slices"], 4, 0.0,
                                               stepper.QOI_JOULE, max_iter=K)
                a = stepper.qoi_finish(stepper.QOI_JOULE, ref["qoi_raw"], steps[2], dts[2])
                c, _, _ = stepper.solve_sample(mesh, p[s], dts[1], steps[1], stepper.QOI_JOULE)
            else:
                a, c = mlmc.level_pair(mesh, p[s], l, lambda k: dts[k],
                                       lambda k: round(T / dts[k]), stepper.QOI_JOULE)
            qf.append(a)
            qc.append(c)
        pairs.append((qf, qc if l else None))
    ref = mlmc.mlmc_estimate(pairs)
    assert est == pytest.approx(ref["estimate"], rel=1e-9)
    assert rmse == pytest.approx(ref["rmse"], rel=1e-6)
    assert lv[:, 0].tolist() == [float(n) for n in N]
