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
