"""The 80k-node annulus (n = 78912, bandwidth 275) on the cluster stepping
kernels: each CTA holds only its own rows of the work vector and a ring of
recently solved rows, so a lane fits 4 or 8 CTAs of shared memory.  Level
pairs and Parareal against the oracle; the multi-wave shape of many lanes
bitwise against a lane alone."""
import numpy as np
import pytest

from oracle import fem, parareal, stepper
from workloads import configs, meshes, params

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2507_19246_gb300 import mqs
    mqs.load()
    return mqs, meshes.annulus("80k")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


def test_annulus80k_level_pair_and_bandwidth(setup):
    mqs, mesh = setup
    p = params.annulus_samples(2, 1, seed=81)
    dt1, dt0 = configs.level_dt(1), configs.level_dt(0)
    with mqs.Context(0) as ctx:
        mid = ctx.upload_mesh(mesh)
        assert ctx.mesh_info(mid)[0] == 78912
        assert ctx.mesh_bandwidth(mid) <= 280
        b = ctx.set_samples(mid, p)
        ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
        ctx.set_time(b, 0.0, 8 * dt1, 50.0, mqs.MQS_QOI_JOULE)
        ctx.propagate(b, 1, dt1, dt_prev=dt0)
        q, st = ctx.read_qoi(b)
        a, ac = ctx.read_state(b, 0), ctx.read_state(b, 1)
    assert not st.any()
    for s in range(2):
        qf, af, _ = stepper.solve_sample(mesh, p[s], dt1, 8, stepper.QOI_JOULE)
        qc, acc, _ = stepper.solve_sample(mesh, p[s], dt0, 4, stepper.QOI_JOULE)
        assert abs(q[s, 0] - qf) <= TOL * abs(qf) and abs(q[s, 1] - qc) <= TOL * abs(qc), s
        assert _rel(a[s], af) <= TOL and _rel(ac[s], acc) <= TOL, s


def test_annulus80k_parareal(setup):
    mqs, mesh = setup
    p = params.annulus_nominal(1)
    n_steps, M, cf, tol = 32, 8, 2, 1e-9
    dt = configs.level_dt(2)
    with mqs.Context(0) as ctx:
        mid = ctx.upload_mesh(mesh)
        b = ctx.set_samples(mid, p)
        ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
        ctx.set_time(b, 0.0, n_steps * dt, 50.0, mqs.MQS_QOI_JOULE)
        K = ctx.propagate(b, 0, dt, n_slices=M, coarse_factor=cf, max_par_iters=M, par_tol=tol)
        q, st = ctx.read_qoi(b)
        a = ctx.read_state(b, 0)
    assert not st.any()
    ref = parareal.parareal_sample(fem.Discretisation(mesh, p[0]), dt, n_steps, M, cf, 0.0,
                                   stepper.QOI_JOULE, max_iter=K)
    q_ref = stepper.qoi_finish(stepper.QOI_JOULE, ref["qoi_raw"], n_steps, dt)
    assert abs(q[0, 0] - q_ref) <= TOL * abs(q_ref)
    assert _rel(a[0], ref["a_end"]) <= TOL


def test_annulus80k_many_lanes_multiwave_is_bitwise_one_lane(setup, monkeypatch):
    """40 lanes (20 level pairs) exceed one wave of 4-CTA clusters (the
    narrowest split that fits); a lane's result is the same alone (forced to 4
    CTAs) as in the many-wave launch."""
    mqs, mesh = setup
    p = params.annulus_samples(20, 2, seed=82)
    dt1, dt0 = configs.level_dt(2), configs.level_dt(1)
    out = []
    with mqs.Context(0) as ctx:
        mid = ctx.upload_mesh(mesh)
        for pp, force in ((p, None), (p[7:8], "4")):
            if force:
                monkeypatch.setenv("MQS_DIRECT_CLUSTER", force)
            b = ctx.set_samples(mid, pp)
            ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
            ctx.set_time(b, 0.0, 4 * dt1, 50.0, mqs.MQS_QOI_JOULE)
            ctx.propagate(b, 2, dt1, dt_prev=dt0)
            q, st = ctx.read_qoi(b)
            assert not st.any()
            out.append((q.copy(), ctx.read_state(b, 0)))
    assert out[0][0][7, 0] == out[1][0][0, 0] and out[0][0][7, 1] == out[1][0][0, 1]
    assert np.array_equal(out[0][1][7], out[1][1][0])


def test_annulus80k_combined_mlmc_parareal_K_equals_M_is_sequential(setup):
    """The combined method (Sec. II-D) on the 80k annulus over a short
    horizon: three levels, the finest by Parareal with coarse propagator =
    level 0 (coarse factor 4) and its level-1 companion solve beside it; with
    tolerance 0 Parareal runs K = M iterations and reproduces the serial fine
    solve, so the MLMC estimate equals an all-sequential run of the same
    samples within 1e-10."""
    mqs, mesh = setup
    T = configs.PERIOD / 8
    dts = [configs.level_dt(l) for l in range(3)]
    N = [4, 2, 2]
    prm = [params.annulus_samples(N[l], l, seed=83) for l in range(3)]
    out = []
    with mqs.Context(0) as ctx:
        mid = ctx.upload_mesh(mesh)
        for parareal_on in (True, False):
            ctx.mlmc_reset(3)
            for l in range(3):
                b = ctx.set_samples(mid, prm[l])
                ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
                ctx.set_time(b, 0.0, T, 50.0, mqs.MQS_QOI_JOULE)
                kw = (dict(n_slices=8, coarse_factor=4, max_par_iters=8, par_tol=0.0)
                      if (parareal_on and l == 2) else {})
                K = ctx.propagate(b, l, dts[l], dt_prev=dts[l - 1] if l else 0.0, **kw)
                if kw:
                    assert K == 8
                q, st = ctx.read_qoi(b)
                assert not st.any()
                ctx.mlmc_accumulate(b, l)
                ctx.free_batch(b)
            out.append(ctx.mlmc_readout())
    (lv_p, est_p, rmse_p), (lv_s, est_s, rmse_s) = out
    assert abs(est_p - est_s) <= 1e-10 * abs(est_s)
    assert rmse_p == pytest.approx(rmse_s, rel=1e-8)
    assert np.allclose(lv_p[:, 1], lv_s[:, 1], rtol=1e-9, atol=1e-12 * abs(est_s))
