"""The banded direct solver (band Cholesky in RCM order) against the oracle."""
import numpy as np
import pytest

from oracle import fem, parareal, stepper
from workloads import configs, meshes, params

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def mqs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2507_19246_gb300 import mqs as m
    m.load()
    return m


@pytest.fixture()
def ctx(mqs):
    c = mqs.Context(0)
    yield c
    c.close()


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


def test_bandwidth_is_reported(ctx):
    for name, lim in (("5k", 60), ("20k", 230)):
        mid = ctx.upload_mesh(meshes.annulus(name))
        bw = ctx.mesh_bandwidth(mid)
        assert 0 < bw <= lim


def test_banded_square_energy_full_config(ctx, mqs):
    cfg = configs.MC_SQUARE
    mesh = meshes.unit_square(16)
    p = params.square_samples(cfg.n_samples)
    dt = cfg.t_end / cfg.n_steps
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, cfg.t_end, 50.0, mqs.MQS_QOI_ENERGY)
    ctx.propagate(b, 0, dt)
    q, st = ctx.read_qoi(b)
    a = ctx.read_state(b, 0)
    assert not st.any()
    for s in range(cfg.n_samples):
        qo, ao, _ = stepper.solve_sample(mesh, p[s], dt, cfg.n_steps, stepper.QOI_ENERGY)
        assert abs(q[s, 0] - qo) <= TOL * abs(qo) and _rel(a[s], ao) <= TOL


@pytest.mark.parametrize("wide", ["1", "0"])
def test_banded_level_pair_ragged_annulus(ctx, mqs, monkeypatch, wide):
    # wide = 1: 1024-thread lane CTAs, work vector in shared memory;
    # wide = 0: 256-thread lane CTAs (4 per SM), work vector in global memory
    monkeypatch.setenv("MQS_DIRECT_WIDE", wide)
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(37, 1)
    dt1, dt0 = configs.level_dt(1), configs.level_dt(0)
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, configs.PERIOD, 50.0, mqs.MQS_QOI_JOULE)
    ctx.propagate(b, 1, dt1, dt_prev=dt0)
    q, st = ctx.read_qoi(b)
    a, ac = ctx.read_state(b, 0), ctx.read_state(b, 1)
    assert not st.any()
    for s in range(p.shape[0]):
        qf, af, _ = stepper.solve_sample(mesh, p[s], dt1, 128, stepper.QOI_JOULE)
        qc, acc, _ = stepper.solve_sample(mesh, p[s], dt0, 64, stepper.QOI_JOULE)
        assert abs(q[s, 0] - qf) <= TOL * abs(qf) and abs(q[s, 1] - qc) <= TOL * abs(qc), s
        assert _rel(a[s], af) <= TOL and _rel(ac[s], acc) <= TOL, s


def test_banded_parareal_matches_oracle_parareal(ctx, mqs):
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(2, 0, seed=8)
    n_steps, M, cf, tol = 256, 16, 4, 1e-8
    dt = configs.PERIOD / 128
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, n_steps * dt, 50.0, mqs.MQS_QOI_JOULE)
    K = ctx.propagate(b, 0, dt, n_slices=M, coarse_factor=cf, max_par_iters=M, par_tol=tol)
    q, st = ctx.read_qoi(b)
    a = ctx.read_state(b, 0)
    assert not st.any()
    # the oracle's jump norms after iterations 2 and 3 are 1.3e-7 / 1.0e-9
    # (sample 0) and 7.7e-8 / 4.5e-10 (sample 1): both samples stop at K = 3,
    # far from the tolerance 1e-8
    assert K == 3
    for s in range(2):
        d = fem.Discretisation(mesh, p[s])
        ref = parareal.parareal_sample(d, dt, n_steps, M, cf, tol, stepper.QOI_JOULE)
        assert ref["iters"] == K, s
        q_ref = stepper.qoi_finish(stepper.QOI_JOULE, ref["qoi_raw"], n_steps, dt)
        assert abs(q[s, 0] - q_ref) <= TOL * abs(q_ref), s
        assert _rel(a[s], ref["a_end"]) <= TOL, s


def test_banded_parareal_K_equals_M_is_serial(ctx, mqs):
    mesh = meshes.annulus("5k")
    p = params.annulus_nominal(1)
    n_steps, M, cf = 64, 8, 2
    dt = configs.PERIOD / 64
    mid = ctx.upload_mesh(mesh)
    q, a = [], []
    for slices in (M, 1):
        b = ctx.set_samples(mid, p)
        ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
        ctx.set_time(b, 0.0, n_steps * dt, 50.0, mqs.MQS_QOI_JOULE)
        ctx.propagate(b, 0, dt, n_slices=slices, coarse_factor=cf, max_par_iters=slices,
                      par_tol=0.0)
        q.append(ctx.read_qoi(b)[0][0, 0])
        a.append(ctx.read_state(b, 0)[0])
    # same kernel, same factor, same per-lane arithmetic: the state is exact, as in
    # the oracle; the QoI differs only by the order of the per-slice partial sums
    assert np.array_equal(a[0], a[1])
    assert q[0] == pytest.approx(q[1], rel=1e-14)


def test_banded_rejects_unknown_solver(ctx, mqs):
    mesh = meshes.unit_square(8)
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, params.square_samples(2))
    with pytest.raises(mqs.MQSError, match="unknown solver"):
        ctx.set_solver(b, 7)


@pytest.mark.parametrize("wide", ["1", "0"])
def test_banded_mixed_precision_qoi(ctx, mqs, monkeypatch, wide):
    """FP32 band factor with FP64 refinement: QoI within 1e-6 of the FP64 oracle."""
    monkeypatch.setenv("MQS_DIRECT_WIDE", wide)
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(8, 2)
    dt1, dt0 = configs.level_dt(1), configs.level_dt(0)
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, configs.PERIOD, 50.0, mqs.MQS_QOI_JOULE)
    ctx.propagate(b, 1, dt1, dt_prev=dt0, precision=mqs.MQS_MIXED, cg_tol=1e-10, cg_max_iters=20)
    q, st = ctx.read_qoi(b)
    a = ctx.read_state(b, 0)
    assert not st.any()
    for s in range(p.shape[0]):
        qf, af, _ = stepper.solve_sample(mesh, p[s], dt1, 128, stepper.QOI_JOULE)
        qc, _, _ = stepper.solve_sample(mesh, p[s], dt0, 64, stepper.QOI_JOULE)
        assert abs(q[s, 0] - qf) <= 1e-6 * abs(qf) and abs(q[s, 1] - qc) <= 1e-6 * abs(qc), s
        assert _rel(a[s], af) <= 1e-8, s


def test_banded_mixed_sweep_limit_is_reported(ctx, mqs):
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(2, 0)
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, configs.PERIOD, 50.0, mqs.MQS_QOI_JOULE)
    ctx.propagate(b, 0, configs.level_dt(0), precision=mqs.MQS_MIXED, cg_tol=1e-15,
                  cg_max_iters=1)
    _, st = ctx.read_qoi(b)
    assert (st & mqs.MQS_ST_NOTCONV).all()


def test_banded_mixed_parareal(ctx, mqs):
    mesh = meshes.annulus("5k")
    p = params.annulus_nominal(1)
    n_steps, M, cf, tol = 256, 16, 4, 1e-8
    dt = configs.PERIOD / 128
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, n_steps * dt, 50.0, mqs.MQS_QOI_JOULE)
    K = ctx.propagate(b, 0, dt, n_slices=M, coarse_factor=cf, max_par_iters=M, par_tol=tol,
                      precision=mqs.MQS_MIXED, cg_tol=1e-10, cg_max_iters=20)
    q, st = ctx.read_qoi(b)
    assert not st.any()
    d = fem.Discretisation(mesh, p[0])
    ref = parareal.parareal_sample(d, dt, n_steps, M, cf, tol, stepper.QOI_JOULE)
    q_ref = stepper.qoi_finish(stepper.QOI_JOULE, ref["qoi_raw"], n_steps, dt)
    assert abs(K - ref["iters"]) <= 1
    assert abs(q[0, 0] - q_ref) <= 1e-6 * abs(q_ref)


# ---------------------------------------------------------------- cluster-split stepping
# MQS_DIRECT_CLUSTER = 0 selects the one-CTA kernels; 1, 2, 4, 8 the stepping
# kernels whose block substitution is spread over warps and over a cluster of
# that many CTAs per lane.
CLUSTERS = ["0", "1", "2", "4", "8"]


@pytest.mark.parametrize("cluster", CLUSTERS)
def test_cluster_split_level_pair(ctx, mqs, monkeypatch, cluster):
    monkeypatch.setenv("MQS_DIRECT_WIDE", "1")
    monkeypatch.setenv("MQS_DIRECT_CLUSTER", cluster)
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(5, 2, seed=11)
    dt1, dt0 = configs.level_dt(2), configs.level_dt(1)
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, configs.PERIOD / 4, 50.0, mqs.MQS_QOI_JOULE)
    ctx.propagate(b, 2, dt1, dt_prev=dt0)
    q, st = ctx.read_qoi(b)
    a, ac = ctx.read_state(b, 0), ctx.read_state(b, 1)
    assert not st.any()
    for s in range(p.shape[0]):
        qf, af, _ = stepper.solve_sample(mesh, p[s], dt1, 64, stepper.QOI_JOULE)
        qc, acc, _ = stepper.solve_sample(mesh, p[s], dt0, 32, stepper.QOI_JOULE)
        assert abs(q[s, 0] - qf) <= TOL * abs(qf) and abs(q[s, 1] - qc) <= TOL * abs(qc), s
        assert _rel(a[s], af) <= TOL and _rel(ac[s], acc) <= TOL, s


@pytest.mark.parametrize("cluster", CLUSTERS)
def test_cluster_split_energy_ragged_small(ctx, mqs, monkeypatch, cluster):
    """n = 49 free unknowns: two 32-row blocks, the second ragged; energy QoI."""
    monkeypatch.setenv("MQS_DIRECT_WIDE", "1")
    monkeypatch.setenv("MQS_DIRECT_CLUSTER", cluster)
    mesh = meshes.unit_square(8)
    p = params.square_samples(3)
    dt = configs.PERIOD / 40
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, 13 * dt, 50.0, mqs.MQS_QOI_ENERGY)
    ctx.propagate(b, 0, dt)
    q, st = ctx.read_qoi(b)
    a = ctx.read_state(b, 0)
    assert not st.any()
    for s in range(3):
        qo, ao, _ = stepper.solve_sample(mesh, p[s], dt, 13, stepper.QOI_ENERGY)
        assert abs(q[s, 0] - qo) <= TOL * abs(qo) and _rel(a[s], ao) <= TOL, s


@pytest.mark.parametrize("cluster", CLUSTERS)
def test_cluster_split_parareal(ctx, mqs, monkeypatch, cluster):
    monkeypatch.setenv("MQS_DIRECT_WIDE", "1")
    monkeypatch.setenv("MQS_DIRECT_CLUSTER", cluster)
    mesh = meshes.annulus("5k")
    p = params.annulus_nominal(1)
    n_steps, M, cf, tol = 128, 8, 4, 1e-8
    dt = configs.PERIOD / 128
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, n_steps * dt, 50.0, mqs.MQS_QOI_JOULE)
    K = ctx.propagate(b, 0, dt, n_slices=M, coarse_factor=cf, max_par_iters=M, par_tol=tol)
    q, st = ctx.read_qoi(b)
    a = ctx.read_state(b, 0)
    assert not st.any()
    d = fem.Discretisation(mesh, p[0])
    ref = parareal.parareal_sample(d, dt, n_steps, M, cf, tol, stepper.QOI_JOULE)
    q_ref = stepper.qoi_finish(stepper.QOI_JOULE, ref["qoi_raw"], n_steps, dt)
    assert K == ref["iters"]
    assert abs(q[0, 0] - q_ref) <= TOL * abs(q_ref)
    assert _rel(a[0], ref["a_end"]) <= TOL


@pytest.mark.parametrize("cluster", ["2", "8"])
def test_cluster_split_lane_is_independent_of_batch(ctx, mqs, monkeypatch, cluster):
    """With the cluster size fixed, a sample's result does not depend on the
    other lanes of its launch: bitwise equal alone and inside a batch."""
    monkeypatch.setenv("MQS_DIRECT_WIDE", "1")
    monkeypatch.setenv("MQS_DIRECT_CLUSTER", cluster)
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(6, 1, seed=5)
    mid = ctx.upload_mesh(mesh)
    out = []
    for pp in (p, p[4:5]):
        b = ctx.set_samples(mid, pp)
        ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
        ctx.set_time(b, 0.0, configs.PERIOD / 8, 50.0, mqs.MQS_QOI_JOULE)
        ctx.propagate(b, 1, configs.level_dt(1))
        out.append((ctx.read_qoi(b)[0], ctx.read_state(b, 0)))
    assert out[0][0][4, 0] == out[1][0][0, 0]
    assert np.array_equal(out[0][1][4], out[1][1][0])


@pytest.mark.parametrize("n_samples", [1, 3])
def test_cluster_band_cholesky_matches_one_cta_bitwise(ctx, mqs, monkeypatch, n_samples):
    """The band Cholesky on a cluster of CTAs (per-column DSMEM exchange)
    performs the same operations per entry as the one-CTA kernel: the states
    after stepping with either factor are bitwise equal, and match the oracle."""
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(n_samples, 0, seed=21)
    mid = ctx.upload_mesh(mesh)
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("MQS_CHOL_CLUSTER", flag)
        b = ctx.set_samples(mid, p)
        ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
        ctx.set_time(b, 0.0, configs.PERIOD / 8, 50.0, mqs.MQS_QOI_JOULE)
        ctx.propagate(b, 0, configs.level_dt(0))
        q, st = ctx.read_qoi(b)
        assert not st.any()
        out.append((q.copy(), ctx.read_state(b, 0)))
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][0], out[1][0])
    qo, ao, _ = stepper.solve_sample(mesh, p[0], configs.level_dt(0), 8, stepper.QOI_JOULE)
    assert abs(out[0][0][0, 0] - qo) <= TOL * abs(qo) and _rel(out[0][1][0], ao) <= TOL


@pytest.mark.parametrize("cluster", ["1", "2", "4", "8"])
def test_cluster_split_ragged_blocks(ctx, mqs, monkeypatch, cluster):
    """n = 225 unknowns: three full 64-row blocks and a ragged fourth, every
    cluster size, energy QoI, plain stepping and Parareal against the oracle."""
    monkeypatch.setenv("MQS_DIRECT_WIDE", "1")
    monkeypatch.setenv("MQS_DIRECT_CLUSTER", cluster)
    mesh = meshes.unit_square(16)
    p = params.square_samples(2)
    dt = configs.PERIOD / 40
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, 24 * dt, 50.0, mqs.MQS_QOI_ENERGY)
    ctx.propagate(b, 0, dt)
    q, st = ctx.read_qoi(b)
    a = ctx.read_state(b, 0)
    assert not st.any()
    for s in range(2):
        qo, ao, _ = stepper.solve_sample(mesh, p[s], dt, 24, stepper.QOI_ENERGY)
        assert abs(q[s, 0] - qo) <= TOL * abs(qo) and _rel(a[s], ao) <= TOL, s
    b = ctx.set_samples(mid, p[:1])
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, 24 * dt, 50.0, mqs.MQS_QOI_ENERGY)
    K = ctx.propagate(b, 0, dt, n_slices=6, coarse_factor=2, max_par_iters=6, par_tol=1e-9)
    q, st = ctx.read_qoi(b)
    assert not st.any()
    ref = parareal.parareal_sample(fem.Discretisation(mesh, p[0]), dt, 24, 6, 2, 1e-9,
                                   stepper.QOI_ENERGY)
    assert K == ref["iters"]
    q_ref = stepper.qoi_finish(stepper.QOI_ENERGY, ref["qoi_raw"], 24, dt)
    assert abs(q[0, 0] - q_ref) <= TOL * abs(q_ref)


def test_cluster_band_cholesky_tiny(ctx, mqs, monkeypatch):
    """9 unknowns on a cluster of 8 CTAs: most CTAs own one row or none."""
    monkeypatch.setenv("MQS_CHOL_CLUSTER", "1")
    mesh = meshes.unit_square(4)
    p = params.square_samples(1)
    dt = configs.PERIOD / 20
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, 5 * dt, 50.0, mqs.MQS_QOI_JOULE)
    ctx.propagate(b, 0, dt)
    q, st = ctx.read_qoi(b)
    a = ctx.read_state(b, 0)
    assert not st.any()
    qo, ao, _ = stepper.solve_sample(mesh, p[0], dt, 5, stepper.QOI_JOULE)
    assert abs(q[0, 0] - qo) <= TOL * abs(qo) and _rel(a[0], ao) <= TOL


def test_banded_parareal_level_pair(ctx, mqs):
    """MLMC level with Parareal on the fine level and the companion level l-1
    solved sequentially (its factor on the main stream, the fine factor on the
    side stream): both QoIs against the oracle."""
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(2, 1, seed=31)
    dt1, dt0 = configs.level_dt(1), configs.level_dt(0)
    n_steps, M, cf, tol = 64, 8, 2, 1e-9
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, n_steps * dt1, 50.0, mqs.MQS_QOI_JOULE)
    K = ctx.propagate(b, 1, dt1, dt_prev=dt0, n_slices=M, coarse_factor=cf, max_par_iters=M,
                      par_tol=tol)
    q, st = ctx.read_qoi(b)
    assert not st.any()
    # oracle jump norms after iterations 3 and 4: 7.9e-9 / 1.5e-10 (sample 0),
    # 5.4e-9 / 9.7e-11 (sample 1): both stop at K = 4, away from 1e-9
    assert K == 4
    for s in range(2):
        d = fem.Discretisation(mesh, p[s])
        ref = parareal.parareal_sample(d, dt1, n_steps, M, cf, tol, stepper.QOI_JOULE)
        assert ref["iters"] == K, s
        qc, _, _ = stepper.solve_sample(mesh, p[s], dt0, n_steps // 2, stepper.QOI_JOULE)
        assert abs(q[s, 1] - qc) <= TOL * abs(qc), s
        q_ref = stepper.qoi_finish(stepper.QOI_JOULE, ref["qoi_raw"], n_steps, dt1)
        assert abs(q[s, 0] - q_ref) <= TOL * abs(q_ref), s


def test_expired_wait_reports_timeout_and_context_stays_usable(ctx, mqs, monkeypatch):
    """A wait on a count nothing reaches (the context's test hook, one-CTA
    form: no cross-CTA traffic) runs out of polls: the lane reports MQS_ST_TIMEOUT, and the same
    context then solves correctly."""
    mesh = meshes.unit_square(8)
    p = params.square_samples(2)
    dt = configs.PERIOD / 20
    mid = ctx.upload_mesh(mesh)
    monkeypatch.setenv("MQS_DIRECT_WIDE", "1")
    monkeypatch.setenv("MQS_DIRECT_CLUSTER", "1")
    ctx.set_test_hook(mqs.MQS_TEST_HOOK_STALL)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, 4 * dt, 50.0, mqs.MQS_QOI_JOULE)
    ctx.propagate(b, 0, dt)
    _, st = ctx.read_qoi(b)
    assert (st & mqs.MQS_ST_TIMEOUT).all()
    ctx.set_test_hook(0)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, 4 * dt, 50.0, mqs.MQS_QOI_JOULE)
    ctx.propagate(b, 0, dt)
    q, st = ctx.read_qoi(b)
    assert not st.any()
    qo, _, _ = stepper.solve_sample(mesh, p[0], dt, 4, stepper.QOI_JOULE)
    assert abs(q[0, 0] - qo) <= TOL * abs(qo)


@pytest.mark.parametrize("n_samples", [75, 160])
def test_banded_default_shapes_many_lanes(ctx, mqs, n_samples):
    """The launch shapes that MLMC levels run, chosen by the library alone (no
    overrides).  A level pair has two lanes per sample.  75 samples = 150
    lanes: too many for 2-CTA clusters in one wave on 152 SMs, so they run as
    2-CTA clusters in several waves.  160 samples = 320 lanes (at least two
    per SM): 256-thread one-CTA lanes with the work vector in L2, four per
    SM.  Every lane against the oracle at 1e-10."""
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(n_samples, 1, seed=40 + n_samples)
    dt1, dt0 = configs.level_dt(1), configs.level_dt(0)
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
    ctx.set_time(b, 0.0, 8 * dt1, 50.0, mqs.MQS_QOI_JOULE)
    ctx.propagate(b, 1, dt1, dt_prev=dt0)
    q, st = ctx.read_qoi(b)
    a, ac = ctx.read_state(b, 0), ctx.read_state(b, 1)
    assert not st.any()
    for s in range(n_samples):
        qf, af, _ = stepper.solve_sample(mesh, p[s], dt1, 8, stepper.QOI_JOULE)
        qc, acc, _ = stepper.solve_sample(mesh, p[s], dt0, 4, stepper.QOI_JOULE)
        assert abs(q[s, 0] - qf) <= TOL * abs(qf) and abs(q[s, 1] - qc) <= TOL * abs(qc), s
        assert _rel(a[s], af) <= TOL and _rel(ac[s], acc) <= TOL, s


@pytest.mark.parametrize("M,cf,n_samples", [(16, 4, 1), (64, 1, 2), (8, 2, 3)])
def test_pipelined_parareal_is_bitwise_the_stepwise_driver(ctx, mqs, monkeypatch, M, cf,
                                                           n_samples):
    """Parareal with the coarse sweep overlapped by the next iteration's fine
    chunks (and that iteration cancelled once the stopping rule holds) runs
    the same per-lane arithmetic as the driver that finishes each iteration
    before the next: same K, bitwise the same QoI and final states; and both
    match the oracle's Parareal.  Chunks of 1 and of 4 slices, several samples."""
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(n_samples, 0, seed=50 + M)
    n_steps, tol = 256, 1e-8
    dt = configs.PERIOD / 128
    mid = ctx.upload_mesh(mesh)
    out = []
    for pipe in ("1", "0"):
        monkeypatch.setenv("MQS_PARAREAL_PIPELINE", pipe)
        b = ctx.set_samples(mid, p)
        ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
        ctx.set_time(b, 0.0, n_steps * dt, 50.0, mqs.MQS_QOI_JOULE)
        K = ctx.propagate(b, 0, dt, n_slices=M, coarse_factor=cf, max_par_iters=M, par_tol=tol)
        q, st = ctx.read_qoi(b)
        assert not st.any()
        out.append((K, q.copy(), ctx.read_state(b, 0), ctx.read_stats(b)))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
    assert np.array_equal(out[0][3], out[1][3])      # the same executed-step counts
    K, q, a = out[0][0], out[0][1], out[0][2]
    for s in range(n_samples):
        d = fem.Discretisation(mesh, p[s])
        ref = parareal.parareal_sample(d, dt, n_steps, M, cf, 0.0, stepper.QOI_JOULE,
                                       max_iter=K)
        q_ref = stepper.qoi_finish(stepper.QOI_JOULE, ref["qoi_raw"], n_steps, dt)
        assert abs(q[s, 0] - q_ref) <= TOL * abs(q_ref), s
        assert _rel(a[s], ref["a_end"]) <= TOL, s


def test_pipelined_parareal_iteration_limit(ctx, mqs):
    """max_par_iters below the slice count: the last allowed iteration ends the
    run without a speculative one; K and the QoI match the oracle's Parareal
    stopped at that iteration."""
    mesh = meshes.annulus("5k")
    p = params.annulus_nominal(1)
    n_steps, M, cf = 128, 16, 2
    dt = configs.PERIOD / 128
    mid = ctx.upload_mesh(mesh)
    for kmax in (1, 2):
        b = ctx.set_samples(mid, p)
        ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
        ctx.set_time(b, 0.0, n_steps * dt, 50.0, mqs.MQS_QOI_JOULE)
        K = ctx.propagate(b, 0, dt, n_slices=M, coarse_factor=cf, max_par_iters=kmax,
                          par_tol=0.0)
        q, st = ctx.read_qoi(b)
        assert K == kmax and not st.any()
        ref = parareal.parareal_sample(fem.Discretisation(mesh, p[0]), dt, n_steps, M, cf, 0.0,
                                       stepper.QOI_JOULE, max_iter=kmax)
        q_ref = stepper.qoi_finish(stepper.QOI_JOULE, ref["qoi_raw"], n_steps, dt)
        assert abs(q[0, 0] - q_ref) <= TOL * abs(q_ref)
        assert _rel(ctx.read_state(b, 0)[0], ref["a_end"]) <= TOL


@pytest.mark.parametrize("cl", [1, 2, 4, 8])
def test_cluster_layouts_are_bitwise_equal(ctx, mqs, monkeypatch, cl):
    """The cluster stepping kernels keep either a full copy of the work vector
    (meshes that fit shared memory) or their own rows plus a ring of recently
    solved rows; the arithmetic and its order are the same, so both layouts
    give bitwise the same QoI, final states and Parareal iterations on every
    cluster size."""
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(3, 0, seed=71 + cl)
    n_steps = 96
    dt = configs.PERIOD / 128
    mid = ctx.upload_mesh(mesh)
    monkeypatch.setenv("MQS_DIRECT_CLUSTER", str(cl))
    monkeypatch.setenv("MQS_CHAIN_CLUSTER", str(cl))
    out = []
    for ring in ("0", "1"):
        monkeypatch.setenv("MQS_CLUSTER_RING", ring)
        b = ctx.set_samples(mid, p)
        ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
        ctx.set_time(b, 0.0, n_steps * dt, 50.0, mqs.MQS_QOI_JOULE)
        ctx.propagate(b, 0, dt)
        q, st = ctx.read_qoi(b)
        assert not st.any()
        b2 = ctx.set_samples(mid, p[:1])
        ctx.set_solver(b2, mqs.MQS_SOLVER_BANDED)
        ctx.set_time(b2, 0.0, n_steps * dt, 50.0, mqs.MQS_QOI_JOULE)
        K = ctx.propagate(b2, 0, dt, n_slices=12, coarse_factor=4, max_par_iters=12,
                          par_tol=1e-8)
        q2, st2 = ctx.read_qoi(b2)
        assert not st2.any()
        out.append((q.copy(), ctx.read_state(b, 0), K, q2.copy(), ctx.read_state(b2, 0)))
    full, ring = out
    assert np.array_equal(full[0], ring[0]) and np.array_equal(full[1], ring[1])
    assert full[2] == ring[2]
    assert np.array_equal(full[3], ring[3]) and np.array_equal(full[4], ring[4])
    q_ref, a_ref, _ = stepper.solve_sample(mesh, p[0], dt, n_steps, stepper.QOI_JOULE)
    assert abs(full[0][0, 0] - q_ref) <= TOL * abs(q_ref)
    assert _rel(full[1][0], a_ref) <= TOL
