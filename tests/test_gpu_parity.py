"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 results within 1e-10 relative (per-sample QoI; final
states normwise); mixed precision within 1e-6 relative on the QoI.
"""
import os

import numpy as np
import pytest

from oracle import fem, mlmc, parareal, stepper
from workloads import configs, meshes, params

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_QOI_TOL = 1e-6
CG_TOL = 1e-13


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
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_region_matrices_and_apply(ctx, mqs):
    rng = np.random.default_rng(0)
    for mesh, p in ((meshes.unit_square(16), params.square_samples(5)),
                    (meshes.annulus("5k"), params.annulus_samples(5, 1))):
        mid = ctx.upload_mesh(mesh)
        n, nnz = ctx.mesh_info(mid)
        assert n == mesh.n_free
        b = ctx.set_samples(mid, p)
        x = rng.normal(size=(p.shape[0], n))
        dt = 1.7e-4
        yM, yK, yA = ctx.apply(b, 0, dt, x), ctx.apply(b, 1, dt, x), ctx.apply(b, 2, dt, x)
        for s in range(p.shape[0]):
            d = fem.Discretisation(mesh, p[s])
            assert _rel(yM[s], d.M @ x[s]) < 1e-13
            assert _rel(yK[s], d.K @ x[s]) < 1e-13
            assert _rel(yA[s], (d.M / dt + d.K) @ x[s]) < 1e-13
        assert nnz == d.M.nnz


def _run_plain(ctx, mqs, mesh, p, t_end, dt, qoi, dt_prev=0.0, precision=0, cg_tol=CG_TOL):
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_time(b, 0.0, t_end, 50.0, qoi)
    ctx.propagate(b, 1 if dt_prev else 0, dt, dt_prev=dt_prev, precision=precision,
                  cg_tol=cg_tol, cg_max_iters=20000)
    q, st = ctx.read_qoi(b)
    a = ctx.read_state(b, 0)
    ac = ctx.read_state(b, 1) if dt_prev else None
    return b, q, st, a, ac


def test_mc_square_full_config(ctx, mqs):
    """Unit square 16x16, 32 samples, 64 steps over one period, energy QoI."""
    cfg = configs.MC_SQUARE
    mesh = meshes.unit_square(16)
    p = params.square_samples(cfg.n_samples)
    dt = cfg.t_end / cfg.n_steps
    _, q, st, a, _ = _run_plain(ctx, mqs, mesh, p, cfg.t_end, dt, mqs.MQS_QOI_ENERGY)
    assert not st.any()
    for s in range(cfg.n_samples):
        qo, ao, _ = stepper.solve_sample(mesh, p[s], dt, cfg.n_steps, stepper.QOI_ENERGY)
        assert abs(q[s, 0] - qo) <= FP64_TOL * abs(qo), s
        assert _rel(a[s], ao) <= FP64_TOL, s
        assert q[s, 1] == 0.0


def test_level_pair_ragged_batch_annulus(ctx, mqs):
    """37 samples (ragged tile), level 1 pair on the 5k annulus, joule QoI."""
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(37, 1)
    T = configs.PERIOD
    dt1, dt0 = configs.level_dt(1), configs.level_dt(0)
    _, q, st, a, ac = _run_plain(ctx, mqs, mesh, p, T, dt1, mqs.MQS_QOI_JOULE, dt_prev=dt0)
    assert not st.any()
    for s in range(p.shape[0]):
        qf, af, _ = stepper.solve_sample(mesh, p[s], dt1, 128, stepper.QOI_JOULE)
        qc, acc, _ = stepper.solve_sample(mesh, p[s], dt0, 64, stepper.QOI_JOULE)
        assert abs(q[s, 0] - qf) <= FP64_TOL * abs(qf), (s, q[s, 0], qf)
        assert abs(q[s, 1] - qc) <= FP64_TOL * abs(qc), (s, q[s, 1], qc)
        assert _rel(a[s], af) <= FP64_TOL and _rel(ac[s], acc) <= FP64_TOL


def test_parareal_matches_oracle_parareal(ctx, mqs):
    mesh = meshes.annulus("5k")
    p = params.annulus_nominal(1)
    n_steps, M, cf, tol = 256, 16, 4, 1e-8
    dt = configs.PERIOD / 128
    T = n_steps * dt
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_time(b, 0.0, T, 50.0, mqs.MQS_QOI_JOULE)
    K = ctx.propagate(b, 0, dt, n_slices=M, coarse_factor=cf, max_par_iters=M, par_tol=tol,
                      cg_tol=CG_TOL, cg_max_iters=20000)
    q, st = ctx.read_qoi(b)
    a = ctx.read_state(b, 0)
    assert not st.any()
    d = fem.Discretisation(mesh, p[0])
    ref = parareal.parareal_sample(d, dt, n_steps, M, cf, tol, stepper.QOI_JOULE)
    # the oracle's jump norms are 5.5e-8 after iteration 2 and 2.9e-10 after
    # iteration 3: the tolerance 1e-8 lies far from both, so K is unique
    assert K == ref["iters"] == 3
    q_ref = stepper.qoi_finish(stepper.QOI_JOULE, ref["qoi_raw"], n_steps, dt)
    assert abs(q[0, 0] - q_ref) <= FP64_TOL * abs(q_ref)
    assert _rel(a[0], ref["a_end"]) <= FP64_TOL
    # and both agree with the serial fine solve to the Parareal tolerance
    q_ser, a_ser, _ = stepper.solve_sample(mesh, p[0], dt, n_steps, stepper.QOI_JOULE)
    assert abs(q[0, 0] - q_ser) <= 1e-6 * abs(q_ser)
    assert _rel(a[0], a_ser) <= 1e-6


def test_parareal_K_equals_M_is_the_serial_solve(ctx, mqs):
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(2, 0, seed=3)
    n_steps, M, cf = 64, 8, 2
    dt = configs.PERIOD / 64
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_time(b, 0.0, n_steps * dt, 50.0, mqs.MQS_QOI_JOULE)
    K = ctx.propagate(b, 0, dt, n_slices=M, coarse_factor=cf, max_par_iters=M, par_tol=0.0,
                      cg_tol=CG_TOL, cg_max_iters=20000)
    assert K == M
    qp, _ = ctx.read_qoi(b)
    ap = ctx.read_state(b, 0)
    b2 = ctx.set_samples(mid, p)
    ctx.set_time(b2, 0.0, n_steps * dt, 50.0, mqs.MQS_QOI_JOULE)
    ctx.propagate(b2, 0, dt, cg_tol=CG_TOL, cg_max_iters=20000)
    qs, _ = ctx.read_qoi(b2)
    as_ = ctx.read_state(b2, 0)
    for s in range(2):
        assert abs(qp[s, 0] - qs[s, 0]) <= 1e-11 * abs(qs[s, 0])
        assert _rel(ap[s], as_[s]) <= 1e-11


def test_mixed_precision_qoi_accuracy(ctx, mqs):
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(8, 2)
    dt = configs.level_dt(1)
    _, q, st, _, _ = _run_plain(ctx, mqs, mesh, p, configs.PERIOD, dt, mqs.MQS_QOI_JOULE,
                                precision=mqs.MQS_MIXED, cg_tol=1e-9)
    assert not st.any()
    for s in range(p.shape[0]):
        qo, _, _ = stepper.solve_sample(mesh, p[s], dt, 128, stepper.QOI_JOULE)
        assert abs(q[s, 0] - qo) <= MIXED_QOI_TOL * abs(qo), (s, q[s, 0], qo)


def test_mlmc_estimator_matches_oracle(ctx, mqs):
    mesh = meshes.annulus("5k")
    N = (12, 6, 3)
    base = 16
    mid = ctx.upload_mesh(mesh)
    ctx.mlmc_reset(len(N))
    pairs, gpu_pairs = [], []
    for l, n in enumerate(N):
        p = params.annulus_samples(n, l, seed=99)
        b = ctx.set_samples(mid, p)
        ctx.set_time(b, 0.0, configs.PERIOD, 50.0, mqs.MQS_QOI_JOULE)
        dtl = configs.level_dt(l, base)
        ctx.propagate(b, l, dtl, dt_prev=configs.level_dt(l - 1, base) if l else 0.0,
                      cg_tol=CG_TOL, cg_max_iters=20000)
        ctx.mlmc_accumulate(b, l)
        qg, _ = ctx.read_qoi(b)
        qf, qc = [], []
        for s in range(n):
            a, c = mlmc.level_pair(mesh, p[s], l, lambda k: configs.level_dt(k, base),
                                   lambda k: configs.level_steps(1, k, base), stepper.QOI_JOULE)
            qf.append(a)
            qc.append(c)
        assert np.allclose(qg[:, 0], qf, rtol=FP64_TOL, atol=0)
        if l:
            assert np.allclose(qg[:, 1], qc, rtol=FP64_TOL, atol=0)
        pairs.append((qf, qc if l else None))
        gpu_pairs.append((qg[:, 0].copy(), qg[:, 1].copy() if l else None))
    lv, est, rmse = ctx.mlmc_readout()
    # (1) the moment kernel on the GPU's own level differences: the oracle's
    # exactly rounded two-pass moments of the same Y, to round-off
    own = mlmc.mlmc_estimate(gpu_pairs)
    assert est == pytest.approx(own["estimate"], rel=1e-14)
    assert rmse == pytest.approx(own["rmse"], rel=1e-12)
    for l, (n, mean, var) in enumerate(own["levels"]):
        scale = np.abs(gpu_pairs[l][0]).max()
        assert lv[l, 0] == n
        assert abs(lv[l, 1] - mean) <= 1e-14 * scale
        assert lv[l, 2] == pytest.approx(var, rel=1e-12)
    # (2) against the oracle's independent solves: each Q is within FP64_TOL
    # relative, so each Y = Q_l - Q_{l-1} is within d_l = FP64_TOL (|Q_l| +
    # |Q_{l-1}|) absolute (larger relative to Y because of the cancellation);
    # a mean moves by at most d_l and an unbiased variance by at most
    # 2 sqrt(N/(N-1)) (2 d_l) sqrt(var) + N/(N-1) (2 d_l)^2
    ref = mlmc.mlmc_estimate(pairs)
    tot = 0.0
    for l, (n, mean, var) in enumerate(ref["levels"]):
        qf, qc = pairs[l]
        d = FP64_TOL * (np.abs(qf).max() + (np.abs(qc).max() if l else 0.0))
        tot += d
        f = n / (n - 1)
        # (+ the round-off of the moment sums themselves, 1e-14 of the scale)
        assert abs(lv[l, 1] - mean) <= d + 1e-14 * np.abs(qf).max()
        assert abs(lv[l, 2] - var) <= (2 * np.sqrt(f) * 2 * d * np.sqrt(var) + f * 4 * d * d
                                       + 1e-12 * var)
    assert abs(est - ref["estimate"]) <= tot + 1e-14 * abs(ref["estimate"])


def test_result_is_the_same_alone_and_in_a_mix(ctx, mqs, monkeypatch):
    """Reduction order depends on the launch shape only: with the shape fixed,
    a sample's result is bitwise the same alone and inside a larger batch."""
    monkeypatch.setenv("MQS_TILE_L", "8")
    monkeypatch.setenv("MQS_CLUSTER", "4")
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(11, 0, seed=5)
    dt = configs.level_dt(0)
    _, q_mix, _, a_mix, _ = _run_plain(ctx, mqs, mesh, p, configs.PERIOD, dt, mqs.MQS_QOI_JOULE)
    _, q_one, _, a_one, _ = _run_plain(ctx, mqs, mesh, p[6:7], configs.PERIOD, dt,
                                       mqs.MQS_QOI_JOULE)
    assert q_one[0, 0] == q_mix[6, 0]
    assert np.array_equal(a_one[0], a_mix[6])


def test_edge_cases_and_errors(ctx, mqs):
    mesh = meshes.unit_square(8)
    p = params.square_samples(1)
    # a single sample, a single step
    _, q, st, a, _ = _run_plain(ctx, mqs, mesh, p, 0.02 / 16, 0.02 / 16, mqs.MQS_QOI_JOULE)
    qo, ao, _ = stepper.solve_sample(mesh, p[0], 0.02 / 16, 1, stepper.QOI_JOULE)
    assert abs(q[0, 0] - qo) <= FP64_TOL * abs(qo) and _rel(a[0], ao) <= FP64_TOL
    # the iteration limit is reported per sample, the call succeeds
    mid = ctx.upload_mesh(mesh)
    b = ctx.set_samples(mid, p)
    ctx.set_time(b, 0.0, 0.02, 50.0, mqs.MQS_QOI_JOULE)
    ctx.propagate(b, 0, 0.02 / 16, cg_tol=1e-14, cg_max_iters=2)
    _, st = ctx.read_qoi(b)
    assert st[0] & mqs.MQS_ST_NOTCONV
    # invalid arguments fail with a message, the context stays usable
    with pytest.raises(mqs.MQSError, match="integer"):
        ctx.propagate(b, 0, 0.03, cg_tol=1e-12)
    with pytest.raises(mqs.MQSError, match="n_params"):
        ctx.set_samples(mid, np.ones((2, 5)))
    with pytest.raises(mqs.MQSError, match="Parareal"):
        ctx.propagate(b, 0, 0.02 / 16, n_slices=3, coarse_factor=1, max_par_iters=3)
    ctx.propagate(b, 0, 0.02 / 16, cg_tol=1e-13)
    q2, st2 = ctx.read_qoi(b)
    assert not st2.any()
