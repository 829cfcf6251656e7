"""The request server (continuous batching of level samples and Parareal
slices on several meshes): every request's result is bitwise the same alone
and in a mix, matches the oracle, and admission follows the HBM budget."""
import numpy as np
import pytest

from oracle import fem, stepper
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


def _requests(mqs, mids):
    """A mix: level samples (levels 0-2, with companions) and slices on the 5k
    annulus, level samples on the 20k annulus and the unit square (energy
    QoI), different step counts."""
    rng = np.random.default_rng(3)
    reqs = []
    m5, m20, msq = mids
    p5 = params.annulus_samples(6, 1, seed=61)
    for j, l in enumerate([0, 1, 2, 1, 2, 0]):
        dt = configs.level_dt(l)
        n = 16 * 2 ** l
        reqs.append(dict(mesh=("5k", m5), p=p5[j], kind=mqs.MQS_REQ_LEVEL, qoi=mqs.MQS_QOI_JOULE,
                         dt=dt, n=n, dt_prev=configs.level_dt(l - 1) if l else 0.0,
                         n_prev=n // 2 if l else 0))
    for j in range(3):
        a0 = rng.normal(size=4608) * 1e-4 if j else None
        reqs.append(dict(mesh=("5k", m5), p=p5[j], kind=mqs.MQS_REQ_SLICE, qoi=mqs.MQS_QOI_JOULE,
                         dt=configs.level_dt(1), n=24 + 8 * j, k0=40 * j, a_init=a0))
    p20 = params.annulus_samples(2, 0, seed=62)
    for j in range(2):
        reqs.append(dict(mesh=("20k", m20), p=p20[j], kind=mqs.MQS_REQ_LEVEL,
                         qoi=mqs.MQS_QOI_JOULE, dt=configs.level_dt(0), n=8, dt_prev=0.0,
                         n_prev=0))
    psq = params.square_samples(2, seed=63)
    for j in range(2):
        reqs.append(dict(mesh=("sq", msq), p=psq[j], kind=mqs.MQS_REQ_LEVEL,
                         qoi=mqs.MQS_QOI_ENERGY, dt=0.02 / 64, n=64, dt_prev=0.02 / 32, n_prev=32))
    return reqs


def _submit(mqs, srv, r):
    import torch
    out = None
    if r["kind"] == mqs.MQS_REQ_SLICE:
        out = torch.full((4608,), float("nan"), dtype=torch.float64, device="cuda")
        rid = srv.submit(r["mesh"][1], r["p"], r["kind"], r["qoi"], 0.0, r["dt"], r["n"],
                         k0=r["k0"], a_init=r["a_init"], a_out=out)
    else:
        rid = srv.submit(r["mesh"][1], r["p"], r["kind"], r["qoi"], 0.0, r["dt"], r["n"],
                         dt_prev=r["dt_prev"], n_steps_prev=r["n_prev"])
    return rid, out


def test_serving_mix_is_bitwise_the_requests_alone_and_matches_the_oracle(mqs):
    import torch
    mesh_objs = {"5k": meshes.annulus("5k"), "20k": meshes.annulus("20k"),
                 "sq": meshes.unit_square(16)}
    with mqs.Context(0) as ctx:
        mids = [ctx.upload_mesh(mesh_objs[k]) for k in ("5k", "20k", "sq")]
        reqs = _requests(mqs, mids)
        # the mix: small batches on 4 streams, so batches overlap and mix meshes
        with mqs.Server(ctx, n_streams=4, max_batch_lanes=5) as srv:
            ids, outs = zip(*[_submit(mqs, srv, r) for r in reqs])
            res = srv.drain()
            torch.cuda.synchronize()
            mix = [(res[i][0], res[i][1], None if o is None else o.cpu().numpy())
                   for i, o in zip(ids, outs)]
        # every request alone on a server of its own
        alone = []
        for r in reqs:
            with mqs.Server(ctx, n_streams=1, max_batch_lanes=2) as srv:
                i, o = _submit(mqs, srv, r)
                res = srv.drain()
                torch.cuda.synchronize()
                alone.append((res[i][0], res[i][1], None if o is None else o.cpu().numpy()))
    for (qm, sm, am), (qa, sa, aa) in zip(mix, alone):
        assert sm == 0 and sa == 0
        assert np.array_equal(qm, qa)
        assert (am is None and aa is None) or np.array_equal(am, aa)
    # against the oracle
    for r, (q, _, a) in zip(reqs, mix):
        mesh = mesh_objs[r["mesh"][0]]
        oq = stepper.QOI_JOULE if r["qoi"] == mqs.MQS_QOI_JOULE else stepper.QOI_ENERGY
        if r["kind"] == mqs.MQS_REQ_LEVEL:
            qf, _, _ = stepper.solve_sample(mesh, r["p"], r["dt"], r["n"], oq)
            assert abs(q[0] - qf) <= TOL * abs(qf)
            if r["dt_prev"]:
                qc, _, _ = stepper.solve_sample(mesh, r["p"], r["dt_prev"], r["n_prev"], oq)
                assert abs(q[1] - qc) <= TOL * abs(qc)
        else:
            d = fem.Discretisation(mesh, r["p"])
            u0 = np.zeros(d.n) if r["a_init"] is None else r["a_init"]
            ae, raw, _ = stepper.ImplicitEuler(d, r["dt"]).run(u0, r["n"], k0=r["k0"], qoi=oq)
            assert abs(q[0] - raw) <= TOL * abs(raw)
            assert np.linalg.norm(a - ae) <= TOL * np.linalg.norm(ae)


def test_serving_admits_by_footprint(mqs):
    """A budget that holds one 5k level sample at a time: requests run one
    after the other (each admitted only once the previous one's memory is
    back), with the same results as with room for all; a request larger than
    the whole budget is refused at submission."""
    mesh = meshes.annulus("5k")
    p = params.annulus_samples(4, 1, seed=71)
    dt1, dt0 = configs.level_dt(1), configs.level_dt(0)
    with mqs.Context(0) as ctx:
        mid = ctx.upload_mesh(mesh)
        out = []
        for tight in (False, True):
            with mqs.Server(ctx, n_streams=4, max_batch_lanes=8) as probe:
                one = probe.footprint(mid, mqs.MQS_QOI_JOULE, 2)
            budget = int(1.5 * one) if tight else 0
            with mqs.Server(ctx, hbm_budget=budget, n_streams=4, max_batch_lanes=8) as srv:
                ids = [srv.submit(mid, p[j], mqs.MQS_REQ_LEVEL, mqs.MQS_QOI_JOULE, 0.0, dt1, 32,
                                  dt_prev=dt0, n_steps_prev=16) for j in range(4)]
                res = srv.drain()
            out.append([res[i] for i in ids])
            if tight:
                times = [r[2] for r in out[-1]]
                for a, b in zip(times, times[1:]):
                    assert b[1] >= a[2]            # admitted after the previous completed
                with mqs.Server(ctx, hbm_budget=budget, n_streams=1, max_batch_lanes=8) as srv:
                    m20 = ctx.upload_mesh(meshes.annulus("20k"))
                    with pytest.raises(mqs.MQSError, match="budget"):
                        srv.submit(m20, params.annulus_samples(1, 0)[0], mqs.MQS_REQ_LEVEL,
                                   mqs.MQS_QOI_JOULE, 0.0, dt0, 8)
        for (qa, sa, _), (qb, sb, _) in zip(*out):
            assert sa == 0 and sb == 0 and np.array_equal(qa, qb)


def test_serving_rejects_bad_requests(mqs):
    with mqs.Context(0) as ctx:
        mid = ctx.upload_mesh(meshes.unit_square(8))
        with mqs.Server(ctx, n_streams=1, max_batch_lanes=4) as srv:
            p = params.square_samples(1)[0]
            with pytest.raises(mqs.MQSError, match="mesh"):
                srv.submit(mid + 7, p, mqs.MQS_REQ_LEVEL, mqs.MQS_QOI_JOULE, 0.0, 1e-3, 4)
            with pytest.raises(mqs.MQSError, match="bad request"):
                srv.submit(mid, p[:3], mqs.MQS_REQ_LEVEL, mqs.MQS_QOI_JOULE, 0.0, 1e-3, 4)
            with pytest.raises(mqs.MQSError, match="bad request"):
                srv.submit(mid, p, 9, mqs.MQS_QOI_JOULE, 0.0, 1e-3, 4)
            rid = srv.submit(mid, p, mqs.MQS_REQ_LEVEL, mqs.MQS_QOI_JOULE, 0.0, 1e-3, 4)
            res = srv.drain()
            assert rid in res and res[rid][1] == 0
