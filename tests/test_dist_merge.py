"""Multi-rank MLMC path on CPU: two gloo ranks each hold part of every level's
samples; the merged estimate equals the estimate over all samples at once."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import mlmc
from paper_2507_19246_gb300 import dist as D


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _levels_of(pairs):
    out = mlmc.mlmc_estimate(pairs)["levels"]
    return np.asarray([(n, m, v) for n, m, v in out])


def _data():
    rng = np.random.default_rng(7)
    sizes = (40, 17, 6)
    pairs = []
    for l, n in enumerate(sizes):
        qf = 50.0 + rng.normal(size=n) * 10.0 ** -l
        qc = qf - 0.1 * 10.0 ** -l + rng.normal(size=n) * 1e-3 if l else None
        pairs.append((qf, qc))
    return pairs


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pairs = _data()
    mine = []
    for qf, qc in pairs:
        idx = np.arange(rank, len(qf), world)          # samples split round-robin
        mine.append((qf[idx], None if qc is None else qc[idx]))
    est, rmse, rows = D.allreduce_levels(_levels_of(mine))
    out[rank] = (est, rmse, rows.tolist())
    dist.destroy_process_group()


def test_two_rank_merge_equals_single_process():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = mlmc.mlmc_estimate(_data())
    e0, e1 = out[0], out[1]
    assert e0[0] == e1[0] and e0[1] == e1[1]            # identical on every rank
    assert e0[0] == pytest.approx(ref["estimate"], rel=1e-14)
    assert e0[1] == pytest.approx(ref["rmse"], rel=1e-12)
    for (n, m, v), (rn, rm, rv) in zip(e0[2], ref["levels"]):
        assert n == rn and m == pytest.approx(rm, rel=1e-13) and v == pytest.approx(rv, rel=1e-10)


def test_merge_is_exact_for_split_batches():
    y = np.random.default_rng(1).normal(size=101) * 3.0 + 7.0
    recs = [D.records_from_levels(_levels_of([(part, None)]))[0]
            for part in (y[:30], y[30:31], y[31:])]
    merged = D.merge_records(D.merge_records(recs[0], recs[1]), recs[2])
    n, m, v = mlmc.level_moments(y)
    assert merged[0] == n and merged[1] == pytest.approx(m, rel=1e-15)
    assert merged[2] / (n - 1) == pytest.approx(v, rel=1e-12)
