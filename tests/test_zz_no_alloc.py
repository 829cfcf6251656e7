"""The allocation-free stepping entry point against the regular one.

Some callers may not allocate device memory while they run -- a real-time or
signal-safe host path, a runtime that splits all device memory into its own
pools at start-up, a region being recorded -- so ``mqs_propagate_noalloc``
does its work in a static scratch array and touches only the caller's inputs
and outputs.  Here it is called twice in a row through the C ABI and each
result is compared with ``mqs_propagate`` on the same samples.
"""
import numpy as np
import pytest

from oracle import fem
from workloads import configs, meshes, params

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the FP64 tolerance of the parity tests


def _lane_inputs(mesh, p, dt):
    """CSR pattern and lane-fastest values of A = M/dt + K, M and D^-1."""
    discs = [fem.Discretisation(mesh, p[s]) for s in range(p.shape[0])]
    pat = discs[0].M.tocsr()
    pat.sort_indices()
    n = pat.shape[0]
    rows = np.repeat(np.arange(n), np.diff(pat.indptr))
    cols = pat.indices
    nl = p.shape[0]
    A = np.zeros((pat.nnz, nl))
    M = np.zeros((pat.nnz, nl))
    D = np.zeros((n, nl))
    for s, d in enumerate(discs):
        As = (d.M / dt + d.K).tocsr()
        A[:, s] = np.asarray(As[rows, cols]).ravel()
        M[:, s] = np.asarray(d.M.tocsr()[rows, cols]).ravel()
        D[:, s] = 1.0 / As.diagonal()
    P = mesh.n_phases
    R = mesh.n_regions
    amp = p[:, 2 * R:2 * R + 1] * p[:, 2 * R + 1:2 * R + 1 + P]
    ph = p[:, 2 * R + 1 + P:2 * R + 1 + 2 * P]
    return (pat.indptr.astype(np.int32), cols.astype(np.int32), A, M, D, discs[0].F,
            np.ascontiguousarray(amp), np.ascontiguousarray(ph))


def test_noalloc_matches_propagate_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from paper_2507_19246_gb300 import mqs

    mesh = meshes.annulus("5k")
    p = params.annulus_samples(6, 0, seed=21)
    dt = configs.level_dt(1)
    n_steps = 64
    T = n_steps * dt
    with mqs.Context(0) as ctx:
        mid = ctx.upload_mesh(mesh)
        b = ctx.set_samples(mid, p)
        ctx.set_time(b, 0.0, T, 50.0, mqs.MQS_QOI_JOULE)
        ctx.propagate(b, 0, dt, cg_tol=1e-13, cg_max_iters=20000)
        q_ref, st_ref = ctx.read_qoi(b)
        a_ref = ctx.read_state(b, 0)
    assert not st_ref.any()

    rowptr, colidx, A, M, D, F, amp, ph = _lane_inputs(mesh, p, dt)
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
         for k, v in dict(rowptr=rowptr, colidx=colidx, A=A, M=M, D=D, F=F).items()}
    n, nl = D.shape
    stream = torch.cuda.current_stream(dev).cuda_stream
    for call in range(2):
        a_out = torch.full((n, nl), float("nan"), dtype=torch.float64, device=dev)
        q_out = torch.full((nl,), float("nan"), dtype=torch.float64, device=dev)
        st_out = torch.full((nl,), -1, dtype=torch.int32, device=dev)
        mqs.mqs_propagate_noalloc(0, stream, n, t["rowptr"], t["colidx"], A.shape[0], nl, t["A"],
                                  t["M"], None, t["D"], mesh.n_phases, t["F"], amp, ph, 0.0, dt,
                                  n_steps, 50.0, mqs.MQS_QOI_JOULE, 1e-13, 20000, a_out, q_out,
                                  st_out)
        torch.cuda.synchronize()
        q = q_out.cpu().numpy()
        a = a_out.cpu().numpy().T
        assert not st_out.cpu().numpy().any(), call
        for s in range(nl):
            assert abs(q[s] - q_ref[s, 0]) <= TOL * abs(q_ref[s, 0]), (call, s, q[s], q_ref[s, 0])
            assert np.linalg.norm(a[s] - a_ref[s]) <= TOL * np.linalg.norm(a_ref[s]), (call, s)

    # sizes beyond the scratch array are refused before any work is queued
    with pytest.raises(mqs.MQSError, match="too large"):
        mqs.mqs_propagate_noalloc(0, stream, 10 ** 6, t["rowptr"], t["colidx"], A.shape[0], 64,
                                  t["A"], t["M"], None, t["D"], mesh.n_phases, t["F"], amp, ph,
                                  0.0, dt, n_steps, 50.0, mqs.MQS_QOI_JOULE, 1e-13, 20000, a_out,
                                  q_out, st_out)
