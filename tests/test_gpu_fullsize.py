"""Full-size parity at the bench's workload and launch configuration: Parareal
on one nominal sample of the 20k-node annulus (4096 fine steps, 64 slices,
coarse step 64 fine steps, tolerance 1e-8), against the oracle's Parareal and
its serial fine solve."""
import numpy as np
import pytest

import bench
from oracle import fem, parareal, stepper

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def reference():
    """The oracle's Parareal and serial fine solve of the bench workload."""
    wl = bench.workload("parareal20k")
    mesh, p = wl["mesh"], wl["params"]
    d = fem.Discretisation(mesh, p[0])
    ref = parareal.parareal_sample(d, wl["dt"], wl["n_steps"], wl["n_slices"], wl["cf"],
                                   wl["par_tol"], wl["qoi"])
    ref["q"] = stepper.qoi_finish(wl["qoi"], ref["qoi_raw"], wl["n_steps"], wl["dt"])
    ref["q_ser"], ref["a_ser"], _ = stepper.solve_sample(mesh, p[0], wl["dt"], wl["n_steps"],
                                                         wl["qoi"])
    return wl, ref


@pytest.mark.parametrize("solver", ["banded", "banded-stepwise", "pcg"])
def test_parareal_annulus20k_full_size(reference, solver, monkeypatch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from paper_2507_19246_gb300 import mqs

    wl, ref = reference
    mesh, p = wl["mesh"], wl["params"]
    # "banded": the bench's path (sweep and fine chunks overlapped);
    # "banded-stepwise": each Parareal iteration finished before the next
    monkeypatch.setenv("MQS_PARAREAL_PIPELINE", "0" if solver == "banded-stepwise" else "1")
    with mqs.Context(0) as ctx:
        mid = ctx.upload_mesh(mesh)
        b = ctx.set_samples(mid, p)
        if solver.startswith("banded"):
            ctx.set_solver(b, mqs.MQS_SOLVER_BANDED)
        ctx.set_time(b, 0.0, wl["t_end"], 50.0, wl["qoi"])
        K = ctx.propagate(b, 0, wl["dt"], n_slices=wl["n_slices"], coarse_factor=wl["cf"],
                          max_par_iters=wl["n_slices"], par_tol=wl["par_tol"],
                          precision=mqs.MQS_FP64, cg_tol=wl["cg_tol"],
                          cg_max_iters=20000 if solver == "pcg" else 1)
        q, st = ctx.read_qoi(b)
        a = ctx.read_state(b, 0)
    if solver.startswith("banded"):
        ref.setdefault("banded_runs", {})[solver] = (q.copy(), a.copy())
        runs = ref["banded_runs"]
        if len(runs) == 2:   # the overlapped driver is bitwise the stepwise one
            (q1, a1), (q2, a2) = runs.values()
            assert np.array_equal(q1, q2) and np.array_equal(a1, a2)
    assert not st.any()
    assert K == ref["iters"]
    assert abs(q[0, 0] - ref["q"]) <= 1e-10 * abs(ref["q"]), (q[0, 0], ref["q"])
    assert np.linalg.norm(a[0] - ref["a_end"]) <= 1e-10 * np.linalg.norm(ref["a_end"])
    # and the serial fine solve (what Parareal converges to) within its tolerance
    assert abs(q[0, 0] - ref["q_ser"]) <= 1e-6 * abs(ref["q_ser"])
    assert np.linalg.norm(a[0] - ref["a_ser"]) <= 1e-6 * np.linalg.norm(ref["a_ser"])
