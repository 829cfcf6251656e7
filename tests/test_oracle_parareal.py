"""Pins for the oracle's Parareal (Eq. 12) against the serial fine solve."""
import numpy as np
import pytest

from oracle import fem, parareal, stepper
from workloads import meshes, params


def _setup(n_steps=64, n_slices=8, cf=4):
    m = meshes.unit_square(8)
    d = fem.Discretisation(m, params.square_samples(2)[1])
    dt = 0.02 / n_steps
    return m, d, dt


def _serial(d, dt, n_steps, qoi):
    prop = stepper.ImplicitEuler(d, dt)
    return prop.run(np.zeros(d.n), n_steps, qoi=qoi, keep_states=True)


@pytest.mark.parametrize("qoi", [stepper.QOI_JOULE, stepper.QOI_ENERGY])
def test_K_equal_M_reproduces_serial_fine_bitwise(qoi):
    n_steps, M, cf = 64, 8, 4
    m, d, dt = _setup(n_steps, M, cf)
    a_ser, raw_ser, states = _serial(d, dt, n_steps, qoi)
    res = parareal.parareal_sample(d, dt, n_steps, M, cf, tol=0.0, qoi=qoi)
    assert res["iters"] == M
    assert np.array_equal(res["a_end"], a_ser)
    S = n_steps // M
    for s in range(M):
        assert np.array_equal(res["U"][s], states[s * S]), s
    assert res["qoi_raw"] == raw_ser
    # effort counts of Eq. 13-14: iteration k runs M-k+1 fine and M-k coarse slices
    assert res["fine_slices"] == sum(M - k + 1 for k in range(1, M + 1))
    assert res["coarse_slices"] == (M - 1) + sum(M - k for k in range(1, M + 1))


def test_exactness_after_k_iterations():
    n_steps, M, cf = 64, 8, 8
    m, d, dt = _setup(n_steps, M, cf)
    _, _, states = _serial(d, dt, n_steps, stepper.QOI_JOULE)
    S = n_steps // M
    for K in (1, 2, 3):
        res = parareal.parareal_sample(d, dt, n_steps, M, cf, tol=0.0, qoi=1, max_iter=K)
        for s in range(K + 1):
            assert np.array_equal(res["U"][s], states[s * S]), (K, s)
        # the first not-yet-exact slice start differs from the fine solution
        assert not np.array_equal(res["U"][K + 1], states[(K + 1) * S])


def test_coarse_equal_fine_converges_in_one_iteration():
    n_steps, M = 64, 8
    m, d, dt = _setup(n_steps, M, 1)
    a_ser, raw_ser, _ = _serial(d, dt, n_steps, stepper.QOI_JOULE)
    res = parareal.parareal_sample(d, dt, n_steps, M, 1, tol=1e-14, qoi=1)
    assert res["iters"] == 1 and res["jumps"][0] == 0.0
    assert np.array_equal(res["a_end"], a_ser)


def test_tolerance_controls_accuracy():
    n_steps, M, cf = 128, 16, 8
    m, d, dt = _setup(n_steps, M, cf)
    a_ser, raw_ser, _ = _serial(d, dt, n_steps, stepper.QOI_JOULE)
    res = parareal.parareal_sample(d, dt, n_steps, M, cf, tol=1e-8, qoi=1)
    assert res["iters"] < M
    assert res["jumps"][-1] <= 1e-8
    assert np.linalg.norm(res["a_end"] - a_ser) <= 1e-6 * np.linalg.norm(a_ser)
    assert res["qoi_raw"] == pytest.approx(raw_ser, rel=1e-6)


def test_fine_map_hook_only_changes_the_evaluation_order():
    """The fine propagations of one iteration are independent: evaluating them
    in reverse order through fine_map gives bitwise the same iterates."""
    from oracle import fem, parareal, stepper
    from workloads import meshes, params
    mesh = meshes.unit_square(8)
    p = params.square_samples(1)[0]
    d = fem.Discretisation(mesh, p)
    dt, n_steps, M, cf = 0.02 / 48, 48, 6, 2
    prop = stepper.ImplicitEuler(d, dt)

    def reversed_map(slices, starts):
        out = {}
        for s, u in reversed(list(zip(slices, starts))):
            a, raw, _ = prop.run(u, n_steps // M, k0=s * (n_steps // M), qoi=stepper.QOI_JOULE)
            out[s] = (a, raw)
        return [out[s] for s in slices]

    a = parareal.parareal_sample(d, dt, n_steps, M, cf, 1e-9, stepper.QOI_JOULE)
    b = parareal.parareal_sample(d, dt, n_steps, M, cf, 1e-9, stepper.QOI_JOULE,
                                 fine_map=reversed_map)
    assert a["iters"] == b["iters"] and a["qoi_raw"] == b["qoi_raw"]
    assert np.array_equal(a["a_end"], b["a_end"])
