"""Pins for the oracle's implicit Euler stepper and QoIs (Eq. 6-7, Eq. 26).

Closed-form mode decay, a long-double recurrence for a forced mode, brute
force against dense Gaussian elimination and convergence to the PDE's exact
solution.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fem, stepper
from workloads import meshes, params


def _uniform_params(mesh, sigma, nu, j0=0.0):
    p = np.zeros(params.n_params(mesh.n_regions, mesh.n_phases))
    R = mesh.n_regions
    p[:R] = sigma
    p[R:2 * R] = nu
    p[2 * R] = j0
    p[2 * R + 1:2 * R + 1 + mesh.n_phases] = 1.0
    return p


def _mode(mesh, disc):
    x, y = mesh.xy[disc.free, 0], mesh.xy[disc.free, 1]
    return np.sin(np.pi * x) * np.sin(np.pi * y)


def test_lumped_mass_mode_decays_in_closed_form():
    nx, sigma, nu = 16, 3.0e6, 7.0e5
    m = meshes.unit_square(nx)
    d = fem.Discretisation(m, _uniform_params(m, sigma, nu), lumped=True)
    h = 1.0 / nx
    lam = 8.0 * nu * math.sin(math.pi * h / 2) ** 2 / (sigma * h * h)
    dt = 2.0e-3
    prop = stepper.ImplicitEuler(d, dt)
    a0 = _mode(m, d)
    a, _, _ = prop.run(a0, 25, qoi=stepper.QOI_ENERGY)
    expect = a0 * (1.0 + dt * lam) ** -25
    assert np.abs(a - expect).max() <= 1e-13 * np.abs(expect).max()


class _ModeSystem:
    """M, K of the 8x8 square and a source r(t) = g sin(w t) M v."""

    def __init__(self, v, lam, g, w, disc):
        self.M, self.K = disc.M, disc.K
        self.v, self.g, self.w = v, g, w
        self.Mv = disc.M @ v

    def source(self, t):
        return self.g * math.sin(self.w * t) * self.Mv


def _generalised_pairs(disc):
    lam, V = sla.eigh(disc.K.toarray(), disc.M.toarray())   # v^T M v = 1
    return lam, V


def test_consistent_mass_eigenpair_decay():
    m = meshes.unit_square(8)
    d = fem.Discretisation(m, _uniform_params(m, 2.0e7, params.NU0))
    lam, V = _generalised_pairs(d)
    dt = 1.0e-4
    prop = stepper.ImplicitEuler(d, dt)
    for idx in (0, 7, 30):
        a, _, _ = prop.run(V[:, idx], 12, qoi=stepper.QOI_ENERGY)
        expect = V[:, idx] * (1.0 + dt * lam[idx]) ** -12
        assert np.abs(a - expect).max() <= 1e-12 * np.abs(V[:, idx]).max(), idx


@pytest.mark.parametrize("qoi", [stepper.QOI_JOULE, stepper.QOI_ENERGY])
def test_forced_mode_against_long_double_recurrence(qoi):
    m = meshes.unit_square(8)
    d = fem.Discretisation(m, _uniform_params(m, 2.0e7, params.NU0))
    lam, V = _generalised_pairs(d)
    v, l = V[:, 3], lam[3]
    g, w, dt, N = 5.0e3, 2 * math.pi * 50.0, 2.5e-4, 40
    sysm = _ModeSystem(v, l, g, w, d)
    prop = stepper.ImplicitEuler(sysm, dt)
    a, raw, _ = prop.run(np.zeros(d.n), N, qoi=qoi)
    # c_{k+1} = (c_k + dt g sin(w t_{k+1})) / (1 + dt lam), a_k = c_k v
    LD = np.longdouble
    c = LD(0)
    terms = []
    for k in range(N):
        t = LD((k + 1) * dt)
        c_new = (c + LD(dt) * LD(g) * np.sin(LD(w) * t)) / (LD(1) + LD(dt) * LD(l))
        if qoi == stepper.QOI_JOULE:
            terms.append((c_new - c) ** 2 / LD(dt))          # v^T M v = 1
        else:
            terms.append(LD(0.5) * c_new * c_new * LD(l))   # v^T K v = lam
        c = c_new
    assert np.abs(a - float(c) * v).max() <= 1e-12 * abs(float(c)) * np.abs(v).max()
    assert raw == pytest.approx(float(sum(terms)), rel=1e-11)


def test_banded_cholesky_matches_dense_elimination():
    m = meshes.unit_square(8)
    p = params.square_samples(3)[2]
    d = fem.Discretisation(m, p)
    dt = 0.02 / 64
    prop = stepper.ImplicitEuler(d, dt)
    A = prop.A.toarray()
    a = np.zeros(d.n)
    for k in range(20):
        a_band = prop.step(a, k)
        b = (d.M @ a) / dt + d.source((k + 1) * dt)
        a_dense = np.linalg.solve(A, b)
        assert np.linalg.norm(a_band - a_dense) <= 1e-13 * np.linalg.norm(a_dense)
        a = a_band
    # the annulus: RCM keeps the periodic seam inside a narrow band
    ma = meshes.annulus("5k")
    da = fem.Discretisation(ma, params.annulus_nominal(1)[0])
    pa = stepper.ImplicitEuler(da, 1e-4)
    assert pa.solver.bandwidth <= 4 * 18          # banded, not dense
    b = np.random.default_rng(0).normal(size=da.n)
    x = pa.solver.solve(b)
    assert np.linalg.norm(pa.A @ x - b) <= 1e-12 * np.linalg.norm(b) * 1e3


def test_converges_to_the_pde_solution():
    """sigma dA/dt - nu Lap A = 0, A(0) = sin(pi x) sin(pi y):
    A(t) = exp(-2 pi^2 nu t / sigma) A(0); error O(h^2 + dt) with dt ~ h^2."""
    T, errs = 0.05, []
    for nx in (8, 16, 32):
        m = meshes.unit_square(nx)
        d = fem.Discretisation(m, _uniform_params(m, 1.0, 1.0))
        n_steps = nx * nx // 4
        prop = stepper.ImplicitEuler(d, T / n_steps)
        a0 = _mode(m, d)
        a, _, _ = prop.run(a0, n_steps, qoi=stepper.QOI_ENERGY)
        exact = math.exp(-2 * math.pi ** 2 * T) * a0
        errs.append(np.abs(a - exact).max() / np.abs(exact).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 2e-3
    assert all(1.7 < r < 2.3 for r in rates), (errs, rates)


def test_qoi_normalisation():
    assert stepper.qoi_finish(stepper.QOI_JOULE, 6.0, 3, 0.5) == 4.0
    assert stepper.qoi_finish(stepper.QOI_ENERGY, 6.0, 3, 0.5) == 2.0
