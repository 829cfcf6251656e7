"""Pins for the oracle's Galerkin assembly (Sec. II-A, Eq. 4-5).

Each check compares against something the oracle does not compute itself:
an independent quadrature, the 5-point finite-difference stencil, exact
integrals and conservation identities.
"""
import numpy as np
import pytest

from oracle import fem
from workloads import meshes, params


def _bary_by_solve(p):
    """Barycentric gradients by inverting the affine map (independent route)."""
    T = np.array([[1.0, p[0, 0], p[0, 1]],
                  [1.0, p[1, 0], p[1, 1]],
                  [1.0, p[2, 0], p[2, 1]]])
    C = np.linalg.inv(T)        # column i holds the coefficients of lambda_i
    return C[1:, :].T           # [3, 2] gradients


def test_element_integrals_against_quadrature():
    rng = np.random.default_rng(1)
    for _ in range(20):
        p = rng.normal(size=(3, 2))
        tri = np.array([[0, 1, 2]], dtype=np.int32)
        area, grad = fem.element_geometry(p, tri)
        # area by the shoelace formula
        e1, e2 = p[1] - p[0], p[2] - p[0]
        shoe = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
        assert area[0] == pytest.approx(shoe, rel=1e-13)
        g = _bary_by_solve(p)
        assert np.allclose(grad[0], g, rtol=1e-11, atol=1e-11 * np.abs(g).max())

        class M1:
            xy = p
            n_nodes = 3
            n_tri = 1
        M1.tri = tri
        Mf, Kf = fem.full_matrices(M1, np.array([2.5]), np.array([0.7]))
        # edge-midpoint rule integrates quadratics exactly on triangles
        mids = [(0, 1), (1, 2), (2, 0)]
        q = np.zeros((3, 3))
        for (a, b) in mids:
            lam = np.zeros(3)
            lam[a] = lam[b] = 0.5
            q += np.outer(lam, lam) * shoe / 3.0
        assert np.allclose(Mf.toarray(), 2.5 * q, rtol=1e-12, atol=0)
        kk = 0.7 * shoe * g @ g.T
        assert np.allclose(Kf.toarray(), kk, rtol=1e-10, atol=1e-12 * np.abs(kk).max())


def test_stiffness_is_five_point_stencil_on_uniform_mesh():
    nx = 8
    m = meshes.unit_square(nx)
    n = m.n_nodes
    _, Kf = fem.full_matrices(m, np.ones(m.n_tri), np.ones(m.n_tri))
    K = Kf.toarray()
    n1 = nx + 1
    for j in range(1, nx):
        for i in range(1, nx):
            k = j * n1 + i
            row = np.zeros(n)
            row[k] = 4.0
            for d in (-1, 1, -n1, n1):
                row[k + d] = -1.0
            assert np.allclose(K[k], row, atol=1e-13), (i, j)


def test_conservation_identities_annulus():
    m = meshes.annulus("5k")
    p = params.annulus_samples(1, 0)[0]
    sig, nu, *_ = fem.split_params(p, m.n_regions, m.n_phases)
    Mf, Kf = fem.full_matrices(m, sig[m.region], nu[m.region])
    area, _ = fem.element_geometry(m.xy, m.tri)
    ones = np.ones(m.n_nodes)
    # K annihilates constants (row sums zero before Dirichlet elimination)
    assert np.abs(Kf @ ones).max() <= 1e-9 * np.abs(Kf.diagonal()).max()
    # total mass = integral of sigma
    assert ones @ (Mf @ ones) == pytest.approx(np.sum(sig[m.region] * area), rel=1e-12)
    # load vectors integrate the winding: 1^T F_p = sum coef |T| over the phase
    F = fem.full_load_vectors(m)
    for ph in range(3):
        sel = m.src_phase == ph
        assert F[ph].sum() == pytest.approx(np.sum(m.src_coef[sel] * area[sel]), rel=1e-12, abs=1e-18)
    # symmetric positive definite after Dirichlet elimination
    d = fem.Discretisation(m, p)
    assert abs(d.K - d.K.T).max() == 0.0 and abs(d.M - d.M.T).max() == 0.0
    # total area of the annulus polygon approaches pi (R^2 - r^2)
    assert area.sum() == pytest.approx(np.pi * (0.1 ** 2 - 0.02 ** 2), rel=1e-3)


def test_dirichlet_elimination_and_source():
    m = meshes.unit_square(16)
    p = params.square_samples(1)[0]
    d = fem.Discretisation(m, p)
    assert d.n == 225 and d.M.shape == (225, 225)
    # source J0 sin(2 pi 50 t) on the 4x4-cell conductor: at t = 1/200 s,
    # sum r = J0 * conductor area (all conductor nodes are interior nodes)
    r = d.source(1.0 / 200.0)
    assert r.sum() == pytest.approx(p[4] * 0.25 ** 2, rel=1e-12)


class _Patch:
    """A hand-built mesh: four triangles, two source phases, one unwound
    triangle (src_phase -1), node 5 touched by no source triangle."""
    xy = np.array([[0.0, 0.0], [2.0, 0.0], [2.0, 1.0], [0.0, 3.0], [4.0, 0.0], [5.0, 5.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3], [1, 4, 2], [2, 4, 5]], dtype=np.int32)
    n_nodes = 6
    n_tri = 4
    n_phases = 2
    # |T| = 1, 3, 1, 3 (shoelace, by hand)
    src_phase = np.array([0, 0, 1, -1], dtype=np.int32)
    src_coef = np.array([1.0, 0.5, -1.0, 7.0])


def test_load_vectors_node_by_node():
    """Eq. 5 with P1 test functions: each vertex of a source triangle T gets
    coef_T |T| / 3, summed over the triangles that share it.  Values worked
    out by hand for _Patch."""
    F = fem.full_load_vectors(_Patch)
    third = 1.0 / 3.0
    expect0 = [third + 0.5, third, third + 0.5, 0.5, 0.0, 0.0]   # T0 (coef 1, |T| 1), T1 (0.5, 3)
    expect1 = [0.0, -third, -third, 0.0, -third, 0.0]            # T2 (coef -1, |T| 1)
    assert F.shape == (2, 6)
    assert np.allclose(F[0], expect0, rtol=1e-15, atol=1e-16)
    assert np.allclose(F[1], expect1, rtol=1e-15, atol=1e-16)


def test_load_vector_single_skewed_triangle():
    class Tri:
        xy = np.array([[0.0, 0.0], [3.0, 0.5], [1.0, 2.0]])   # |T| = |3*2 - 1*0.5| / 2 = 2.75
        tri = np.array([[2, 0, 1]], dtype=np.int32)            # vertex order does not matter
        n_nodes = 3
        n_tri = 1
        n_phases = 1
        src_phase = np.array([0], dtype=np.int32)
        src_coef = np.array([-1.5])
    F = fem.full_load_vectors(Tri)
    assert np.allclose(F[0], [-1.375, -1.375, -1.375], rtol=1e-15, atol=0)


def test_three_phase_currents_by_hand():
    """J_p(t) = J0 amp_p sin(2 pi f t - 2 pi p / 3 + phase_p) with P = 3 and
    nonzero phase shifts (radians), evaluated by hand at two instants:
      t = 1/600 s (2 pi f t = pi/6): arguments pi/2, 0, -pi/2;
      t = 1/200 s (2 pi f t = pi/2): arguments 5pi/6, pi/3, -pi/6."""
    m = meshes.annulus("5k")
    R = m.n_regions
    assert m.n_phases == 3
    J0, amp, ph = 2.0, [1.0, 0.9, 1.1], [np.pi / 3, np.pi / 2, 2 * np.pi / 3]
    p = np.concatenate([np.ones(R), np.ones(R), [J0], amp, ph])
    d = fem.Discretisation(m, p, freq_hz=50.0)
    assert np.allclose(d.phase_currents(1.0 / 600.0), [2.0, 0.0, -2.2], rtol=0, atol=1e-14)
    assert np.allclose(d.phase_currents(1.0 / 200.0), [1.0, 0.9 * np.sqrt(3.0), -1.1],
                       rtol=0, atol=1e-14)
    # r(t) = sum_p J_p(t) F_p: at t = 1/600 s only phases 0 and 2 contribute
    r = d.source(1.0 / 600.0)
    assert np.allclose(r, 2.0 * d.F[0] - 2.2 * d.F[2], rtol=1e-14, atol=1e-14 * np.abs(r).max())


# ---------------------------------------------------------------- annulus closed forms
# On the annulus meshes with one material everywhere, the continuous problem
# behind Eq. 2-5 (Sec. II-A) is radially symmetric and has closed forms: the
# steady state of a uniform current density, and the slowest decaying mode.
# The oracle's P1 matrices must reach both at second order in the mesh size
# (nodes lie on the circles; the 80k mesh halves both spacings of the 20k one).
R_IN, R_OUT = 0.02, 0.10
NU_ANN = 1.0 / (4e-7 * np.pi * 100.0)        # a relative permeability of 100
SIGMA_ANN, J_ANN = 3.0e7, 1.0e6


def _uniform_annulus(kind, sigma, j0, all_source):
    from dataclasses import replace
    m = meshes.annulus(kind)
    kw = {"region": np.zeros_like(m.region)}
    if all_source:
        kw.update(src_phase=np.zeros_like(m.src_phase), src_coef=np.ones_like(m.src_coef))
    mm = replace(m, **kw)
    r, p = mm.n_regions, mm.n_phases
    prm = np.concatenate([np.full(r, sigma), np.full(r, NU_ANN), [j0],
                          [1.0] + [0.0] * (p - 1), [0.0] * p])
    return mm, fem.Discretisation(mm, prm)


def _steady_errors(kind):
    """-nu (1/r)(r A')' = J, A(R_IN) = A(R_OUT) = 0:
    A = -J r^2/(4 nu) + c1 ln r + c2."""
    import scipy.sparse.linalg as spla
    from scipy.integrate import quad
    c1 = J_ANN * (R_OUT ** 2 - R_IN ** 2) / (4 * NU_ANN * np.log(R_OUT / R_IN))
    c2 = J_ANN * R_IN ** 2 / (4 * NU_ANN) - c1 * np.log(R_IN)
    exact = lambda r: -J_ANN * r ** 2 / (4 * NU_ANN) + c1 * np.log(r) + c2
    dexact = lambda r: -J_ANN * r / (2 * NU_ANN) + c1 / r
    energy = 0.5 * quad(lambda r: NU_ANN * dexact(r) ** 2 * 2 * np.pi * r, R_IN, R_OUT,
                        limit=200, epsabs=0.0, epsrel=1e-13)[0]
    mm, d = _uniform_annulus(kind, 1.0, J_ANN, True)
    a = spla.spsolve(d.K.tocsc(), J_ANN * d.F[0])
    r = np.hypot(*mm.xy[d.free].T)
    nodal = np.max(np.abs(a - exact(r))) / np.max(np.abs(exact(r)))
    return nodal, (0.5 * a @ (d.K @ a) - energy) / energy


def test_annulus_steady_state_matches_the_radial_closed_form():
    """K and F (Eq. 4-5) on the annulus against the closed-form steady state
    of a uniform current density: nodal error and energy converge at second
    order, and the discrete energy lies below the exact one (Galerkin)."""
    n20, e20 = _steady_errors("20k")
    n80, e80 = _steady_errors("80k")
    assert n20 < 5e-4 and n80 < 1.2e-4
    assert 3.2 < n20 / n80 < 4.8
    assert e20 < 0 and e80 < 0
    assert 3.2 < e20 / e80 < 4.8 and abs(e80) < 2e-4


def _slowest_mode_error(kind):
    """Slowest mode exp(-lam t) R(r): R = J0(k r) Y0(k R_IN) - Y0(k r) J0(k R_IN)
    with R(R_OUT) = 0, lam = nu k^2 / sigma."""
    import scipy.sparse.linalg as spla
    from scipy.optimize import brentq
    from scipy.special import j0, y0
    f = lambda k: j0(k * R_IN) * y0(k * R_OUT) - y0(k * R_IN) * j0(k * R_OUT)
    ks = np.linspace(1.0, 200.0, 4000)
    v = f(ks)
    i = np.flatnonzero(np.sign(v[:-1]) != np.sign(v[1:]))[0]
    k1 = brentq(f, ks[i], ks[i + 1], xtol=1e-14)
    lam = NU_ANN * k1 ** 2 / SIGMA_ANN
    _, d = _uniform_annulus(kind, SIGMA_ANN, 0.0, False)
    lam_h = spla.eigsh(d.K.tocsc(), k=1, M=d.M.tocsc(), sigma=0.0, which="LM",
                       return_eigenvectors=False)[0]
    return (lam_h - lam) / lam


def test_annulus_slowest_mode_matches_the_bessel_root():
    """M and K (Eq. 4) together on the annulus: the smallest generalised
    eigenvalue of (K, M) approaches the slowest radial mode's decay rate from
    above (Rayleigh-Ritz with the consistent mass) at second order."""
    d20 = _slowest_mode_error("20k")
    d80 = _slowest_mode_error("80k")
    assert d20 > 0 and d80 > 0
    assert d80 < 1.5e-4
    assert 3.2 < d20 / d80 < 4.8
