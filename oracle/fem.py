"""Galerkin discretisation of the 2D eddy-current problem (oracle).

Sec. II-A, Eq. 1-5.  In 2D with A = A_z(x, y) e_z the basis functions of
Eq. 2 are w_i = N_i e_z with N_i the piecewise-linear (P1) nodal hat
functions, so that w_i . w_j = N_i N_j and curl w_i . curl w_j =
grad N_i . grad N_j.  With sigma, nu = 1/mu and J_s constant on each
triangle T the entries of Eq. 4 and Eq. 5 are exact element integrals:

    int_T N_i N_j     = |T| (1 + delta_ij) / 12
    int_T grad N_i . grad N_j = |T| grad N_i . grad N_j
    int_T N_i         = |T| / 3

Homogeneous Dirichlet nodes (A_z = 0) are removed from rows and columns.
The unknowns are the free nodes in increasing node id.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def element_geometry(xy: np.ndarray, tri: np.ndarray):
    """Area |T| and gradients of the three barycentric functions per triangle.

    Returns (area [n_tri], grad [n_tri, 3, 2]).
    """
    p1, p2, p3 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    d = (p2[:, 0] - p1[:, 0]) * (p3[:, 1] - p1[:, 1]) - \
        (p3[:, 0] - p1[:, 0]) * (p2[:, 1] - p1[:, 1])          # 2 * signed area
    grad = np.empty((tri.shape[0], 3, 2))
    grad[:, 0, 0] = (p2[:, 1] - p3[:, 1]) / d
    grad[:, 0, 1] = (p3[:, 0] - p2[:, 0]) / d
    grad[:, 1, 0] = (p3[:, 1] - p1[:, 1]) / d
    grad[:, 1, 1] = (p1[:, 0] - p3[:, 0]) / d
    grad[:, 2, 0] = (p1[:, 1] - p2[:, 1]) / d
    grad[:, 2, 1] = (p2[:, 0] - p1[:, 0]) / d
    return 0.5 * np.abs(d), grad


def _scatter(tri, vals_e, n):
    """Sum 3x3 element blocks vals_e [n_tri, 3, 3] into an n x n CSR matrix."""
    rows = np.repeat(tri, 3, axis=1).ravel()
    cols = np.tile(tri, (1, 3)).ravel()
    return sp.csr_matrix((vals_e.ravel(), (rows, cols)), shape=(n, n))


def full_matrices(mesh, sigma_e: np.ndarray, nu_e: np.ndarray, lumped: bool = False):
    """M and K of Eq. 4 over all nodes (before Dirichlet elimination).

    sigma_e, nu_e: per-triangle conductivity and reluctivity.
    lumped=True replaces the consistent mass by its row sums (used only by the
    closed-form eigenmode check; the method itself uses the consistent mass).
    """
    area, grad = element_geometry(mesh.xy, mesh.tri)
    n = mesh.n_nodes
    gg = np.einsum("eik,ejk->eij", grad, grad)                    # grad N_i . grad N_j
    ke = (nu_e * area)[:, None, None] * gg
    if lumped:
        me = np.zeros((mesh.n_tri, 3, 3))
        for i in range(3):
            me[:, i, i] = sigma_e * area / 3.0
    else:
        base = (np.ones((3, 3)) + np.eye(3)) / 12.0                # (1 + delta_ij)/12
        me = (sigma_e * area)[:, None, None] * base[None, :, :]
    return _scatter(mesh.tri, me, n), _scatter(mesh.tri, ke, n)


def full_load_vectors(mesh):
    """Per-phase load vectors F_p (Eq. 5 with unit current density), all nodes.

    F_p[i] = sum over triangles T of phase p of coef_T * |T| / 3 for i in T,
    so that r(t) = sum_p J_p(t) F_p for phase current densities J_p(t).
    """
    area, _ = element_geometry(mesh.xy, mesh.tri)
    F = np.zeros((mesh.n_phases, mesh.n_nodes))
    for p in range(mesh.n_phases):
        sel = mesh.src_phase == p
        w = mesh.src_coef[sel] * area[sel] / 3.0
        for loc in range(3):
            np.add.at(F[p], mesh.tri[sel, loc], w)
    return F


def free_nodes(mesh) -> np.ndarray:
    return np.flatnonzero(mesh.dirichlet == 0)


def split_params(params: np.ndarray, n_regions: int, n_phases: int):
    """Unpack one sample's parameter vector.

    Layout: sigma[R], nu[R], J0, amp[P], phase[P].
    """
    R, P = n_regions, n_phases
    sigma = params[0:R]
    nu = params[R:2 * R]
    j0 = params[2 * R]
    amp = params[2 * R + 1:2 * R + 1 + P]
    phase = params[2 * R + 1 + P:2 * R + 1 + 2 * P]
    return sigma, nu, j0, amp, phase


class Discretisation:
    """M, K and the source of one sample on one mesh, Dirichlet eliminated.

    Attributes: M, K (CSR, n_free x n_free), F (n_phases x n_free), and the
    sample's source parameters.  ``source(t)`` returns r(t) of Eq. 5:

        J_p(t) = J0 * amp_p * sin(2 pi f t - 2 pi p / P + phase_p)
        r(t)   = sum_p J_p(t) F_p
    """

    def __init__(self, mesh, params, freq_hz: float = 50.0, lumped: bool = False):
        sigma, nu, j0, amp, phase = split_params(np.asarray(params, dtype=np.float64),
                                                 mesh.n_regions, mesh.n_phases)
        self.mesh = mesh
        self.free = free_nodes(mesh)
        Mf, Kf = full_matrices(mesh, sigma[mesh.region], nu[mesh.region], lumped=lumped)
        sel = self.free
        self.M = Mf[sel][:, sel].tocsr()
        self.K = Kf[sel][:, sel].tocsr()
        self.F = full_load_vectors(mesh)[:, sel]
        self.j0, self.amp, self.phase = j0, amp, phase
        self.freq = freq_hz
        self.n_phases = mesh.n_phases

    @property
    def n(self) -> int:
        return self.M.shape[0]

    def phase_currents(self, t: float) -> np.ndarray:
        P = self.n_phases
        p = np.arange(P)
        arg = 2.0 * np.pi * self.freq * t - 2.0 * np.pi * p / P + self.phase
        return self.j0 * self.amp * np.sin(arg)

    def source(self, t: float) -> np.ndarray:
        return self.phase_currents(t) @ self.F
