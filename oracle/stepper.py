"""Implicit Euler time stepping and quantities of interest (oracle).

Sec. II-A, Eq. 6-7: with the backward difference of Eq. 6 the semi-discrete
system M da/dt + K a = r (Eq. 3) becomes, per step,

    (M/dt + K) a_{k+1} = (M/dt) a_k + r(t_{k+1}),   t_{k+1} = t0 + (k+1) dt.

The system matrix is factored once per (sample, step size) by a banded
Cholesky decomposition after a reverse Cuthill-McKee reordering and the two
triangular solves are repeated every step.

Quantities of interest, accumulated over the steps of a run:

* joule loss, Eq. 26 with the backward difference of Eq. 6 for da/dt and the
  rectangle rule in time:
      Q = (1/T) sum_{k=0}^{N-1} dt * (da_k/dt)^T M (da_k/dt),  da_k = a_{k+1} - a_k
        = (1/T) sum_k da_k^T M da_k / dt,   T = N dt;
* time-averaged magnetic energy per unit length:
      Q = (1/N) sum_{k=1}^{N} 1/2 a_k^T K a_k.

``run`` returns the raw sum S of the per-step terms (S/T resp. S/N is Q) so
that Parareal slices can add their partial sums.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
from scipy.linalg import cho_solve_banded, cholesky_banded
from scipy.sparse.csgraph import reverse_cuthill_mckee

QOI_ENERGY = 0
QOI_JOULE = 1


class BandedCholesky:
    """Direct SPD solver: RCM ordering, LAPACK banded Cholesky factor."""

    def __init__(self, A: sp.spmatrix):
        A = sp.csr_matrix(A)
        self.perm = reverse_cuthill_mckee(A, symmetric_mode=True)
        Ap = A[self.perm][:, self.perm].tocoo()
        n = A.shape[0]
        upper = Ap.col >= Ap.row
        r, c, v = Ap.row[upper], Ap.col[upper], Ap.data[upper]
        self.bandwidth = int((c - r).max()) if r.size else 0
        u = self.bandwidth
        ab = np.zeros((u + 1, n))
        ab[u + r - c, c] = v                      # LAPACK upper band storage
        self.factor = cholesky_banded(ab, lower=False)
        self.n = n

    def solve(self, b: np.ndarray) -> np.ndarray:
        x = np.empty_like(b)
        x[self.perm] = cho_solve_banded((self.factor, False), b[self.perm])
        return x


def qoi_finish(kind: int, raw_sum: float, n_steps: int, dt: float) -> float:
    """Normalise the raw per-step sum: joule by T = N dt, energy by N."""
    if kind == QOI_JOULE:
        return raw_sum / (n_steps * dt)
    return raw_sum / n_steps


class ImplicitEuler:
    """Implicit Euler propagator for one discretisation and one step size."""

    def __init__(self, disc, dt: float, t0: float = 0.0):
        self.disc = disc
        self.dt = dt
        self.t0 = t0
        self.A = (disc.M / dt + disc.K).tocsr()
        self.solver = BandedCholesky(self.A)

    def step(self, a: np.ndarray, k: int) -> np.ndarray:
        """a_{k+1} from a_k; k is the global step index (t_{k+1} = t0 + (k+1) dt)."""
        t = self.t0 + (k + 1) * self.dt
        b = (self.disc.M @ a) / self.dt + self.disc.source(t)
        return self.solver.solve(b)

    def run(self, a0: np.ndarray, n_steps: int, k0: int = 0, qoi: int = QOI_JOULE,
            keep_states: bool = False):
        """n_steps steps from a0 starting at global step k0.

        Returns (a_end, raw QoI sum over these steps, states or None).
        """
        a = np.array(a0, dtype=np.float64, copy=True)
        terms = []
        states = [a.copy()] if keep_states else None
        for k in range(k0, k0 + n_steps):
            a_new = self.step(a, k)
            if qoi == QOI_JOULE:
                d = a_new - a
                terms.append(float(d @ (self.disc.M @ d)) / self.dt)
            else:
                terms.append(0.5 * float(a_new @ (self.disc.K @ a_new)))
            a = a_new
            if keep_states:
                states.append(a.copy())
        return a, math.fsum(terms), states


def solve_sample(mesh, params, dt: float, n_steps: int, qoi: int = QOI_JOULE,
                 t0: float = 0.0, freq_hz: float = 50.0, keep_states: bool = False):
    """Serial implicit Euler for one sample from a(t0) = 0.

    Returns (Q, a_end, states or None).
    """
    from .fem import Discretisation
    disc = Discretisation(mesh, params, freq_hz=freq_hz)
    prop = ImplicitEuler(disc, dt, t0)
    a_end, raw, states = prop.run(np.zeros(disc.n), n_steps, 0, qoi, keep_states)
    return qoi_finish(qoi, raw, n_steps, dt), a_end, states
