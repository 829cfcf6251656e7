"""Parareal (oracle), Sec. II-C, Eq. 12.

The interval [T_0, T_M] is cut into M slices of S fine steps each; slice s
covers [T_s, T_{s+1}].  U[s] is the initial value used for slice s
(U[0] = a(T_0) never changes).  F_s propagates slice s with the fine step
dt_F, C_s with the coarse step dt_C = coarse_factor * dt_F.

    k = 0:  U[s+1] = C_s(U[s]) for s = 0 .. M-2 (sequential coarse sweep)
    k >= 1: E[s] = F_s(U[s])            for s = k-1 .. M-1   (independent)
            for s = k-1 .. M-2 (sequential):
                G_new   = C_s(U[s])                           (U[s] of iteration k)
                U[s+1]  = E[s] + (G_new - G_old[s])           (Eq. 12)
                G_old[s] = G_new

After iteration k the slice starts U[0..k] equal the serial fine solution
(up to round-off; exactly, because G_new == G_old for an unchanged input),
so iteration k runs the fine propagator on M-k+1 slices and the coarse one
on M-k slices, as in Eq. 13-14.  Stopping rule (the paper only asks for the
interface discontinuities to reach a tolerance): after iteration k,

    max_s ||U[s]^k - U[s]^{k-1}||_2 / max_s ||U[s]^k||_2 <= tol,  or k = M.

The quantity of interest is the sum of the per-slice partial sums of the
most recent fine run of every slice.
"""
from __future__ import annotations

import math

import numpy as np


def parareal(fine, coarse, u0: np.ndarray, n_slices: int, tol: float, max_iter: int = None,
             fine_map=None):
    """Run Parareal.

    fine(s, u)   -> (u_end, qoi_partial)  fine propagation of slice s from u
    coarse(s, u) -> u_end                 coarse propagation of slice s from u
    fine_map(slices, starts) -> [(u_end, qoi_partial)]: how the independent
        fine propagations of one iteration are evaluated (default: one after
        the other with `fine`; a process pool may run them on several cores,
        as the method intends -- the arithmetic of each is the same)
    Returns dict(iters, a_end, qoi_raw, U (slice starts), jumps (per iteration),
                 fine_slices (fine solves executed), coarse_slices).
    """
    M = n_slices
    if max_iter is None:
        max_iter = M
    U = [np.array(u0, dtype=np.float64)] + [None] * (M - 1)
    G_old = [None] * M
    n_coarse = 0
    for s in range(M - 1):
        G_old[s] = coarse(s, U[s])
        n_coarse += 1
        U[s + 1] = G_old[s]
    E = [None] * M
    q = [0.0] * M
    jumps = []
    n_fine = 0
    k = 0
    for k in range(1, max_iter + 1):
        slices = list(range(k - 1, M))
        if fine_map is None:
            results = [fine(s, U[s]) for s in slices]
        else:
            results = fine_map(slices, [U[s] for s in slices])
        for s, (e, qs) in zip(slices, results):
            E[s], q[s] = e, qs
            n_fine += 1
        U_prev = [u.copy() for u in U]
        for s in range(k - 1, M - 1):
            G_new = coarse(s, U[s])
            n_coarse += 1
            U[s + 1] = E[s] + (G_new - G_old[s])
            G_old[s] = G_new
        num = max(float(np.linalg.norm(U[s] - U_prev[s])) for s in range(M))
        den = max(float(np.linalg.norm(U[s])) for s in range(M))
        jump = num / den if den > 0.0 else num
        jumps.append(jump)
        if jump <= tol or k >= M:
            break
    return dict(iters=k, a_end=E[M - 1], qoi_raw=math.fsum(q), U=U, jumps=jumps,
                fine_slices=n_fine, coarse_slices=n_coarse)


def parareal_sample(disc, dt_fine: float, n_steps: int, n_slices: int, coarse_factor: int,
                    tol: float, qoi: int, t0: float = 0.0, max_iter: int = None,
                    fine_map=None):
    """Parareal for one sample with implicit-Euler fine and coarse propagators.

    Slice s starts at global fine step s*S (S = n_steps / n_slices) and the
    coarse propagator takes S / coarse_factor steps of coarse_factor * dt_fine.
    fine_map: see parareal(); it receives slice indices and start states and
    must apply the same fine propagator (dt_fine, S steps from step s*S).
    """
    from .stepper import ImplicitEuler
    if n_steps % n_slices or (n_steps // n_slices) % coarse_factor:
        raise ValueError("slices must hold a whole number of coarse steps")
    S = n_steps // n_slices
    Sc = S // coarse_factor
    fine_p = ImplicitEuler(disc, dt_fine, t0)
    coarse_p = ImplicitEuler(disc, dt_fine * coarse_factor, t0)

    def fine(s, u):
        a, raw, _ = fine_p.run(u, S, k0=s * S, qoi=qoi)
        return a, raw

    def coarse(s, u):
        a, _, _ = coarse_p.run(u, Sc, k0=s * Sc, qoi=qoi)
        return a

    return parareal(fine, coarse, np.zeros(disc.n), n_slices, tol, max_iter, fine_map)
