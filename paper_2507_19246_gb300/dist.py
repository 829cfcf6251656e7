"""Merging MLMC level records across independent GPU replicas.

Samples are independent (Sec. II-B), so a level's samples can be split over
ranks with no exchange during the solves; only the per-level moment records
{N, mean, M2} (M2 = sum of squared deviations from the mean) are combined at
the end, with the same pairwise update the library applies across batches
(Chan, Golub & LeVeque): n = na + nb, d = mb - ma, mean = ma + d nb / n,
M2 = M2a + M2b + d^2 na nb / n.  Ranks are merged in rank order so every
rank obtains bitwise the same estimate.
"""
from __future__ import annotations

import math

import numpy as np


def merge_records(a, b):
    """Pairwise merge of two level records (N, mean, M2)."""
    na, ma, m2a = a
    nb, mb, m2b = b
    if na == 0:
        return (nb, mb, m2b)
    if nb == 0:
        return (na, ma, m2a)
    n = na + nb
    d = mb - ma
    return (n, ma + d * (nb / n), m2a + m2b + d * d * (na * nb / n))


def records_from_levels(levels):
    """Library readout rows [N, mean, var] -> records (N, mean, M2)."""
    return [(float(n), float(m), float(v) * (n - 1.0) if n > 1 else 0.0) for n, m, v in levels]


def estimate(records):
    """(estimate, rmse, per-level [N, mean, var]) from merged records (Eq. 9)."""
    est, vs, rows = 0.0, 0.0, []
    for n, m, m2 in records:
        var = m2 / (n - 1.0) if n > 1 else 0.0
        rows.append((n, m, var))
        est += m
        if n > 0:
            vs += var / n
    return est, math.sqrt(vs), np.asarray(rows)


def allreduce_levels(levels, group=None):
    """Merge this rank's level readout with every other rank's (torch.distributed).

    `levels` is this rank's [n_levels][3] array from mqs_mlmc_readout; returns
    (estimate, rmse, merged [n_levels][3]) identical on every rank.
    """
    import torch.distributed as dist
    world = dist.get_world_size(group)
    mine = records_from_levels(np.asarray(levels, dtype=np.float64))
    gathered = [None] * world
    dist.all_gather_object(gathered, mine, group=group)
    merged = gathered[0]
    for r in range(1, world):
        merged = [merge_records(a, b) for a, b in zip(merged, gathered[r])]
    return estimate(merged)
