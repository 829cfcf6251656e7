"""Seeded sample parameters xi for Monte Carlo / MLMC runs.

Every random input is drawn from a counter-based generator keyed by
(seed, level, sample index, draw slot), so that any sample of any level can be
regenerated on its own and the draws do not depend on batch composition.  The
generator is SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a hash: the key words are absorbed one
at a time by adding the golden-ratio increment and applying the SplitMix64
finaliser.  Uniforms take the top 53 bits; normals use the Box-Muller
transform on two uniforms.

The parameter vector of one sample has the layout the C-ABI and the oracle
both read:

    [sigma_0 .. sigma_{R-1}, nu_0 .. nu_{R-1}, J0, amp_0 .. amp_{P-1},
     phase_0 .. phase_{P-1}]

with R material regions and P source phases (n_params = 2R + 1 + 2P).
"""
from __future__ import annotations

import numpy as np

MU0 = 4.0e-7 * np.pi          # vacuum permeability (H/m), the pre-2019 exact value
NU0 = 1.0 / MU0               # reluctivity of air, 795774.7154594767 m/H
SIGMA_FLOOR = 1.0e-6          # S/m, stands in for sigma = 0 in non-conductors
DEFAULT_SEED = 20250725

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _fmix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def hash_u64(seed, level, sample, slot) -> np.ndarray:
    """SplitMix64 hash of the key (seed, level, sample, slot); broadcasts."""
    with np.errstate(over="ignore"):
        z = np.asarray(seed, dtype=np.uint64).copy()
        for w in (level, sample, slot):
            z = _fmix(z + _GOLDEN * (np.asarray(w, dtype=np.uint64) + np.uint64(1)))
    return z


def uniform01(seed, level, sample, slot) -> np.ndarray:
    """Uniform on [0, 1) from the top 53 bits of the hash."""
    return (hash_u64(seed, level, sample, slot) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal(seed, level, sample, q) -> np.ndarray:
    """Standard normal number q of a sample: Box-Muller on slots (2q, 2q+1)."""
    q = np.asarray(q, dtype=np.uint64)
    u1 = 1.0 - uniform01(seed, level, sample, np.uint64(2) * q)          # (0, 1]
    u2 = uniform01(seed, level, sample, np.uint64(2) * q + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def lognormal_mean_cv(mean, cv, z):
    """Lognormal with the given mean and coefficient of variation from N(0,1) z."""
    s2 = np.log1p(cv * cv)
    return np.exp(np.log(mean) - 0.5 * s2 + np.sqrt(s2) * z)


def n_params(n_regions: int, n_phases: int) -> int:
    return 2 * n_regions + 1 + 2 * n_phases


def square_samples(n: int, seed: int = DEFAULT_SEED, level: int = 0, first: int = 0) -> np.ndarray:
    """Unit-square Monte Carlo parameters, [n, 7] (R = 2, P = 1).

    sigma_conductor = 5.8e7 (1 + 0.1 U(-1, 1)), J0 = 1e6 (1 + 0.05 N(0, 1));
    background sigma = 1e-6, nu = 1/mu0 everywhere, amplitude 1, phase 0.
    """
    k = np.arange(first, first + n, dtype=np.uint64)
    u = 2.0 * uniform01(seed, level, k, 100) - 1.0
    z = normal(seed, level, k, 0)
    p = np.zeros((n, n_params(2, 1)))
    p[:, 0] = SIGMA_FLOOR
    p[:, 1] = 5.8e7 * (1.0 + 0.1 * u)
    p[:, 2] = NU0
    p[:, 3] = NU0
    p[:, 4] = 1.0e6 * (1.0 + 0.05 * z)
    p[:, 5] = 1.0
    p[:, 6] = 0.0
    return p


# Nominal annulus materials per region (rotor iron, bars, gap, stator iron, coils A/B/C).
ANNULUS_SIGMA = np.array([SIGMA_FLOOR, 3.5e7, SIGMA_FLOOR, SIGMA_FLOOR,
                          SIGMA_FLOOR, SIGMA_FLOOR, SIGMA_FLOOR])
ANNULUS_NU = np.array([NU0 / 1000.0, NU0, NU0, NU0 / 1000.0, NU0, NU0, NU0])
ANNULUS_J0 = 3.0e6   # A/m^2


def annulus_nominal(n: int = 1) -> np.ndarray:
    """Nominal annulus parameters ([n, 21]): no randomness."""
    p = np.zeros((n, n_params(7, 3)))
    p[:, 0:7] = ANNULUS_SIGMA
    p[:, 7:14] = ANNULUS_NU
    p[:, 14] = ANNULUS_J0
    p[:, 15:18] = 1.0
    p[:, 18:21] = 0.0
    return p


def annulus_samples(n: int, level: int, seed: int = DEFAULT_SEED, first: int = 0,
                    cv: float = 0.10) -> np.ndarray:
    """Annulus MLMC parameters ([n, 21]), 20 random inputs per sample.

    Per region sigma_r and nu_r lognormal with mean = nominal and CV 10%;
    per phase amplitude N(1, 0.05) and phase shift N(0, 2 degrees); J0 fixed.
    Normal draw q: 0..6 sigma, 7..13 nu, 14..16 amplitude, 17..19 phase.
    """
    k = np.arange(first, first + n, dtype=np.uint64)[:, None]
    q = np.arange(20, dtype=np.uint64)[None, :]
    z = normal(seed, level, k, q)
    p = np.zeros((n, n_params(7, 3)))
    p[:, 0:7] = lognormal_mean_cv(ANNULUS_SIGMA[None, :], cv, z[:, 0:7])
    p[:, 7:14] = lognormal_mean_cv(ANNULUS_NU[None, :], cv, z[:, 7:14])
    p[:, 14] = ANNULUS_J0
    p[:, 15:18] = 1.0 + 0.05 * z[:, 14:17]
    p[:, 18:21] = np.deg2rad(2.0) * z[:, 17:20]
    return p
