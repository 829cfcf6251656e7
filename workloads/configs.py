"""Standard synthetic workloads, named by what they are.

Frequencies and step sizes follow a 50 Hz supply: one electrical period is
20 ms and level l of the time hierarchy uses dt_l = period / (64 * 2**l).
"""
from __future__ import annotations

from dataclasses import dataclass

FREQ_HZ = 50.0
PERIOD = 1.0 / FREQ_HZ

QOI_ENERGY = 0    # time-averaged magnetic energy, (1/N) sum_k 1/2 a_k^T K a_k
QOI_JOULE = 1     # mean joule loss over [0, T]


def level_steps(periods: int, level: int, base: int = 64) -> int:
    """Implicit-Euler steps of level l over `periods` periods (dt = period/(base 2^l))."""
    return periods * base * (2 ** level)


def level_dt(level: int, base: int = 64) -> float:
    return PERIOD / (base * (2 ** level))


@dataclass(frozen=True)
class MCSquare:
    """Plain Monte Carlo on the 16x16 unit square, FP64: 32 samples, 64 steps
    over one period, magnetic-energy QoI."""
    mesh: str = "square16"
    n_samples: int = 32
    n_steps: int = 64
    t_end: float = PERIOD
    qoi: int = QOI_ENERGY


@dataclass(frozen=True)
class PararealAnnulus:
    """Parareal on one nominal sample of the 20k-node annulus, FP64: fine
    dt = period/512 over 8 periods (4096 steps), coarse dt = 64 fine, 64 slices,
    relative jump tolerance 1e-8, joule-loss QoI."""
    mesh: str = "annulus20k"
    periods: int = 8
    fine_per_period: int = 512
    coarse_factor: int = 64
    n_slices: int = 64
    tol: float = 1e-8
    qoi: int = QOI_JOULE

    @property
    def n_steps(self) -> int:
        return self.periods * self.fine_per_period

    @property
    def dt(self) -> float:
        return PERIOD / self.fine_per_period


@dataclass(frozen=True)
class MLMCAnnulus:
    """MLMC in time on the 20k-node annulus: 4 levels, dt_l = period/(64 2^l)
    over 4 periods, N_l = 4096/1024/256/64, 20 random inputs, joule-loss QoI,
    FP32 PCG with FP64 iterative refinement."""
    mesh: str = "annulus20k"
    periods: int = 4
    n_per_level: tuple = (4096, 1024, 256, 64)
    qoi: int = QOI_JOULE

    @property
    def n_levels(self) -> int:
        return len(self.n_per_level)

    def steps(self, level: int) -> int:
        return level_steps(self.periods, level)

    def solve_steps(self) -> int:
        """Implicit-Euler solve-steps of one estimate (both solves of a pair)."""
        tot = 0
        for l, n in enumerate(self.n_per_level):
            tot += n * self.steps(l)
            if l > 0:
                tot += n * self.steps(l - 1)
        return tot


@dataclass(frozen=True)
class MLMCPararealAnnulus:
    """MLMC + Parareal on the 80k-node annulus: 5 levels over 8 periods,
    N_l = 8192/2048/512/128/32; the finest level runs Parareal with 32 slices
    and the level-2 step as coarse propagator."""
    mesh: str = "annulus80k"
    periods: int = 8
    n_per_level: tuple = (8192, 2048, 512, 128, 32)
    parareal_slices: int = 32
    coarse_level: int = 2
    qoi: int = QOI_JOULE


MC_SQUARE = MCSquare()
PARAREAL_ANNULUS = PararealAnnulus()
MLMC_ANNULUS = MLMCAnnulus()
MLMC_PARAREAL_ANNULUS = MLMCPararealAnnulus()
