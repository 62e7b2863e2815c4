"""Seeded synthetic inputs shared by the tests, the smoke check and bench.py.

Holds no arithmetic of the method itself: only the workload recipe of the
paper's Example section (LJ liquid at reduced density 0.8442 in a cubic box,
geometric temperature ladders) and seeded random budgets / perturbations.
"""
from __future__ import annotations

import numpy as np

RHO = 0.8442


def box_length(N: int, rho: float = RHO) -> float:
    """Side of the cubic box holding N atoms at reduced density rho."""
    return (N / rho) ** (1.0 / 3.0)


def geometric_ladder(t_min: float, t_max: float, R: int) -> np.ndarray:
    """R temperatures spaced geometrically from t_min to t_max (Example section)."""
    if R == 1:
        return np.array([t_min])
    return t_min * (t_max / t_min) ** (np.arange(R) / (R - 1))


def paper_ladder(R: int, t_min: float = 0.7, ratio: float = 1.0275) -> np.ndarray:
    """The paper's ladder: T_k = 0.7 * 1.0275^k, k = 0..R-1."""
    return t_min * ratio ** np.arange(R)


def random_budgets(R: int, cycles: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Per replica and per exchange cycle a step budget drawn uniformly in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(cycles, R), dtype=np.int32)


def jittered_lattice(N: int, L: float, amp: float, seed: int, lattice: np.ndarray) -> np.ndarray:
    """lattice (N, 3) plus uniform jitter in [-amp, amp), wrapped into [0, L)."""
    rng = np.random.default_rng(seed)
    return (lattice + rng.uniform(-amp, amp, size=(N, 3))) % L


def random_temps_energies(R: int, seed: int, t_min=0.7, t_max=3.0, u_mean=-5000.0, u_sd=50.0):
    """Distinct temperatures (a shuffled geometric ladder) and Gaussian energies."""
    rng = np.random.default_rng(seed)
    T = rng.permutation(geometric_ladder(t_min, t_max, R))
    U = rng.normal(u_mean, u_sd, R)
    return T, U
