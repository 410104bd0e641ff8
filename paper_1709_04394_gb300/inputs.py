"""Seeded synthetic inputs shared by tests and benchmarks.

Holds none of the method's arithmetic: only numpy draws of spin configurations
and energy lists with the shapes of the paper's workloads (square/cubic
periodic lattices of +-1 spins; populations of integer energies that are
multiples of 4 apart, as Metropolis flips change E by multiples of 4).
"""
from __future__ import annotations

import numpy as np


def random_spins(n: int, seed: int) -> np.ndarray:
    """n independent +-1 int8 spins, each sign with probability 1/2."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)


def population_energies(R: int, n_sites: int, dim: int, seed: int, spread: float = 0.05) -> np.ndarray:
    """R integer energies in [-dim*N, dim*N], all congruent mod 4 to -dim*N,
    Gaussian around -dim*N/2 with relative width `spread` (a thermalised
    population's histogram is close to this shape)."""
    rng = np.random.default_rng(seed)
    lo = -dim * n_sites
    centre = lo / 2
    e = centre + spread * abs(lo) * rng.standard_normal(R)
    k = np.clip(np.round((e - lo) / 4), 0, dim * n_sites // 2).astype(np.int64)
    return lo + 4 * k
