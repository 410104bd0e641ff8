"""Brute-force exact results for tiny lattices (test pins, independent of both the
oracle and the CUDA library): full enumeration and transfer matrices."""
from __future__ import annotations

import math

import numpy as np


def all_states(n: int) -> np.ndarray:
    st = np.arange(2 ** n, dtype=np.int64)
    return (1 - 2 * ((st[:, None] >> np.arange(n)) & 1)).astype(np.int64)


def ising2d_energies(L: int) -> np.ndarray:
    """Energies E = -sum_<ij> s_i s_j of all 2^(L*L) periodic L x L states (state bit i = site i)."""
    s = all_states(L * L).reshape(-1, L, L)
    return -(s * np.roll(s, 1, axis=1)).sum((1, 2)) - (s * np.roll(s, 1, axis=2)).sum((1, 2))


def ea3d_energies(L: int, J: np.ndarray) -> np.ndarray:
    """Energies of all states of an L^3 periodic lattice with forward couplings J[site, mu]."""
    N = L ** 3
    s = all_states(N)
    E = np.zeros(s.shape[0], dtype=np.int64)
    for site in range(N):
        x, y, z = site % L, (site // L) % L, site // (L * L)
        for mu, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            nb = (((z + dz) % L) * L + (y + dy) % L) * L + (x + dx) % L
            E -= int(J[site, mu]) * s[:, site] * s[:, nb]
    return E


def lnZ_from_energies(E: np.ndarray, beta: float) -> float:
    e0 = E.min()
    return -beta * float(e0) + math.log(float(np.sum(np.exp(-beta * (E - e0).astype(np.float64)))))


def mean_energy(E: np.ndarray, beta: float):
    w = np.exp(-beta * (E - E.min()).astype(np.float64))
    w /= w.sum()
    m1 = float(np.sum(w * E))
    m2 = float(np.sum(w * E.astype(np.float64) ** 2))
    return m1, m2


def ising2d_lnZ_transfer(L: int, beta: float) -> float:
    """ln Z of the periodic L x L Ising model by the row-to-row transfer matrix."""
    rows = all_states(L)  # [2^L, L]
    h_in = (rows * np.roll(rows, 1, axis=1)).sum(1).astype(np.float64)
    inter = rows.astype(np.float64) @ rows.T.astype(np.float64)
    logT = beta * (0.5 * h_in[:, None] + inter + 0.5 * h_in[None, :])
    shift = logT.max()
    lam = np.linalg.eigvalsh(np.exp(logT - shift))
    lmax = np.max(np.abs(lam))
    return L * (shift + math.log(lmax)) + math.log(float(np.sum((lam / lmax) ** L)))
