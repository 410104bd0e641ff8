"""Pins for the oracle's multi-spin-coded random numbers (Sec. 5.4: 32 replicas
coded together draw their uniforms from an LCG re-seeded per site and sweep
by Philox; reading R18).

The LCG outputs are checked against the closed form of the recurrence
(x_n = a^n x_0 + c (a^n - 1) / (a - 1) mod 2^32, exact big-integer
arithmetic) from the Philox seed word; the sweeps keep the Metropolis rule
(beta = 0 flips everything, single-site flip frequencies follow the
acceptance law for every bit position), sample the 4x4 Boltzmann distribution
(enumeration), and population annealing with them reaches the exact 4x4 and
Kaufman 8x8 free energies.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import exact
from tests import exact_small

A, C = 1664525, 1013904223


def test_lcg_outputs_follow_the_closed_form_from_the_philox_seed():
    rng = np.random.default_rng(8)
    for _ in range(20):
        seed = int(rng.integers(0, 2 ** 63))
        k, t, group = int(rng.integers(0, 2 ** 20)), int(rng.integers(0, 2 ** 20)), int(rng.integers(0, 4000))
        colour, inst = int(rng.integers(0, 2)), int(rng.integers(0, 1000))
        ctr = [k >> 2, t, group, (5 << 28) | (colour << 27) | inst]
        x0 = int(oracle.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])[0][k & 3])
        u = oracle.msc_uniforms(seed, k, t, group, colour, inst)
        for b in range(32):
            n = b + 1
            an = pow(A, n, 2 ** 32 * (A - 1))
            want = (an * x0 + C * ((an - 1) // (A - 1))) % 2 ** 32
            assert int(u[b]) == want


def test_msc_uniforms_are_uniform_and_uncorrelated_across_bits():
    u = np.stack([oracle.msc_uniforms(77, k, 3, 1, 0, 0) for k in range(4000)]).astype(np.float64) / 2 ** 32
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
    corr = np.corrcoef(u.T)
    off = corr[~np.eye(32, dtype=bool)]
    assert np.max(np.abs(off)) < 5 / math.sqrt(4000)


def test_msc_beta_zero_flips_every_spin():
    s0 = oracle.init_spins(2, 8, 5, 0, 0, True)
    for r in (0, 13, 31, 70):
        s = s0.copy()
        oracle.msc_sweeps(2, 8, s, None, 0.0, 5, 0, r, 0, 1)
        np.testing.assert_array_equal(s, -s0)


@pytest.mark.parametrize("replica", [0, 1, 17, 31, 32, 63])
def test_msc_single_site_flip_frequency_matches_acceptance_law(replica):
    L, beta, n = 4, 0.35, 3000
    s0 = oracle.init_spins(2, L, 3, 0, 0, True)
    T = oracle.thresholds(beta, 2)
    flips = np.zeros(L * L)
    for t in range(n):
        s = s0.copy()
        oracle.msc_sweeps(2, L, s, None, beta, 9, 0, replica, t, 1)
        flips += s != s0
    # colour-0 sites are updated first, against the untouched start, and the
    # colour-1 half-sweep leaves them alone: they flip with the acceptance law
    for i in range(L * L):
        x, y = i % L, i // L
        if (x + y) % 2:
            continue
        h = sum(int(s0[j]) for j in ((y * L + (x + 1) % L), (y * L + (x - 1) % L),
                                     (((y + 1) % L) * L + x), (((y - 1) % L) * L + x)))
        dE = 2 * int(s0[i]) * h
        p = 1.0 if dE <= 0 else (int(T[dE // 4 - 1]) + 1) / 2 ** 32
        sd = math.sqrt(max(p * (1 - p), 1e-12) / n)
        assert abs(flips[i] / n - p) <= 5 * sd + 1e-12, (i, dE, flips[i] / n, p)


@pytest.mark.parametrize("replica", [0, 19, 44])
def test_msc_4x4_energy_matches_enumeration(replica):
    E_all = exact_small.ising2d_energies(4)
    beta = 0.4406868
    s = oracle.init_spins(2, 4, 2, 0, replica, True)
    n = 40000
    E = np.empty(n)
    for t in range(n):
        oracle.msc_sweeps(2, 4, s, None, beta, 2, 0, replica, t, 1)
        E[t] = oracle.observables(2, 4, s)[0]
    E = E[1000:]
    b = E[: len(E) // 50 * 50].reshape(50, -1).mean(1)
    m1, _ = exact_small.mean_energy(E_all, beta)
    assert abs(b.mean() - m1) < 4 * b.std(ddof=1) / math.sqrt(50)


def test_pa_msc_4x4_and_8x8_match_exact_free_energies():
    E_all = exact_small.ising2d_energies(4)
    betas = oracle.linear_betas(1.0, 20)
    lnZ = np.array([oracle.pa_run(2, 4, seed, 0, 2000, betas, 4, msc=True)["lnZ"] for seed in range(1, 7)])
    for i, b in enumerate(betas):
        ex = exact_small.lnZ_from_energies(E_all, b)
        assert abs(lnZ[:, i].mean() - ex) < 0.02 + 4 * lnZ[:, i].std() / math.sqrt(6)
    L = 8
    f = np.array([oracle.pa_run(2, L, seed, 0, 1000, oracle.linear_betas(1.0, 100), 5, msc=True)["lnZ"][-1] / L ** 2
                  for seed in range(1, 5)])
    assert abs(f.mean() - exact.ising2d_lnZ_per_site(L, 1.0)) < 4 * f.std(ddof=1) / 2 + 2e-4
