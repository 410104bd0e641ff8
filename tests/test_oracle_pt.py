"""Pins for the oracle's parallel tempering (Sec. 5.1, Eq. (10)): equal
temperatures always exchange; the label maps stay permutations; frozen
configurations exchange with probability min(1, exp((b_i - b_j)(E_i - E_j)));
each temperature samples the Boltzmann distribution (4x4, enumeration)."""
import math

import numpy as np
import pytest

import oracle
from tests import exact_small


def test_equal_temperatures_always_exchange():
    betas = np.full(5, 0.4)
    _, rep, acc, _ = oracle.pt_run(2, 4, 3, 0, betas, 1, 1)
    np.testing.assert_array_equal(rep, [1, 0, 3, 2, 4])   # round 0: pairs (0,1), (2,3)
    np.testing.assert_array_equal(acc, [1, 0, 1, 0])
    _, rep, acc, _ = oracle.pt_run(2, 4, 3, 0, betas, 1, 1, round0=1)
    np.testing.assert_array_equal(rep, [0, 2, 1, 4, 3])   # round 1: pairs (1,2), (3,4)


def test_labels_remain_a_permutation():
    s, rep, acc, E = oracle.pt_run(3, 4, 9, 2, np.linspace(0.1, 1.2, 7), 2, 40, J=oracle.couplings(4, 9, 2))
    assert sorted(rep.tolist()) == list(range(7))
    assert acc.max() <= 20
    for r in range(7):
        assert E[r] == oracle.observables(3, 4, s[r], oracle.couplings(4, 9, 2))[0]


def test_frozen_pair_exchanges_with_the_metropolis_probability():
    # theta = 0: no sweeps, energies frozen; track how often the low-energy
    # configuration leaves the colder temperature
    L, N = 4, 16
    up = np.ones(N, dtype=np.int8)
    other = np.array([1, -1] * 8, dtype=np.int8)  # rows alternate: E = 0
    betas = np.array([0.30, 0.33])
    E_up, E_other = -2 * N, oracle.observables(2, L, other)[0]
    p = math.exp(-(betas[1] - betas[0]) * (E_other - E_up))
    spins = np.stack([other, up])  # config 1 (low E) starts at the colder temperature 1
    rep = np.array([0, 1], dtype=np.uint32)
    acc = np.zeros(1, dtype=np.uint32)
    tries = moves = 0
    for rnd in range(0, 16000, 2):
        cold_is_up = rep[1] == 1
        spins, rep, acc, _ = oracle.pt_run(2, L, 5, 0, betas, 0, 1, spins=spins, rep_of=rep, accepted=acc, round0=rnd)
        if cold_is_up:
            tries += 1
            moves += rep[1] != 1
        else:
            assert rep[1] == 1  # a high-energy configuration at the cold end always moves up
    assert abs(moves / tries - p) < 5 * math.sqrt(p * (1 - p) / tries)


def test_each_temperature_samples_boltzmann_4x4():
    E_all = exact_small.ising2d_energies(4)
    betas = np.array([0.2, 0.35, 0.5, 0.7])
    spins, rep, acc = None, None, None
    samples = [[] for _ in betas]
    for step in range(20000):
        spins, rep, acc, E = oracle.pt_run(2, 4, 17, 0, betas, 1, 1, spins=spins, rep_of=rep, accepted=acc,
                                           t0=step, round0=step)
        if step >= 500:
            for k in range(4):
                samples[k].append(E[rep[k]])
    for k, b in enumerate(betas):
        x = np.array(samples[k], dtype=np.float64)
        m1, _ = exact_small.mean_energy(E_all, b)
        bins = x[: len(x) // 40 * 40].reshape(40, -1).mean(1)
        err = bins.std(ddof=1) / math.sqrt(40)
        assert abs(x.mean() - m1) < 4.5 * err, (b, x.mean(), m1, err)
    assert acc.min() > 0
