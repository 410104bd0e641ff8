"""Pins for the oracle's double-checkerboard sweeps with k hits per tile
(Sec. 3.1, Fig. 5 right, the multi-hit variant).

The law of the state after a round is fixed by the order the paper gives:
tiles of one coarse colour first, each swept k times with the rest of the
lattice held fixed, then the other coarse colour. On a 4 x 4 lattice with
2 x 2 tiles that law is computed here exactly, by applying each single-site
Metropolis kernel to a probability vector over all 2^16 states, and the
oracle's empirical site magnetisations over many seeds must agree with it;
the plain checkerboard order gives a law far outside the error bars, so the
test sees the order.
"""
import numpy as np
import pytest

import oracle

L4 = 4
N4 = L4 * L4
STATES = np.arange(1 << N4)
SPINS = (1 - 2 * ((STATES[:, None] >> np.arange(N4)) & 1)).astype(np.int64)  # bit 1 = spin down


def _neighbours(i):
    x, y = i % L4, i // L4
    return [y * L4 + (x + 1) % L4, y * L4 + (x - 1) % L4, ((y + 1) % L4) * L4 + x, ((y - 1) % L4) * L4 + x]


def _site_kernel(dist, i, T):
    # one Metropolis update of site i: flip with probability 1 (dE <= 0) or
    # (T(dE) + 1) / 2^32, the law of the integer comparison u <= T(dE)
    h = SPINS[:, _neighbours(i)].sum(1)
    dE = 2 * SPINS[:, i] * h
    pf = np.ones(STATES.size)
    for m in (1, 2):
        pf[dE == 4 * m] = (int(T[m - 1]) + 1) / 2.0 ** 32
    b = 1 << i
    return dist * (1 - pf) + dist[STATES ^ b] * pf[STATES ^ b]


def _exact_law(start, beta, order):
    T = oracle.thresholds(beta, 2)
    d = np.zeros(STATES.size)
    d[start] = 1.0
    for i in order:
        d = _site_kernel(d, i, T)
    return d


def _dcb_order(tile, k, rounds):
    order = []
    for _ in range(rounds):
        for coarse in (0, 1):
            for _j in range(k):
                for c in (0, 1):
                    order += [i for i in range(N4) if (i % L4 + i // L4) % 2 == c
                              and ((i % L4) // tile + (i // L4) // tile) % 2 == coarse]
    return order


def _plain_order(sweeps):
    return [i for _ in range(sweeps) for c in (0, 1) for i in range(N4) if (i % L4 + i // L4) % 2 == c]


@pytest.mark.parametrize("k,rounds", [(2, 1), (1, 2)])
def test_dcb_round_law_matches_exact_4x4(k, rounds):
    beta, n = 0.5, 20000
    s0 = np.random.default_rng(0).choice([-1, 1], N4).astype(np.int8)
    start = int(sum(((1 - int(s0[i])) // 2) << i for i in range(N4)))
    exact = _exact_law(start, beta, _dcb_order(2, k, rounds)) @ SPINS
    plain = _exact_law(start, beta, _plain_order(k * rounds)) @ SPINS
    acc = np.zeros(N4)
    for seed in range(1, n + 1):
        s = s0.copy()
        oracle.dcb_sweeps(L4, 2, s, beta, seed, 0, 0, 0, k, rounds)
        acc += s
    mean = acc / n
    sigma = np.sqrt(np.maximum(1 - exact ** 2, 1e-12) / n)
    assert np.max(np.abs(mean - exact) / sigma) < 5.0
    assert np.max(np.abs(plain - exact) / sigma) > 20.0  # the order is visible


def test_dcb_beta_zero_flips_every_site_on_every_visit():
    L = 16
    s0 = oracle.init_spins(2, L, 3, 0, 0, True)
    for k, rounds in ((1, 1), (3, 1), (2, 2)):
        s = s0.copy()
        oracle.dcb_sweeps(L, 4, s, 0.0, 3, 0, 0, 0, k, rounds)
        np.testing.assert_array_equal(s, s0 * (-1) ** (k * rounds))


def test_dcb_zero_temperature_keeps_ground_state_and_heals_defects():
    L = 8
    s = np.ones(L * L, dtype=np.int8)
    oracle.dcb_sweeps(L, 2, s, 50.0, 1, 0, 0, 0, 3, 2)
    np.testing.assert_array_equal(s, np.ones(L * L, dtype=np.int8))
    # isolated defects have dE = -8 and are flipped on their first visit
    s[[9, 27, 45]] = -1
    oracle.dcb_sweeps(L, 2, s, 50.0, 1, 0, 0, 0, 1, 1)
    np.testing.assert_array_equal(s, np.ones(L * L, dtype=np.int8))


def test_dcb_rejects_tiles_that_do_not_tile_the_torus():
    s = np.ones(36, dtype=np.int8)
    with pytest.raises(ValueError):
        oracle.dcb_sweeps(6, 2, s, 0.4, 1, 0, 0, 0, 1, 1)  # 3 tiles per row: no coarse checkerboard
