"""Pins for the oracle's checkerboard Metropolis sweep (Sec. 3.1, Eq. (8); Sec. 6 couplings).

Each test checks the oracle against something other than itself: exact
rational arithmetic, hand-derived zero- and infinite-temperature outcomes,
single-site flip frequencies against the acceptance law, the Boltzmann
distribution of tiny lattices by enumeration, Kaufman's exact energy at
L = 16 (the Ising application test of Sec. 4), and gauge covariance of the
+-J model.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import exact
from tests import exact_small

NEVER = np.array([-1, -1, -1], dtype=np.int64)          # reject every dE > 0
ALWAYS = np.array([2 ** 32 - 1] * 3, dtype=np.int64)   # accept every dE > 0


@pytest.mark.parametrize("beta", [0.0, 1e-9, 0.1, 0.2231435513142097, 0.4406868, 1.0, 3.0, 7.5])
def test_threshold_is_exact_strict_comparison(beta):
    # u * 2^-32 < p  <=>  u <= T  for every integer u  <=>  T < p 2^32 <= T + 1
    T = oracle.thresholds(beta, 3)
    for m, t in enumerate(T):
        p = Fraction(math.exp(-(beta * 4.0 * (m + 1))))
        assert Fraction(int(t)) < p * 2 ** 32 <= Fraction(int(t) + 1)
        assert -1 <= t <= 2 ** 32 - 1


def test_beta_zero_flips_every_spin_every_half_sweep():
    s0 = oracle.init_spins(2, 8, 5, 0, 0, True)
    s = s0.copy()
    oracle.sweeps(2, 8, s, None, 0.0, 5, 0, 0, 0, 1)
    np.testing.assert_array_equal(s, -s0)
    x, y = np.meshgrid(np.arange(8), np.arange(8))
    even = ((x + y) % 2 == 0).reshape(-1)
    s = s0.copy()
    oracle.halfsweep(2, 8, s, None, ALWAYS, 5, 0, 0, 0, 0)
    np.testing.assert_array_equal(s[even], -s0[even])
    np.testing.assert_array_equal(s[~even], s0[~even])


def test_zero_temperature_single_defect_heals_on_its_own_sublattice():
    L = 4
    s = np.ones(L * L, dtype=np.int8)
    s[0 * L + 1] = -1  # site (x=1, y=0) is on the odd sub-lattice
    before = s.copy()
    oracle.halfsweep(2, L, s, None, NEVER, 1, 0, 0, 0, 0)
    np.testing.assert_array_equal(s, before)  # even sites: dE = +4 or +8, all rejected
    oracle.halfsweep(2, L, s, None, NEVER, 1, 0, 0, 0, 1)
    np.testing.assert_array_equal(s, np.ones(L * L, dtype=np.int8))  # defect: dE = -8


def test_zero_temperature_flips_zero_energy_sites():
    # vertical stripes of width 1: every site has dE = 0 and is flipped (dE <= 0 accepted)
    L = 6
    x = np.tile(np.arange(L), L)
    y = np.repeat(np.arange(L), L)
    s = np.where(x % 2 == 0, 1, -1).astype(np.int8)
    s0 = s.copy()
    oracle.halfsweep(2, L, s, None, NEVER, 1, 0, 0, 0, 0)
    even = (x + y) % 2 == 0
    np.testing.assert_array_equal(s[even], -s0[even])
    np.testing.assert_array_equal(s[~even], s0[~even])


def _flip_frequencies(dim, L, s0, J, beta, colour, n, seed=11):
    thr = oracle.thresholds(beta, 3)
    flips = np.zeros(s0.size)
    for t in range(n):
        s = s0.copy()
        oracle.halfsweep(dim, L, s, J, thr, seed, 0, 0, t, colour)
        flips += (s != s0)
    return flips / n, thr


def _local_dE(dim, L, s, J, i):
    coords = np.unravel_index(i, (L,) * dim)[::-1]  # x, y[, z]
    h = 0
    for axis in range(dim):
        for sgn in (1, -1):
            c = list(coords)
            c[axis] = (c[axis] + sgn) % L
            nb = int(np.ravel_multi_index(tuple(c[::-1]), (L,) * dim))
            Jb = 1 if J is None else int(J[i, axis] if sgn == 1 else J[nb, axis])
            h += Jb * int(s[nb])
    return 2 * int(s[i]) * h


@pytest.mark.parametrize("dim,L,model", [(2, 4, "fm"), (2, 6, "fm"), (3, 4, "ea")])
def test_single_site_flip_frequency_matches_acceptance_law(dim, L, model):
    beta = 0.35
    s0 = oracle.init_spins(dim, L, 3, 0, 0, True)
    J = oracle.couplings(L, 9, 0) if model == "ea" else None
    n = 4000
    for colour in (0, 1):
        freq, thr = _flip_frequencies(dim, L, s0, J, beta, colour, n)
        for i in range(s0.size):
            c = np.unravel_index(i, (L,) * dim)
            if sum(c) % 2 != colour:
                assert freq[i] == 0.0
                continue
            dE = _local_dE(dim, L, s0, J, i)
            p = 1.0 if dE <= 0 else (int(thr[dE // 4 - 1]) + 1) / 2 ** 32
            sd = math.sqrt(max(p * (1 - p), 1e-12) / n)
            assert abs(freq[i] - p) <= 5 * sd + 1e-12, (i, dE, freq[i], p)


def _series(dim, L, s, J, beta, n, seed=2):
    E = np.empty(n)
    for t in range(n):
        oracle.sweeps(dim, L, s, J, beta, seed, 0, 0, t, 1)
        E[t] = oracle.observables(dim, L, s, J)[0]
    return E


def _binned_mean(x, nbins=50):
    b = x[: len(x) // nbins * nbins].reshape(nbins, -1).mean(1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nbins)


@pytest.mark.parametrize("beta", [0.25, 0.4406868, 0.6])
def test_4x4_energy_moments_match_enumeration(beta):
    E_all = exact_small.ising2d_energies(4)
    m1, m2 = exact_small.mean_energy(E_all, beta)
    s = oracle.init_spins(2, 4, 7, 0, 0, True)
    E = _series(2, 4, s, None, beta, 60000)[1000:]
    mean, err = _binned_mean(E)
    assert abs(mean - m1) < 4.5 * err, (mean, m1, err)
    mean2, err2 = _binned_mean(E ** 2)
    assert abs(mean2 - m2) < 4.5 * err2


def test_3d_ea_2x2x2_energy_matches_enumeration():
    J = oracle.couplings(2, 4, 1)
    beta = 0.5
    E_all = exact_small.ea3d_energies(2, J)
    m1, _ = exact_small.mean_energy(E_all, beta)
    s = oracle.init_spins(3, 2, 4, 1, 0, True)
    E = _series(3, 2, s, J, beta, 60000)[1000:]
    mean, err = _binned_mean(E)
    assert abs(mean - m1) < 4.5 * err, (mean, m1, err)


def test_config_L16_energy_matches_kaufman():
    # 2D Ising L = 16 at beta = 0.4406868, all-up start, 10^4 sweeps, seed 1;
    # discard 10^3 sweeps, binned error bars (the Ising application test of Sec. 4)
    L, beta = 16, 0.4406868
    s = oracle.init_spins(2, L, 1, 0, 0, False)
    E = _series(2, L, s, None, beta, 10000, seed=1)[1000:] / (L * L)
    mean, err = _binned_mean(E, nbins=30)
    u = exact.ising2d_energy_per_site(L, beta)
    assert abs(mean - u) < 4 * err, (mean, u, err)


def test_gauge_covariance_of_pm_j_dynamics():
    # J_ij -> e_i J_ij e_j together with s_i -> e_i s_i leaves every dE unchanged, so
    # with the same random words the transformed trajectory is e * (original) exactly.
    L = 4
    N = L ** 3
    J = oracle.couplings(L, 21, 3).copy()
    rng = np.random.default_rng(0)
    eps = rng.choice(np.array([-1, 1], dtype=np.int8), size=N)
    Jg = J.copy()
    for i in range(N):
        x, y, z = i % L, (i // L) % L, i // (L * L)
        for mu, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            nb = (((z + dz) % L) * L + (y + dy) % L) * L + (x + dx) % L
            Jg[i, mu] = eps[i] * J[i, mu] * eps[nb]
    s = oracle.init_spins(3, L, 21, 3, 0, True)
    sg = (eps * s).astype(np.int8)
    for t in range(20):
        oracle.sweeps(3, L, s, J, 0.8, 21, 3, 0, t, 1)
        oracle.sweeps(3, L, sg, Jg, 0.8, 21, 3, 0, t, 1)
        np.testing.assert_array_equal(sg, eps * s)
    assert oracle.observables(3, L, s, J)[0] == oracle.observables(3, L, sg, Jg)[0]


def test_all_plus_couplings_reduce_to_ferromagnet():
    L = 4
    J = np.ones((L ** 3, 3), dtype=np.int8)
    a = oracle.init_spins(3, L, 8, 0, 0, True)
    b = a.copy()
    oracle.sweeps(3, L, a, J, 0.3, 8, 0, 0, 0, 7)
    oracle.sweeps(3, L, b, None, 0.3, 8, 0, 0, 0, 7)
    np.testing.assert_array_equal(a, b)


def test_energy_of_ordered_and_checkerboard_states():
    for dim, L in ((2, 4), (2, 8), (3, 4)):
        N = L ** dim
        up = np.ones(N, dtype=np.int8)
        assert oracle.observables(dim, L, up) == (-dim * N, N)
        idx = np.indices((L,) * dim).sum(0).reshape(-1)
        neel = np.where(idx % 2 == 0, 1, -1).astype(np.int8)
        assert oracle.observables(dim, L, neel) == (dim * N, 0)


def _sweep_kernel_applied(pi, L, acc):
    states = exact_small.all_states(L * L)
    v = pi.copy()
    for colour in (0, 1):
        for i in range(L * L):
            x, y = i % L, i // L
            if (x + y) % 2 != colour:
                continue
            nbs = [y * L + (x + 1) % L, y * L + (x - 1) % L, ((y + 1) % L) * L + x, ((y - 1) % L) * L + x]
            dE = 2 * states[:, i] * states[:, nbs].sum(1)
            a = np.where(dE <= 0, 1.0, np.where(dE == 4, acc[4], np.where(dE == 8, acc[8], 0.0)))
            partner = np.arange(states.shape[0]) ^ (1 << i)
            v = v * (1 - a) + v[partner] * a[partner]
    return v


def test_stationarity_of_checkerboard_sweep_4x4():
    # Balance, Eq. (3): the Boltzmann vector is a fixed point of the two-colour sweep.
    # With the exact law exp(-beta dE) the residual is rounding only; with the law the
    # 32-bit thresholds implement, (T+1)/2^32, it is bounded by the 2^-32 quantisation.
    L, beta = 4, 0.4406868
    E = exact_small.ising2d_energies(L).astype(np.float64)
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    exact_law = {4: math.exp(-4 * beta), 8: math.exp(-8 * beta)}
    v = _sweep_kernel_applied(pi, L, exact_law)
    assert np.max(np.abs(v - pi) / pi) < 1e-12
    T = oracle.thresholds(beta, 2)
    thr_law = {4: (int(T[0]) + 1) / 2 ** 32, 8: (int(T[1]) + 1) / 2 ** 32}
    assert all(0 < thr_law[d] - exact_law[d] <= 2.0 ** -32 for d in (4, 8))
    v = _sweep_kernel_applied(pi, L, thr_law)
    assert np.max(np.abs(v - pi) / pi) < 1e-6
    # a factor-2 slip in the exponent is far outside that band
    wrong = {4: math.exp(-2 * beta), 8: math.exp(-4 * beta)}
    v = _sweep_kernel_applied(pi, L, wrong)
    assert np.max(np.abs(v - pi) / pi) > 1e-2
