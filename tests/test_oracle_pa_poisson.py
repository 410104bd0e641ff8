"""Pins for the oracle's Poisson resampling with a variable population
(Sec. 5.4 step 2, Eq. (13) with R_{i-1}; reading R20).

Its e^{-x} (range reduction + Taylor series in plain IEEE operations) is
checked against libm; the inversion sampler against the Poisson
distribution's own CDF (scipy) at the interval edges and in law; the
resampling counts against mean = variance = tau_j; population annealing with
it against the 4x4 partition function by enumeration.
"""
import math

import numpy as np
import pytest

import oracle
from tests import exact_small

stats = pytest.importorskip("scipy.stats")


def test_exp_neg_matches_libm():
    xs = np.concatenate([[0.0, 1e-300, 0.5, math.log(2.0), 1.0, 699.9],
                         np.random.default_rng(2).uniform(0, 700, 20000),
                         np.random.default_rng(3).uniform(0, 2, 5000)])
    for x in xs:
        assert abs(oracle.exp_neg(x) / math.exp(-x) - 1.0) <= 4 * 2.0 ** -52, x
    assert oracle.exp_neg(0.0) == 1.0
    assert oracle.exp_neg(700.5) == 0.0


@pytest.mark.parametrize("tau", [0.3, 1.0, 2.5, 7.0, 40.0])
def test_poisson_inversion_edges_follow_the_cdf(tau):
    # u just below / above the CDF value F(n) must give n / n + 1
    for n in range(0, int(tau + 5 * math.sqrt(tau)) + 2):
        F = stats.poisson.cdf(n, tau)
        if not 1e-9 < F < 1 - 1e-9:
            continue
        for delta, want in ((-1e-9, n), (1e-9, n + 1)):
            u = F + delta
            U64 = int(u * 2.0 ** 53) << 11
            assert oracle.poisson(tau, U64) == want, (tau, n, delta)


@pytest.mark.parametrize("tau", [0.3, 2.5, 40.0])
def test_poisson_law(tau):
    rng = np.random.default_rng(11)
    U = rng.integers(0, 2 ** 64, size=20000, dtype=np.uint64)
    n = np.array([oracle.poisson(tau, int(u)) for u in U])
    assert abs(n.mean() - tau) < 5 * math.sqrt(tau / n.size)
    assert abs(n.var() / tau - 1) < 5 * math.sqrt(2 / n.size) + 0.02
    assert oracle.poisson(750.0, 0) == 2 ** 32 - 1


def test_poisson_resampling_counts_have_mean_and_variance_tau():
    rng = np.random.default_rng(6)
    E = (4 * rng.integers(-8, 1, size=30)).astype(np.int64)
    dbeta, R0, n = 0.2, 60, 3000
    w = np.exp(-dbeta * (E - E.min()))
    tau = R0 * w / w.sum()
    c = np.stack([oracle.resample_poisson(E, dbeta, R0, 64, 2, 1, step)[0] for step in range(1, n + 1)])
    assert np.max(np.abs(c.mean(0) - tau) / np.sqrt(tau / n)) < 5
    # sample variance of Poisson counts: Var(s^2) / tau^2 = (1/tau + 2) / n
    assert np.max(np.abs(c.var(0) / tau - 1) / np.sqrt((1 / tau + 2) / n)) < 5
    sizes = c.sum(1)
    assert abs(sizes.mean() - R0) < 5 * math.sqrt(R0 / n)
    # one replica takes all the weight: tau = 2000 > 500 is drawn as 4 pieces of Poisson(500)
    sizes = [oracle.resample_poisson(np.array([0, -4000], dtype=np.int64), 1.0, 2000, 4096, 2, 1, st)[1]
             for st in range(1, 401)]
    assert abs(np.mean(sizes) - 2000) < 5 * math.sqrt(2000 / 400)
    assert abs(np.var(sizes) / 2000 - 1) < 5 * math.sqrt(2 / 400)


def test_pa_poisson_4x4_matches_enumeration():
    E_all = exact_small.ising2d_energies(4)
    betas = oracle.linear_betas(1.0, 20)
    runs = [oracle.pa_run_nearest(2, 4, seed, 0, 2000, 2600, betas, 4, poisson=True) for seed in range(1, 7)]
    assert all(r["ok"] for r in runs)
    lnZ = np.array([r["lnZ"] for r in runs])
    for i, b in enumerate(betas):
        ex = exact_small.lnZ_from_energies(E_all, b)
        assert abs(lnZ[:, i].mean() - ex) < 0.02 + 4 * lnZ[:, i].std() / math.sqrt(6)
    dev = lnZ[:, -1] - exact_small.lnZ_from_energies(E_all, 1.0)
    assert abs(dev.mean()) < 4 * dev.std(ddof=1) / math.sqrt(len(dev)) + 1e-3
