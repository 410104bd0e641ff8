"""Pins for the oracle's population annealing (Sec. 5.4, Eq. (13)).

Checked against: the exact ln Z(beta_0 = 0) = N ln 2; Eq. (13) evaluated
directly in 50-digit arithmetic; the multinomial law of the resampling counts
(chi-square over many independent draws); the exact free energy and energy of
small lattices by enumeration (2D 4x4, 3D +-J 2x2x2) and Kaufman's closed form
(2D 8x8).
"""
import math

import mpmath
import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import exact
from tests import exact_small


def test_ln_q_matches_direct_evaluation_of_eq13():
    mpmath.mp.dps = 50
    rng = np.random.default_rng(1)
    for trial in range(20):
        R = int(rng.integers(1, 300))
        E = rng.integers(-400, 400, size=R) * 4 + (trial % 4) * 2  # ties and offsets
        dbeta = float(rng.choice([0.0, 1e-3, 0.01, 0.05, 0.3]))
        counts, lnQ = oracle.resample(E, dbeta, 3, 0, trial + 1)
        direct = mpmath.log(mpmath.fsum(mpmath.exp(-mpmath.mpf(dbeta) * int(e)) for e in E) / R)
        assert lnQ == pytest.approx(float(direct), rel=1e-13, abs=1e-13)
        assert int(counts.sum()) == R


def test_zero_dbeta_gives_ln_q_zero_and_uniform_draws():
    E = np.arange(50) * 4 - 100
    total = np.zeros(50)
    for step in range(1, 401):
        counts, lnQ = oracle.resample(E, 0.0, 5, 0, step)
        assert lnQ == 0.0
        total += counts
    chi2 = float(((total - 400) ** 2 / 400).sum())
    assert chi2 < 49 + 6 * math.sqrt(98)


def test_counts_follow_multinomial_law():
    E = np.array([-8, -4, -4, 0, 4, 12, 0, -8], dtype=np.int64)
    dbeta = 0.2
    R = E.size
    w = np.exp(-dbeta * (E - E.min()))
    p = w / w.sum()
    n_steps = 5000
    total = np.zeros(R)
    per_step = []
    for step in range(1, n_steps + 1):
        counts, _ = oracle.resample(E, dbeta, 77, 2, step)
        total += counts
        per_step.append(counts[0])
    expected = n_steps * R * p
    chi2 = float(((total - expected) ** 2 / expected).sum())
    assert chi2 < (R - 1) + 6 * math.sqrt(2 * (R - 1)), chi2
    # single-category marginal variance of a multinomial: R p (1 - p)
    var = np.var(per_step)
    assert var == pytest.approx(R * p[0] * (1 - p[0]), rel=0.1)


def test_weights_never_overflow_and_children_are_contiguous():
    for R in (1, 2, 3, 1023, 1024, 1025, 4096):
        E = np.zeros(R, dtype=np.int64)  # all weights equal to 2^s: largest total
        counts, _ = oracle.resample(E, 0.7, 1, 0, 1)
        assert int(counts.sum()) == R
        parent = oracle.children_order(counts)
        assert np.all(np.diff(parent.astype(np.int64)) >= 0)
        np.testing.assert_array_equal(np.bincount(parent, minlength=R), counts)


def test_lowest_energy_dominates_at_large_dbeta():
    E = np.array([0, -40, 8, -40, 100], dtype=np.int64)
    counts, _ = oracle.resample(E, 5.0, 1, 0, 3)
    assert counts[1] + counts[3] == 5  # weights e^{-200} and below quantise to zero


def test_pa_beta_zero_and_invariants():
    r = oracle.pa_run(2, 8, 1, 0, 64, oracle.linear_betas(1.0, 5), 2)
    assert r["lnZ"][0] == 64 * math.log(2.0)
    np.testing.assert_allclose(np.cumsum(r["lnQ"]) + 64 * math.log(2.0), r["lnZ"], rtol=1e-15)
    for i in range(r["spins"].shape[0]):
        assert oracle.observables(2, 8, r["spins"][i])[0] == r["E"][i]
    assert r["sumE"][-1] == r["E"].sum()


def test_pa_4x4_matches_enumeration():
    E_all = exact_small.ising2d_energies(4)
    betas = oracle.linear_betas(1.0, 20)
    runs = [oracle.pa_run(2, 4, seed, 0, 2000, betas, 4) for seed in range(1, 7)]
    lnZ = np.array([r["lnZ"] for r in runs])
    meanE = np.array([r["sumE"] / 2000.0 for r in runs])
    for i, b in enumerate(betas):
        exact_lnZ = exact_small.lnZ_from_energies(E_all, b)
        assert abs(lnZ[:, i].mean() - exact_lnZ) < 0.02 + 4 * lnZ[:, i].std() / math.sqrt(6)
        m1, m2 = exact_small.mean_energy(E_all, b)
        sd = math.sqrt(max(m2 - m1 * m1, 1e-9) / 2000.0)
        assert abs(meanE[:, i].mean() - m1) < 6 * sd / math.sqrt(6) + 0.05
    # at beta_f the free-energy estimate is tight
    assert abs(lnZ[:, -1].mean() - exact_small.lnZ_from_energies(E_all, 1.0)) < 0.01


def test_pa_8x8_free_energy_matches_kaufman():
    L, R = 8, 1000
    betas = oracle.linear_betas(1.0, 100)
    f = []
    for seed in range(1, 5):
        r = oracle.pa_run(2, L, seed, 0, R, betas, 5)
        f.append(r["lnZ"][-1] / (L * L))
    ref = exact.ising2d_lnZ_per_site(L, 1.0)
    f = np.array(f)
    assert abs(f.mean() - ref) < 4 * f.std(ddof=1) / 2 + 2e-4, (f, ref)
    # a dropped ln R (Eq. (13)) or a sign slip in dbeta would miss by far more
    assert abs(f.mean() - ref) < 1e-3


def test_pa_3d_ea_2x2x2_matches_enumeration():
    J = oracle.couplings(2, 13, 4)
    E_all = exact_small.ea3d_energies(2, J)
    betas = oracle.linear_betas(2.0, 40)
    lnZ = np.array([oracle.pa_run(3, 2, seed, 4, 3000, betas, 4, J=J)["lnZ"] for seed in (1, 2, 3, 4)])
    for i in (10, 20, 40):
        ex = exact_small.lnZ_from_energies(E_all, betas[i])
        assert abs(lnZ[:, i].mean() - ex) < 0.01, (i, lnZ[:, i], ex)
