"""Pins for the oracle's nearest-integer resampling with a variable population
(Sec. 5.4 step 2 and Eq. (13) with R_{i-1}; reading R17).

Replica j gets floor(tau_j) or floor(tau_j) + 1 copies, tau_j = R0 e^{-dbeta E_j} /
sum_k e^{-dbeta E_k}, the extra copy with probability frac(tau_j); the
population size is random with mean R0. Checked here against those closed
forms, exactly where they are deterministic, and PA with this law against the
4x4 Ising partition function by enumeration at every temperature.
"""
import math

import numpy as np

import oracle
from tests import exact_small


def test_zero_dbeta_copies_every_replica_r0_over_r_times():
    E = np.array([-32, -8, 0, -24, -32, 16, 4, -4], dtype=np.int64)
    counts, Rn, lnQ = oracle.resample_nearest(E, 0.0, 8, 64, 3, 0, 1)
    assert (counts == 1).all() and Rn == 8 and lnQ == 0.0
    counts, Rn, _ = oracle.resample_nearest(E, 0.0, 16, 64, 3, 0, 1)  # R0 = 2 R_prev: every replica doubles
    assert (counts == 2).all() and Rn == 16
    counts, Rn, _ = oracle.resample_nearest(E, 0.0, 4, 64, 3, 0, 1)   # R0 = R_prev / 2: each kept w.p. 1/2
    assert set(counts.tolist()) <= {0, 1}


def test_counts_follow_nearest_integer_law():
    rng = np.random.default_rng(4)
    E = (4 * rng.integers(-8, 1, size=40)).astype(np.int64)
    dbeta, R0, n = 0.17, 50, 4000
    w = np.exp(-dbeta * (E - E.min()))
    tau = R0 * w / w.sum()
    lo = np.floor(tau)
    acc = np.zeros(E.size)
    sizes = []
    for step in range(1, n + 1):
        counts, Rn, _ = oracle.resample_nearest(E, dbeta, R0, 64, 11, 2, step)
        assert ((counts == lo) | (counts == lo + 1)).all()
        assert Rn == counts.sum()
        acc += counts
        sizes.append(Rn)
    frac = tau - lo
    sigma = np.sqrt(np.maximum(frac * (1 - frac), 1e-12) / n)
    assert np.max(np.abs(acc / n - tau) / sigma) < 5.0
    sd_size = math.sqrt((frac * (1 - frac)).sum() / n)
    assert abs(np.mean(sizes) - R0) < 5 * sd_size


def test_pa_nearest_4x4_matches_enumeration():
    E_all = exact_small.ising2d_energies(4)
    betas = oracle.linear_betas(1.0, 20)
    runs = [oracle.pa_run_nearest(2, 4, seed, 0, 2000, 2400, betas, 4) for seed in range(1, 7)]
    assert all(r["ok"] for r in runs)
    lnZ = np.array([r["lnZ"] for r in runs])
    meanE = np.array([r["sumE"] / r["nrep"] for r in runs])
    sizes = np.array([r["nrep"] for r in runs])
    assert (sizes[:, 0] == 2000).all() and abs(sizes.mean() - 2000) < 20
    for i, b in enumerate(betas):
        exact_lnZ = exact_small.lnZ_from_energies(E_all, b)
        assert abs(lnZ[:, i].mean() - exact_lnZ) < 0.02 + 4 * lnZ[:, i].std() / math.sqrt(6)
        m1, m2 = exact_small.mean_energy(E_all, b)
        sd = math.sqrt(max(m2 - m1 * m1, 1e-9) / 2000.0)
        assert abs(meanE[:, i].mean() - m1) < 6 * sd / math.sqrt(6) + 0.05
    # at beta_f: within 4 standard errors of the seed mean; a dropped ln R_{i-1}
    # or a population-size slip would miss by far more (ln(2400/2000) = 0.18)
    dev = lnZ[:, -1] - exact_small.lnZ_from_energies(E_all, 1.0)
    assert abs(dev.mean()) < 4 * dev.std(ddof=1) / math.sqrt(len(dev)) + 1e-3
    assert abs(dev.mean()) < 0.05


def test_pa_nearest_reports_overflow():
    # capacity equal to R0: some step needs more replicas than there are slots
    betas = oracle.linear_betas(3.0, 10)
    r = oracle.pa_run_nearest(2, 4, 5, 0, 40, 40, betas, 1)
    assert not r["ok"]
