"""The stored fixtures of tests/golden/ (written by tests/golden/make_golden.py
from the oracle): the oracle still reproduces them, and they satisfy what the
physics fixes independently of the oracle -- parity and range of E and M on
the 16 x 16 torus (Eq. (7)), and ln Z of the annealing run within a bound of
Kaufman's exact finite-lattice value (Sec. 5.4, Eq. (13))."""
import math
import os

import numpy as np

import oracle
from paper_1709_04394_gb300 import exact

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def test_series_fixture_is_reproduced_and_physical():
    rows = load("config1_L16_series.txt").astype(np.int64)
    N = 256
    # E = -(bonds) + 2 (unsatisfied bonds): even, in [-2N, 2N]; M = N - 2 (down spins): even
    assert np.all(rows[:, 1] % 4 == 0) and np.all(np.abs(rows[:, 1]) <= 2 * N)
    assert np.all(rows[:, 2] % 2 == 0) and np.all(np.abs(rows[:, 2]) <= N)
    s = oracle.init_spins(2, 16, 1, 0, 0, False)
    for t, E, M in rows:
        oracle.sweeps(2, 16, s, None, 0.4406868, 1, 0, 0, int(t), 1)
        assert oracle.observables(2, 16, s) == (E, M), t


def test_pa_fixture_is_reproduced_and_close_to_kaufman():
    rows = load("pa_L8_R2000.txt")
    betas = oracle.linear_betas(1.0, 40)
    np.testing.assert_array_equal(rows[:, 1], betas)
    r = oracle.pa_run(2, 8, 6, 0, 2000, betas, 3)
    np.testing.assert_array_equal(rows[:, 2].astype(np.int64), r["sumE"])
    np.testing.assert_allclose(rows[:, 3], r["lnZ"], rtol=1e-13, atol=0)
    assert rows[0, 3] == 64 * math.log(2.0)
    for b, lnz in zip(rows[:, 1], rows[:, 3]):
        assert abs(lnz - exact.ising2d_lnZ(8, float(b))) / 64 < 3e-3, b
