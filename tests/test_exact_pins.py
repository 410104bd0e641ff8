"""Pins for the exact finite-lattice free energy used to judge population annealing
(Kaufman's closed form, in paper_1709_04394_gb300.exact) against full enumeration
(4x4) and the row transfer matrix (6x6, 8x8), plus its Onsager limit."""
import math

import numpy as np
import pytest

from paper_1709_04394_gb300 import exact
from tests import exact_small


def test_4x4_density_of_states_by_enumeration():
    E = exact_small.ising2d_energies(4)
    vals, cnt = np.unique(E, return_counts=True)
    g = dict(zip(vals.tolist(), cnt.tolist()))
    assert sum(g.values()) == 65536
    assert -28 not in g  # no state one bond above the ground state pair
    assert g[-32] == 2 and g[32] == 2
    for e, c in g.items():
        assert g[-e] == c  # E -> -E symmetry of the bipartite lattice


@pytest.mark.parametrize("beta", [0.05, 0.1, 0.3, 0.4406868, 0.7, 1.0, 2.0])
def test_kaufman_equals_enumeration_4x4(beta):
    E = exact_small.ising2d_energies(4)
    assert exact.ising2d_lnZ(4, beta) == pytest.approx(exact_small.lnZ_from_energies(E, beta), rel=1e-13)


@pytest.mark.parametrize("L", [6, 8])
@pytest.mark.parametrize("beta", [0.2, 0.4406868, 0.6, 1.0])
def test_kaufman_equals_transfer_matrix(L, beta):
    assert exact.ising2d_lnZ(L, beta) == pytest.approx(exact_small.ising2d_lnZ_transfer(L, beta), rel=1e-12)


def test_kaufman_energy_equals_enumeration_4x4():
    E = exact_small.ising2d_energies(4)
    for beta in (0.3, 0.4406868, 0.8):
        m1, _ = exact_small.mean_energy(E, beta)
        assert exact.ising2d_energy_per_site(4, beta) == pytest.approx(m1 / 16, rel=1e-8)


def test_beta_zero_is_n_ln2():
    assert exact.ising2d_lnZ(64, 0.0) == 4096 * math.log(2.0)


def test_converges_to_onsager_at_criticality():
    target = exact.onsager_lnZ_per_site_at_critical()
    d = [abs(exact.ising2d_lnZ_per_site(L, exact.BETA_C) - target) for L in (16, 32, 64, 128)]
    assert d[-1] < 1e-4 and all(a > b for a, b in zip(d, d[1:]))
    # the critical energy per site tends to -sqrt(2)
    assert exact.ising2d_energy_per_site(256, exact.BETA_C) == pytest.approx(-math.sqrt(2), abs=5e-3)
