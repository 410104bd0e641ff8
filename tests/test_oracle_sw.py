"""Pins for the oracle's Swendsen-Wang update (Sec. 3.3, its three steps;
reading R19).

The clusters are checked against networkx's connected components of the
active-bond graph (named by their smallest site); the bond law against
p = 1 - exp(-2 beta); the whole update on a 2 x 2 torus against its exact
transition law, obtained by enumerating every bond configuration and cluster
coin; and the chain against the 4 x 4 Boltzmann distribution (enumeration).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from tests import exact_small

nx = pytest.importorskip("networkx")


def _forward(dim, L, i, mu):
    c = list(np.unravel_index(i, (L,) * dim)[::-1])  # x, y[, z]
    c[mu] = (c[mu] + 1) % L
    return int(np.ravel_multi_index(tuple(c[::-1]), (L,) * dim))


@pytest.mark.parametrize("dim,L,beta", [(2, 16, 0.44), (2, 9, 0.8), (3, 6, 0.22), (2, 12, 0.05)])
def test_clusters_are_the_connected_components_named_by_their_smallest_site(dim, L, beta):
    s = oracle.init_spins(dim, L, 4, 0, 0, True)
    for t in range(3):
        active = oracle.sw_bonds(dim, L, s, beta, 4, 0, 0, t)
        g = nx.Graph()
        g.add_nodes_from(range(s.size))
        for i in range(s.size):
            for mu in range(dim):
                if active[i, mu]:
                    g.add_edge(i, _forward(dim, L, i, mu))
        want = np.empty(s.size, dtype=np.int32)
        for comp in nx.connected_components(g):
            want[list(comp)] = min(comp)
        before = s.copy()
        lab = oracle.sw_update(dim, L, s, beta, 4, 0, 0, t, want_labels=True)
        np.testing.assert_array_equal(lab, want)
        # every cluster flipped as a whole (or not at all)
        flipped = s != before
        for comp in nx.connected_components(g):
            comp = list(comp)
            assert flipped[comp].all() or not flipped[comp].any()


def test_bond_law_parallel_spins_only():
    L, beta, n = 8, 0.3, 400
    s = oracle.init_spins(2, L, 7, 0, 0, True)
    Tb = oracle.sw_bond_threshold(beta)
    p = (Tb + 1) / 2 ** 32
    assert Tb < (1 - math.exp(-2 * beta)) * 2 ** 32 <= Tb + 1
    par = np.array([[s[i] == s[_forward(2, L, i, mu)] for mu in range(2)] for i in range(L * L)])
    acc = np.zeros((L * L, 2))
    for t in range(n):
        acc += oracle.sw_bonds(2, L, s, beta, 7, 0, 0, t)
    assert acc[~par].sum() == 0
    freq = acc[par].sum() / (par.sum() * n)
    assert abs(freq - p) < 5 * math.sqrt(p * (1 - p) / (par.sum() * n))
    assert oracle.sw_bond_threshold(0.0) == -1  # beta = 0: no bond is ever active


def _exact_sw_law_2x2(start, beta):
    """Final-state distribution of one SW update of a 2 x 2 torus (4 sites, 8
    forward bonds, each neighbour pair joined by two bonds)."""
    L, N = 2, 4
    p = (oracle.sw_bond_threshold(beta) + 1) / 2 ** 32
    s0 = np.array([1 - 2 * ((start >> i) & 1) for i in range(N)])
    bonds = [(i, _forward(2, L, i, mu)) for i in range(N) for mu in range(2)]
    law = np.zeros(1 << N)
    for act in itertools.product((0, 1), repeat=len(bonds)):
        w = 1.0
        for (i, j), a in zip(bonds, act):
            if s0[i] != s0[j]:
                if a:
                    w = 0.0
                    break
            else:
                w *= p if a else 1 - p
        if w == 0.0:
            continue
        parent = list(range(N))

        def find(x):
            while parent[x] != x:
                x = parent[x]
            return x

        for (i, j), a in zip(bonds, act):
            if a:
                parent[find(i)] = find(j)
        roots = sorted({find(i) for i in range(N)})
        for coins in itertools.product((0, 1), repeat=len(roots)):
            flip = dict(zip(roots, coins))
            final = 0
            for i in range(N):
                si = -s0[i] if flip[find(i)] else s0[i]
                final |= (1 if si < 0 else 0) << i
            law[final] += w / 2 ** len(roots)
    return law


@pytest.mark.parametrize("start,beta", [(0b0000, 0.4), (0b0110, 0.7), (0b0001, 0.25)])
def test_sw_update_2x2_matches_exact_transition_law(start, beta):
    law = _exact_sw_law_2x2(start, beta)
    assert abs(law.sum() - 1) < 1e-12
    n = 20000
    counts = np.zeros(16)
    s0 = np.array([1 - 2 * ((start >> i) & 1) for i in range(4)], dtype=np.int8)
    for t in range(n):
        s = s0.copy()
        oracle.sw_update(2, 2, s, beta, 3, 0, 0, t)
        counts[int(sum(((1 - int(v)) // 2) << i for i, v in enumerate(s)))] += 1
    freq = counts / n
    sigma = np.sqrt(np.maximum(law * (1 - law), 1e-12) / n)
    assert np.max(np.abs(freq - law) / sigma) < 5.0
    assert (counts[law == 0] == 0).all()


@pytest.mark.parametrize("beta", [0.3, 0.4406868, 0.6])
def test_sw_chain_4x4_energy_matches_enumeration(beta):
    E_all = exact_small.ising2d_energies(4)
    s = oracle.init_spins(2, 4, 5, 0, 0, True)
    n = 30000
    E = np.empty(n)
    for t in range(n):
        oracle.sw_update(2, 4, s, beta, 5, 0, 0, t)
        E[t] = oracle.observables(2, 4, s)[0]
    b = E[: n // 50 * 50].reshape(50, -1).mean(1)
    m1, _ = exact_small.mean_energy(E_all, beta)
    assert abs(b.mean() - m1) < 4 * b.std(ddof=1) / math.sqrt(50) + 1e-9


def test_sw_limits():
    # beta = 0: single-site clusters, each flips with probability 1/2, independently
    L, n = 8, 2000
    s0 = oracle.init_spins(2, L, 2, 0, 0, True)
    flips = np.zeros(L * L)
    for t in range(n):
        s = s0.copy()
        lab = oracle.sw_update(2, L, s, 0.0, 2, 0, 0, t, want_labels=True)
        assert (lab == np.arange(L * L)).all()
        flips += s != s0
    assert np.max(np.abs(flips / n - 0.5)) < 5 * math.sqrt(0.25 / n)
    # large beta from the ordered state: one cluster, the whole lattice flips together
    for t in range(20):
        s = np.ones(L * L, dtype=np.int8)
        lab = oracle.sw_update(2, L, s, 30.0, 2, 0, 0, t, want_labels=True)
        assert (lab == 0).all() and abs(int(s.sum())) == L * L
