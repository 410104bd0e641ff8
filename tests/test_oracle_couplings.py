"""Pins for the oracle's bimodal +-J couplings (Sec. 6: J_ij = +1 or -1 with
probability 1/2 each, independently for every bond and disorder instance).

The sign of bond b = 3 site + mu of an instance is the top bit of the Philox
word (q = b >> 2, t = 0, r = 0, 3 << 28 | instance), word b & 3: here that
word comes from PyTorch's independent Philox engine, not from the oracle. The
law is checked on many instances: the fraction of negative bonds is 1/2, the
three bond directions are uncorrelated with each other, and neighbouring
instances are uncorrelated.
"""
import numpy as np

import oracle

from .test_oracle_philox import torch_philox  # noqa: F401  (fixture)

PURPOSE_COUPLING = 3


def test_each_bond_is_the_top_bit_of_its_coupling_word(torch_philox):  # noqa: F811
    for L, seed, inst in [(4, 1, 0), (6, 0x0123456789ABCDEF, 7), (8, 99, (1 << 27) - 1)]:
        J = oracle.couplings(L, seed, inst).reshape(-1)
        nb = J.size
        rng = np.random.default_rng(L * 1000 + inst % 1000)
        bonds = np.unique(np.concatenate([np.arange(min(nb, 64)), rng.integers(0, nb, 200)]))
        ctr = np.stack([bonds >> 2, np.zeros_like(bonds), np.zeros_like(bonds),
                        np.full_like(bonds, (PURPOSE_COUPLING << 28) | inst)], axis=1).astype(np.uint32)
        key = np.array([[seed & 0xFFFFFFFF, seed >> 32]] * len(bonds), dtype=np.uint32)
        words = torch_philox(ctr, key)[np.arange(len(bonds)), bonds & 3]
        expect = np.where(words >> 31, -1, 1).astype(np.int8)
        np.testing.assert_array_equal(J[bonds], expect)


def _many(L=6, n_inst=400, seed=2024):
    return np.stack([oracle.couplings(L, seed, i) for i in range(n_inst)]).astype(np.float64)  # [inst][site][mu]


def test_bimodal_law_is_fair():
    J = _many()
    n = J.size
    assert set(np.unique(J)) == {-1.0, 1.0}
    frac = (J < 0).mean()
    assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(n)
    # each direction on its own, and each instance's mean over bonds, has the fair law
    for mu in range(3):
        f = (J[:, :, mu] < 0).mean()
        assert abs(f - 0.5) < 5 * 0.5 / np.sqrt(J[:, :, mu].size)
    per_inst = J.reshape(J.shape[0], -1).mean(axis=1)
    nb = J.shape[1] * 3
    # variance of an instance's mean bond = 1 / nb for independent fair signs
    assert abs(per_inst.var() * nb - 1.0) < 5 * np.sqrt(2.0 / len(per_inst))


def test_directions_and_instances_are_uncorrelated():
    J = _many()
    n = J.shape[0] * J.shape[1]
    for a, b in [(0, 1), (0, 2), (1, 2)]:
        c = (J[:, :, a] * J[:, :, b]).mean()
        assert abs(c) < 5 / np.sqrt(n)
    # the same bond in consecutive instances, and a bond with the next site's bond
    c_inst = (J[1:] * J[:-1]).mean()
    assert abs(c_inst) < 5 / np.sqrt(J[1:].size)
    c_site = (J[:, 1:, :] * J[:, :-1, :]).mean()
    assert abs(c_site) < 5 / np.sqrt(J[:, 1:, :].size)


def test_seed_changes_every_instance():
    a = oracle.couplings(6, 1, 3)
    b = oracle.couplings(6, 2, 3)
    c = oracle.couplings(6, 1, 4)
    # two independent fair sign fields agree on about half the bonds
    for other in (b, c):
        agree = (a == other).mean()
        assert abs(agree - 0.5) < 5 * 0.5 / np.sqrt(a.size)
