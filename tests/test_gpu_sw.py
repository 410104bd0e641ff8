"""GPU parity of the Swendsen-Wang cluster updates (Sec. 3.3): spins, the
cluster name of every site (smallest site of its cluster), E and M after each
update, against the oracle's breadth-first labelling, bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, device_i32, spins_out, torch  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,L,I,R,n,beta", [
    (2, 16, 1, 3, 6, 0.4406868),
    (2, 64, 2, 2, 4, 0.3),
    (2, 100, 1, 1, 3, 0.5),
    (2, 6, 1, 5, 10, 1.2),
    (2, 32, 1, 2, 3, 0.0),      # beta = 0: every site its own cluster
    (3, 8, 1, 3, 4, 0.2216544),
    (3, 16, 1, 1, 2, 0.3),
    (2, 96, 1, 1, 3, 0.4406868),  # 3 x 3 tiles: L not a power of two
    (2, 64, 1, 2, 3, 1.5),        # ordered: clusters span every tile
    (3, 32, 1, 1, 2, 0.5),        # 3D tiles, ordered
])
def test_sw_matches_oracle(ctx, dim, L, I, R, n, beta):
    seed = 41 + L
    lat = gbmc.lattice_init(ctx, dim, L, n_instances=I, n_replicas=R, seed=seed, instance_base=3)
    gbmc.lattice_set_sweep_counter(lat, 11)
    N, C = L ** dim, I * R
    Es, Ms = device_i32(n * C), device_i32(n * C)
    labels = device_i32(C * N)
    gbmc.swendsen_wang(ctx, lat, beta, n, Es, Ms, labels)
    got = spins_out(ctx, lat)
    Es, Ms = Es.cpu().numpy().reshape(n, C), Ms.cpu().numpy().reshape(n, C)
    labels = labels.cpu().numpy().reshape(C, N)
    for i in range(I):
        for r in range(R):
            c = i * R + r
            s = oracle.init_spins(dim, L, seed, 3 + i, r, True)
            for u in range(n):
                lab = oracle.sw_update(dim, L, s, beta, seed, 3 + i, r, 11 + u, want_labels=True)
                assert (Es[u, c], Ms[u, c]) == oracle.observables(dim, L, s), (c, u)
            np.testing.assert_array_equal(labels[c], lab, err_msg="copy %d labels" % c)
            np.testing.assert_array_equal(got[c], s, err_msg="copy %d spins" % c)
    assert gbmc.lattice_info(lat).sweep_counter == 11 + n
    gbmc.lattice_free(lat)


def test_sw_full_lattice_l4096(ctx):
    # the single-lattice benchmark size: two updates near the critical point
    L, seed, beta = 4096, 1, 0.4406868
    lat = gbmc.lattice_init(ctx, 2, L, seed=seed)
    labels = device_i32(L * L)
    gbmc.swendsen_wang(ctx, lat, beta, 2, labels=labels)
    s = oracle.init_spins(2, L, seed, 0, 0, True)
    oracle.sw_update(2, L, s, beta, seed, 0, 0, 0)
    lab = oracle.sw_update(2, L, s, beta, seed, 0, 0, 1, want_labels=True)
    np.testing.assert_array_equal(labels.cpu().numpy(), lab)
    np.testing.assert_array_equal(spins_out(ctx, lat)[0], s)
    gbmc.lattice_free(lat)


def test_sw_interleaves_with_metropolis_sweeps(ctx):
    L, seed = 32, 6
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=2, seed=seed)
    gbmc.metropolis_sweeps(ctx, lat, 0.44, 3)
    gbmc.swendsen_wang(ctx, lat, 0.44, 2)
    gbmc.metropolis_sweeps(ctx, lat, 0.44, 1)
    got = spins_out(ctx, lat)
    for r in range(2):
        s = oracle.init_spins(2, L, seed, 0, r, True)
        oracle.sweeps(2, L, s, None, 0.44, seed, 0, r, 0, 3)
        oracle.sw_update(2, L, s, 0.44, seed, 0, r, 3)
        oracle.sw_update(2, L, s, 0.44, seed, 0, r, 4)
        oracle.sweeps(2, L, s, None, 0.44, seed, 0, r, 5, 1)
        np.testing.assert_array_equal(got[r], s)
    gbmc.lattice_free(lat)


def test_sw_rejects_unsupported_lattices(ctx):
    for kw in (dict(dim=3, L=8, model=gbmc.GBMC_EA_PMJ), dict(dim=2, L=64, layout=gbmc.GBMC_BITPACK)):
        lat = gbmc.lattice_init(ctx, kw.pop("dim"), kw.pop("L"), seed=1, **kw)
        with pytest.raises(gbmc.GbmcError) as e:
            gbmc.swendsen_wang(ctx, lat, 0.4, 1)
        assert e.value.status == gbmc.GBMC_ERR_ARG
        gbmc.lattice_free(lat)
