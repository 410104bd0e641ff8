"""Every launch shape of the shared-memory sweep kernel (threads per copy,
copies per CTA, row-wise or flat walk) gives the oracle's spins bit for bit,
and the autotuner picks one of them without changing the lattice."""
import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, spins_out, torch  # noqa: F401

pytestmark = pytest.mark.gpu

SHAPES = [(8, 32, True), (16, 16, False), (32, 8, True), (64, 4, True), (64, 2, False), (128, 2, True),
          (128, 1, False), (256, 1, True), (256, 1, False)]


@pytest.mark.parametrize("dim,L,model,R", [(2, 64, gbmc.GBMC_ISING_FM, 37), (2, 16, gbmc.GBMC_ISING_FM, 41),
                                           (3, 8, gbmc.GBMC_EA_PMJ, 19), (2, 24, gbmc.GBMC_ISING_FM, 9)])
def test_every_shape_matches_oracle(ctx, dim, L, model, R):
    beta, n, seed = 0.41, 6, 99
    ref = []
    J = oracle.couplings(L, seed, 0) if model == gbmc.GBMC_EA_PMJ else None
    for r in range(R):
        s = oracle.init_spins(dim, L, seed, 0, r, True)
        oracle.sweeps(dim, L, s, J, beta, seed, 0, r, 0, n)
        ref.append(s)
    ref = np.stack(ref)
    try:
        for tpr, rpc, rw in SHAPES:
            for pers in (False, True):
                gbmc.gbmc_set_tuning(dim, model, L, tpr, rpc, rw, persistent=pers)
                lat = gbmc.lattice_init(ctx, dim, L, model=model, n_replicas=R, seed=seed)
                gbmc.metropolis_sweeps(ctx, lat, beta, n)
                np.testing.assert_array_equal(spins_out(ctx, lat), ref, err_msg=str((tpr, rpc, rw, pers)))
                gbmc.lattice_free(lat)
    finally:
        gbmc.gbmc_set_tuning(dim, model, L, None)


def test_persistent_launch_with_many_more_units_than_ctas(ctx):
    # 25000 copies of L = 16 in groups of 8: 3125 units for at most
    # 152 x 8 resident CTAs, so CTAs claim several units each; the claim
    # counter must be back at 0 for each of the consecutive launches
    L, R, beta, seed = 16, 25000, 0.44, 21
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=seed)
    gbmc.gbmc_set_sweep_launch(ctx, gbmc.GBMC_LAUNCH_PERSISTENT)
    try:
        for _ in range(3):
            gbmc.metropolis_sweeps(ctx, lat, beta, 2)
    finally:
        gbmc.gbmc_set_sweep_launch(ctx, gbmc.GBMC_LAUNCH_AUTO)
    got = spins_out(ctx, lat)
    E, M = torch.empty(R, dtype=torch.int32, device="cuda"), torch.empty(R, dtype=torch.int32, device="cuda")
    gbmc.observables(ctx, lat, E, M)
    E = E.cpu().numpy()
    for r in list(range(0, R, 997)) + [R - 1]:
        s = oracle.init_spins(2, L, seed, 0, r, True)
        oracle.sweeps(2, L, s, None, beta, seed, 0, r, 0, 6)
        np.testing.assert_array_equal(got[r], s, err_msg="replica %d" % r)
        assert E[r] == oracle.observables(2, L, s)[0]
    gbmc.lattice_free(lat)


def test_sweep_launch_mode_is_checked(ctx):
    with pytest.raises(gbmc.GbmcError) as e:
        gbmc.gbmc_set_sweep_launch(ctx, 7)
    assert e.value.status == gbmc.GBMC_ERR_ARG


def test_autotune_leaves_lattice_and_results_unchanged(ctx):
    L, R = 32, 300
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=4)
    before = spins_out(ctx, lat)
    t = gbmc.gbmc_autotune(ctx, lat, 0.44, 3)
    try:
        assert t.resident == 1 and t.n_candidates >= 2 and t.ms_per_sweep > 0
        assert t.threads_per_copy in (8, 16, 32, 64, 128, 256) and t.persistent in (0, 1)
        np.testing.assert_array_equal(spins_out(ctx, lat), before)
        assert gbmc.lattice_info(lat).sweep_counter == 0
        pa = gbmc.pa_create(ctx, [lat], 2, 3)
        stats, _ = gbmc.pa_run(ctx, pa, capacity=4)
        ref = oracle.pa_run(2, L, 4, 0, R, oracle.linear_betas(1.0, 3), 2)
        np.testing.assert_array_equal(stats[:, 0]["sumE"], ref["sumE"])
        np.testing.assert_array_equal(spins_out(ctx, lat), ref["spins"])
        gbmc.pa_free(pa)
    finally:
        gbmc.gbmc_set_tuning(2, gbmc.GBMC_ISING_FM, L, None)
    gbmc.lattice_free(lat)


def test_global_lattice_is_not_tuned(ctx):
    lat = gbmc.lattice_init(ctx, 2, 512, seed=1)
    assert gbmc.gbmc_autotune(ctx, lat, 0.44, 1).resident == 0
    gbmc.lattice_free(lat)
