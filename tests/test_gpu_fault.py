"""Failure detection without a GPU fault: every grid-barrier wait of the fused
resampling, and every neighbour wait of the strip-resident bit-packed sweeps,
is bounded. A test makes the wait run out (each wait asks for one arrival or
one half-sweep more than will ever come, with a short cycle budget); the
kernel returns, the host reports GBMC_ERR_TIMEOUT, and the context stays
usable."""
import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, spins_out, torch  # noqa: F401

pytestmark = pytest.mark.gpu


def test_barrier_wait_runs_out_and_is_reported(ctx):
    lat = gbmc.lattice_init(ctx, 2, 16, n_replicas=3000, seed=5)
    pa = gbmc.pa_create(ctx, [lat], 2, 4)
    gbmc.gbmc_test_barrier_wait(ctx, 1, 2_000_000)  # ~1 ms budget, one phantom arrival
    try:
        with pytest.raises(gbmc.GbmcError) as e:
            gbmc.pa_step(ctx, pa)
        assert e.value.status == gbmc.GBMC_ERR_TIMEOUT
    finally:
        gbmc.gbmc_test_barrier_wait(ctx, 0, 2_000_000_000)
    gbmc.gbmc_sync(ctx)  # flag was cleared when reported
    # the context and the run are usable again after a reset
    gbmc.pa_reset(ctx, pa, True, 5)
    stats, n = gbmc.pa_run(ctx, pa, capacity=5)
    ref = oracle.pa_run(2, 16, 5, 0, 3000, oracle.linear_betas(1.0, 4), 2)
    np.testing.assert_array_equal(stats[:, 0]["sumE"], ref["sumE"])
    np.testing.assert_array_equal(spins_out(ctx, lat), ref["spins"])
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)


def test_strip_neighbour_wait_runs_out_and_is_reported(ctx):
    L = 1024
    lat = gbmc.lattice_init(ctx, 2, L, seed=6, layout=gbmc.GBMC_BITPACK)
    gbmc.gbmc_test_barrier_wait(ctx, 1, 2_000_000)  # ~1 ms budget, one phantom half-sweep
    try:
        gbmc.metropolis_sweeps(ctx, lat, 0.44, 2)
        with pytest.raises(gbmc.GbmcError) as e:
            gbmc.gbmc_sync(ctx)
        assert e.value.status == gbmc.GBMC_ERR_TIMEOUT
    finally:
        gbmc.gbmc_test_barrier_wait(ctx, 0, 2_000_000_000)
    gbmc.gbmc_sync(ctx)
    gbmc.lattice_free(lat)
    # the context is usable again
    lat = gbmc.lattice_init(ctx, 2, L, seed=6, layout=gbmc.GBMC_BITPACK)
    gbmc.metropolis_sweeps(ctx, lat, 0.44, 2)
    s = oracle.init_spins(2, L, 6, 0, 0, True)
    oracle.sweeps(2, L, s, None, 0.44, 6, 0, 0, 0, 2)
    np.testing.assert_array_equal(spins_out(ctx, lat)[0], s)
    gbmc.lattice_free(lat)


def test_int8_strip_neighbour_wait_runs_out_and_is_reported(ctx):
    L = 1024
    lat = gbmc.lattice_init(ctx, 2, L, seed=8)
    gbmc.gbmc_test_barrier_wait(ctx, 1, 2_000_000)
    gbmc.gbmc_set_sweep_kernel(ctx, gbmc.GBMC_KERNEL_BYTES)  # the int8 strip kernel itself
    try:
        gbmc.metropolis_sweeps(ctx, lat, 0.44, 2)
        with pytest.raises(gbmc.GbmcError) as e:
            gbmc.gbmc_sync(ctx)
        assert e.value.status == gbmc.GBMC_ERR_TIMEOUT
    finally:
        gbmc.gbmc_test_barrier_wait(ctx, 0, 2_000_000_000)
        gbmc.gbmc_set_sweep_kernel(ctx, gbmc.GBMC_KERNEL_AUTO)
    gbmc.gbmc_sync(ctx)
    gbmc.lattice_free(lat)
    lat = gbmc.lattice_init(ctx, 2, L, seed=8)
    gbmc.metropolis_sweeps(ctx, lat, 0.44, 2)
    s = oracle.init_spins(2, L, 8, 0, 0, True)
    oracle.sweeps(2, L, s, None, 0.44, 8, 0, 0, 0, 2)
    np.testing.assert_array_equal(spins_out(ctx, lat)[0], s)
    gbmc.lattice_free(lat)
