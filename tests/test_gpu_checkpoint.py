"""Checkpoint / resume: the generator is stateless (Sec. 4: counter-based, no
state to save), so a checkpoint is the configuration plus the sweep counter;
a run split in two with a checkpoint in the middle is bit-identical to the
uninterrupted run (sweeps) -- and population annealing runs are reproducible
from (seed, schedule) alone."""
import numpy as np
import pytest

from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, spins_out, torch  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,L,model,layout", [(2, 64, gbmc.GBMC_ISING_FM, gbmc.GBMC_INT8),
                                                (3, 8, gbmc.GBMC_EA_PMJ, gbmc.GBMC_INT8),
                                                (2, 512, gbmc.GBMC_ISING_FM, gbmc.GBMC_INT8),
                                                (2, 128, gbmc.GBMC_ISING_FM, gbmc.GBMC_BITPACK)])
def test_split_run_equals_uninterrupted_run(ctx, dim, L, model, layout):
    kw = dict(model=model, n_replicas=3, seed=2024, layout=layout)
    full = gbmc.lattice_init(ctx, dim, L, **kw)
    gbmc.metropolis_sweeps(ctx, full, 0.5, 9)
    # first half, checkpoint to host (configuration + sweep counter), resume in a new lattice
    a = gbmc.lattice_init(ctx, dim, L, **kw)
    gbmc.metropolis_sweeps(ctx, a, 0.5, 4)
    ckpt_spins, ckpt_t = spins_out(ctx, a), gbmc.lattice_info(a).sweep_counter
    gbmc.lattice_free(a)
    b = gbmc.lattice_init(ctx, dim, L, start=gbmc.GBMC_START_ALL_UP, **kw)
    gbmc.lattice_copy_in(ctx, b, np.ascontiguousarray(ckpt_spins))
    gbmc.lattice_set_sweep_counter(b, ckpt_t)
    gbmc.metropolis_sweeps(ctx, b, 0.5, 5)
    np.testing.assert_array_equal(spins_out(ctx, b), spins_out(ctx, full))
    gbmc.lattice_free(b)
    gbmc.lattice_free(full)


def test_pa_run_is_reproducible_from_seed(ctx):
    lat = gbmc.lattice_init(ctx, 2, 32, n_replicas=1500, seed=31)
    pa = gbmc.pa_create(ctx, [lat], 3, 5)
    s1, _ = gbmc.pa_run(ctx, pa, capacity=6)
    x1 = spins_out(ctx, lat)
    gbmc.pa_reset(ctx, pa, True, 0)
    s2, _ = gbmc.pa_run(ctx, pa, capacity=6)
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(spins_out(ctx, lat), x1)
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)
