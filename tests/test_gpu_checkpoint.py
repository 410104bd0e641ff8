"""Checkpoint / resume: the generator is stateless (Sec. 4: counter-based, no
state to save), so a checkpoint is the configuration plus the sweep counter;
a run split in two with a checkpoint in the middle is bit-identical to the
uninterrupted run (sweeps) -- and population annealing runs are reproducible
from (seed, schedule) alone. An annealing run saved between steps (pa_state_save
plus the spins) and restored into a new run continues bit for bit: the same
step records, spins, parents and temperatures as the run never stopped, for
fixed and adaptive schedules and a variable population."""
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


def _pa_run_split(ctx, make_lats, k, cfg, insts=None):
    """A whole annealing run, and the same run stopped after k steps, saved
    (state + spins), restored into a new run on new lattices and finished."""
    lats = make_lats()
    pa = gbmc.pa_create(ctx, lats, **cfg)
    whole, n_whole = gbmc.pa_run(ctx, pa, capacity=cfg["n_steps"] + 1)
    ref = dict(stats=whole, n=n_whole, spins=[spins_out(ctx, l) for l in lats],
               parents=[_parents(ctx, pa, i, l) for i, l in enumerate(lats)],
               betas=[gbmc.pa_betas(pa, i) for i in range(len(lats))])
    gbmc.pa_free(pa)
    for l in lats:
        gbmc.lattice_free(l)
    # first part, checkpoint
    lats = make_lats()
    pa = gbmc.pa_create(ctx, lats, **cfg)
    for _ in range(k):
        gbmc.pa_step(ctx, pa)
    state = gbmc.pa_state_save(ctx, pa)
    saved = [spins_out(ctx, l) for l in lats]
    gbmc.pa_free(pa)
    for l in lats:
        gbmc.lattice_free(l)
    # resume in a new run on new lattices (their own random start is replaced)
    lats = make_lats()
    pa = gbmc.pa_create(ctx, lats, **cfg)
    gbmc.pa_state_load(ctx, pa, state)
    for l, s in zip(lats, saved):
        gbmc.lattice_copy_in(ctx, l, np.ascontiguousarray(s))
    got, n_got = gbmc.pa_run(ctx, pa, capacity=cfg["n_steps"] + 1)
    assert n_got == ref["n"]
    np.testing.assert_array_equal(got, ref["stats"])
    pop = 0
    for i, l in enumerate(lats):
        info = gbmc.lattice_info(l)
        # spins and parents of the live slots (with a variable population the
        # slots beyond it hold stale values)
        n_inst = insts[i] if insts else 1
        R = info.n_copies // n_inst
        sp, sp_ref = spins_out(ctx, l).reshape(n_inst, R, -1), ref["spins"][i].reshape(n_inst, R, -1)
        par, par_ref = _parents(ctx, pa, i, l).reshape(n_inst, R), ref["parents"][i].reshape(n_inst, R)
        for k in range(n_inst):
            live = int(got[n_got, pop + k]["n_replicas"]) if "resample" in cfg else R
            np.testing.assert_array_equal(sp[k, :live], sp_ref[k, :live])
            np.testing.assert_array_equal(par[k, :live], par_ref[k, :live])
        pop += n_inst
        np.testing.assert_array_equal(gbmc.pa_betas(pa, i), ref["betas"][i])
    gbmc.pa_free(pa)
    for l in lats:
        gbmc.lattice_free(l)


def _parents(ctx, pa, i, lat):
    par = np.empty(gbmc.lattice_info(lat).n_copies, dtype=np.uint32)
    gbmc.pa_parents_out(ctx, pa, i, par)
    return par


def test_pa_split_at_step_k_equals_whole_run_fixed_schedule(ctx):
    # two lattice sizes in one run (byte-plane and bit-sliced sweeps), linear schedule
    def make():
        return [gbmc.lattice_init(ctx, 2, 32, n_replicas=700, seed=5, instance_base=0),
                gbmc.lattice_init(ctx, 2, 64, n_replicas=300, seed=5, instance_base=1)]
    _pa_run_split(ctx, make, 3, dict(theta=2, n_steps=7, beta_f=1.0))


def test_pa_split_at_step_k_equals_whole_run_adaptive_and_variable(ctx):
    def make_ad():
        return [gbmc.lattice_init(ctx, 2, 16, n_replicas=800, seed=8, instance_base=0),
                gbmc.lattice_init(ctx, 2, 32, n_replicas=300, seed=8, instance_base=1)]
    _pa_run_split(ctx, make_ad, 6, dict(theta=2, n_steps=400, schedule=gbmc.GBMC_SCHED_BISECTION, beta_f=1.0,
                                        target_overlap=0.85, dbeta_max=0.1))

    def make_ea():
        return [gbmc.lattice_init(ctx, 3, 8, model=gbmc.GBMC_EA_PMJ, n_instances=3, n_replicas=500, seed=12)]
    _pa_run_split(ctx, make_ea, 4, dict(theta=2, n_steps=8, beta_f=2.0, resample=gbmc.GBMC_RESAMPLE_NEAREST,
                                        initial_replicas=400), insts=[3])


def test_pa_state_load_rejects_another_configuration(ctx):
    lat = gbmc.lattice_init(ctx, 2, 16, n_replicas=100, seed=1)
    pa = gbmc.pa_create(ctx, [lat], 2, 5)
    gbmc.pa_step(ctx, pa)
    state = gbmc.pa_state_save(ctx, pa)
    gbmc.pa_free(pa)
    pa = gbmc.pa_create(ctx, [lat], 2, 6)
    with pytest.raises(gbmc.GbmcError) as e:
        gbmc.pa_state_load(ctx, pa, state)
    assert e.value.status == gbmc.GBMC_ERR_ARG
    with pytest.raises(gbmc.GbmcError):
        gbmc.pa_state_load(ctx, pa, state[:-3])
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)
