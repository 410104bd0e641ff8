"""GPU parity: population annealing with nearest-integer or Poisson
resampling and a variable population size (Sec. 5.4, Eq. (13) with R_{i-1})
against the CPU oracle. Population sizes, exact energy sums, the live spins, energies and
parents are compared bit for bit; ln Q and ln Z to a relative 1e-12."""
import math

import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, spins_out, torch  # noqa: F401

pytestmark = pytest.mark.gpu

RTOL = 1e-12
NEAREST = gbmc.GBMC_RESAMPLE_NEAREST
POISSON = gbmc.GBMC_RESAMPLE_POISSON
LAWS = [NEAREST, POISSON]


def _compare(stats, ref, pop, N):
    st = stats[:, pop]
    np.testing.assert_array_equal(st["n_replicas"], ref["nrep"])
    np.testing.assert_array_equal(st["sumE"], ref["sumE"])
    assert st["lnZ"][0] == ref["lnZ"][0] == N * math.log(2.0)
    np.testing.assert_allclose(st["lnZ"], ref["lnZ"], rtol=RTOL, atol=0)
    np.testing.assert_allclose(st["lnQ"], ref["lnQ"], rtol=RTOL, atol=1e-13)


def _live_state(ctx, pa, lat, li, n_inst, cap, nrep):
    """Per instance: (spins, E, parents) of its live replicas."""
    sp = spins_out(ctx, lat).reshape(n_inst, cap, -1)
    E = np.empty(n_inst * cap, dtype=np.int32)
    gbmc.pa_energies_out(ctx, pa, li, E)
    par = np.empty(n_inst * cap, dtype=np.uint32)
    gbmc.pa_parents_out(ctx, pa, li, par)
    E, par = E.reshape(n_inst, cap), par.reshape(n_inst, cap)
    return [(sp[i, :nrep[i]], E[i, :nrep[i]], par[i, :nrep[i]]) for i in range(n_inst)]


@pytest.mark.parametrize("law", LAWS)
@pytest.mark.parametrize("L,R0,cap,S,theta", [(16, 600, 800, 6, 2), (8, 50, 100, 8, 3), (32, 2100, 2500, 4, 2)])
def test_pa_nearest_2d_matches_oracle(ctx, law, L, R0, cap, S, theta):
    seed = 21 + L
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=cap, seed=seed)
    pa = gbmc.pa_create(ctx, [lat], theta, S, resample=law, initial_replicas=R0)
    stats, n = gbmc.pa_run(ctx, pa, capacity=S + 1)
    assert n == S
    ref = oracle.pa_run_nearest(2, L, seed, 0, R0, cap, oracle.linear_betas(1.0, S), theta, poisson=law == POISSON)
    assert ref["ok"]
    _compare(stats, ref, 0, L * L)
    (sp, E, par), = _live_state(ctx, pa, lat, 0, 1, cap, [ref["nrep"][-1]])
    np.testing.assert_array_equal(sp, ref["spins"])
    np.testing.assert_array_equal(E, ref["E"])
    np.testing.assert_array_equal(par, ref["parents"])
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)


@pytest.mark.parametrize("law", LAWS)
@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("mode", [gbmc.GBMC_LAUNCH_GRID, gbmc.GBMC_LAUNCH_PERSISTENT])
def test_pa_nearest_3d_ea_instances_and_launch_forms(ctx, law, fused, mode):
    L, I, R0, cap, S, theta, seed = 4, 3, 300, 400, 6, 2, 5
    lat = gbmc.lattice_init(ctx, 3, L, model=gbmc.GBMC_EA_PMJ, n_instances=I, n_replicas=cap, seed=seed,
                            instance_base=2)
    gbmc.gbmc_set_resample_mode(ctx, fused)
    gbmc.gbmc_set_sweep_launch(ctx, mode)
    try:
        pa = gbmc.pa_create(ctx, [lat], theta, S, beta_f=2.0, resample=law, initial_replicas=R0)
        stats, _ = gbmc.pa_run(ctx, pa, capacity=S + 1)
    finally:
        gbmc.gbmc_set_resample_mode(ctx, True)
        gbmc.gbmc_set_sweep_launch(ctx, gbmc.GBMC_LAUNCH_AUTO)
    betas = oracle.linear_betas(2.0, S)
    refs = [oracle.pa_run_nearest(3, L, seed, 2 + i, R0, cap, betas, theta, J=oracle.couplings(L, seed, 2 + i),
                                  poisson=law == POISSON) for i in range(I)]
    for i, ref in enumerate(refs):
        assert ref["ok"]
        _compare(stats, ref, i, L ** 3)
    live = _live_state(ctx, pa, lat, 0, I, cap, [r["nrep"][-1] for r in refs])
    for (sp, E, par), ref in zip(live, refs):
        np.testing.assert_array_equal(sp, ref["spins"])
        np.testing.assert_array_equal(E, ref["E"])
        np.testing.assert_array_equal(par, ref["parents"])
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)


@pytest.mark.parametrize("law", LAWS)
def test_pa_nearest_mixed_batch_and_graph_replay(ctx, law):
    S, theta = 5, 2
    a = gbmc.lattice_init(ctx, 2, 16, n_replicas=520, seed=3, instance_base=0)
    b = gbmc.lattice_init(ctx, 2, 32, n_replicas=520, seed=3, instance_base=1)
    pa = gbmc.pa_create(ctx, [a, b], theta, S, resample=law, initial_replicas=420)
    stats, _ = gbmc.pa_run(ctx, pa, capacity=S + 1)
    for pop, L in enumerate((16, 32)):
        ref = oracle.pa_run_nearest(2, L, 3, pop, 420, 520, oracle.linear_betas(1.0, S), theta,
                                    poisson=law == POISSON)
        assert ref["ok"]
        _compare(stats, ref, pop, L * L)
    first = spins_out(ctx, b).copy()
    for _ in range(2):  # the captured run replays to the same state
        gbmc.pa_reset(ctx, pa, True, 3)
        gstats, n = gbmc.pa_run_graph(ctx, pa, capacity=S + 1)
        assert n == S
        np.testing.assert_array_equal(gstats["n_replicas"], stats["n_replicas"])
        np.testing.assert_array_equal(gstats["sumE"], stats["sumE"])
        np.testing.assert_array_equal(spins_out(ctx, b), first)
    gbmc.pa_free(pa)
    gbmc.lattice_free(a)
    gbmc.lattice_free(b)


@pytest.mark.parametrize("law", LAWS)
def test_pa_nearest_full_size_resampling_step_l64(ctx, law):
    # R_0 = 10^5 replicas of L = 64 (capacity 1.05 10^5): the whole resampling
    # (counts, R_i, children order, ln Q) of step 3 and of the last step 100
    # (beta = 1) from the library's own energies, and the last step's theta
    # sweeps on sampled slots
    L, R0, cap, seed, theta = 64, 100000, 105000, 9, 10
    betas = oracle.linear_betas(1.0, 100)
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=cap, seed=seed)
    pa = gbmc.pa_create(ctx, [lat], theta, 100, resample=law, initial_replicas=R0)
    resample = oracle.resample_poisson if law == POISSON else oracle.resample_nearest
    done, n_prev = 0, R0
    for step in (3, 100):
        while done < step - 1:
            n_prev = int(gbmc.pa_step(ctx, pa)[0]["n_replicas"])
            done += 1
        E = np.empty(cap, dtype=np.int32)
        gbmc.pa_energies_out(ctx, pa, 0, E)
        prev = spins_out(ctx, lat) if step == 100 else None
        row = gbmc.pa_step(ctx, pa)
        done += 1
        par = np.empty(cap, dtype=np.uint32)
        gbmc.pa_parents_out(ctx, pa, 0, par)
        counts, Rn, lnQ = resample(E[:n_prev].astype(np.int64), betas[step] - betas[step - 1], R0, cap, seed, 0,
                                   step)
        assert int(row[0]["n_replicas"]) == Rn and abs(Rn - R0) < 3000
        np.testing.assert_array_equal(par[:Rn], oracle.children_order(counts))
        assert abs(row[0]["lnQ"] - lnQ) <= RTOL * abs(lnQ) + 1e-13
        if prev is not None:
            cur = spins_out(ctx, lat)
            for slot in np.random.default_rng(step).integers(Rn, size=8):
                s = prev[par[slot]].copy()
                oracle.sweeps(2, L, s, None, betas[step], seed, 0, int(slot), (step - 1) * theta, theta)
                np.testing.assert_array_equal(cur[slot], s)
        n_prev = Rn
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)


def test_pa_nearest_overflow_is_reported(ctx):
    # capacity = R_0 and a steep schedule: some step needs more slots; the
    # library keeps the first `capacity` children and reports it at the sync
    lat = gbmc.lattice_init(ctx, 2, 4, n_replicas=40, seed=5)
    pa = gbmc.pa_create(ctx, [lat], 1, 10, beta_f=3.0, resample=NEAREST, initial_replicas=40)
    ref = oracle.pa_run_nearest(2, 4, 5, 0, 40, 40, oracle.linear_betas(3.0, 10), 1)
    assert not ref["ok"]
    with pytest.raises(gbmc.GbmcError) as e:
        gbmc.pa_run(ctx, pa, capacity=11)
    assert e.value.status == gbmc.GBMC_ERR_STATE
    gbmc.gbmc_sync(ctx)  # the flag was cleared by the report
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)


def test_pa_nearest_argument_checks(ctx):
    lat = gbmc.lattice_init(ctx, 2, 8, n_replicas=100, seed=1)
    with pytest.raises(gbmc.GbmcError):
        gbmc.pa_create(ctx, [lat], 1, 4, resample=NEAREST, initial_replicas=101)  # beyond the capacity
    with pytest.raises(gbmc.GbmcError):
        gbmc.pa_create(ctx, [lat], 1, 4, resample=NEAREST, schedule=gbmc.GBMC_SCHED_BISECTION)
    with pytest.raises(gbmc.GbmcError):
        gbmc.pa_create(ctx, [lat], 1, 4, initial_replicas=50)  # multinomial keeps R
    with pytest.raises(gbmc.GbmcError):
        gbmc.pa_create(ctx, [lat], 1, 4, resample=7)
    gbmc.lattice_free(lat)
