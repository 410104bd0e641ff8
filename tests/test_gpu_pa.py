"""GPU parity: population annealing (Sec. 5.4, Eq. (13)) of the CUDA library
against the CPU oracle. Spins, energies, resampling parents and the exact
integer population sums are compared bit for bit; ln Q and ln Z in fp64 to a
relative 1e-12 (the two sides sum the same terms in different orders)."""
import math

import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, spins_out, torch  # noqa: F401

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def _compare_run(stats, ref, pop, N):
    """stats: [S+1, P] records of the library; ref: oracle.pa_run dict of one population."""
    st = stats[:, pop]
    np.testing.assert_array_equal(st["step"], np.arange(st.shape[0]))
    np.testing.assert_array_equal(st["sumE"], ref["sumE"])
    np.testing.assert_array_equal(st["sumAbsM"], ref["sumAbsM"])
    np.testing.assert_array_equal(st["sumE2"].astype(np.float64), ref["sumE2"])
    np.testing.assert_array_equal(st["sumM2"].astype(np.float64), ref["sumM2"])
    np.testing.assert_array_equal(st["beta"], ref["betas"])
    assert st["lnZ"][0] == ref["lnZ"][0] == N * math.log(2.0)
    np.testing.assert_allclose(st["lnZ"], ref["lnZ"], rtol=RTOL, atol=0)
    np.testing.assert_allclose(st["lnQ"], ref["lnQ"], rtol=RTOL, atol=1e-13)


def _run_gpu(ctx, lats, theta, S, beta_f=1.0, betas=None):
    sched = gbmc.GBMC_SCHED_LIST if betas is not None else gbmc.GBMC_SCHED_LINEAR
    pa = gbmc.pa_create(ctx, lats, theta, S, schedule=sched, beta_f=beta_f, betas=betas)
    stats, n = gbmc.pa_run(ctx, pa, capacity=S + 1)
    assert n == S
    return pa, stats


@pytest.mark.parametrize("L,R,S,theta", [(16, 3000, 6, 3), (6, 100, 5, 2), (8, 1, 4, 2), (32, 2048, 3, 2)])
def test_pa_2d_matches_oracle(ctx, L, R, S, theta):
    seed = 7 + L
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=seed)
    pa, stats = _run_gpu(ctx, [lat], theta, S)
    ref = oracle.pa_run(2, L, seed, 0, R, oracle.linear_betas(1.0, S), theta)
    _compare_run(stats, ref, 0, L * L)
    np.testing.assert_array_equal(spins_out(ctx, lat), ref["spins"])
    par = np.empty(R, dtype=np.uint32)
    gbmc.pa_parents_out(ctx, pa, 0, par)
    np.testing.assert_array_equal(par, ref["parents"])
    E = np.empty(R, dtype=np.int32)
    M = np.empty(R, dtype=np.int32)
    gbmc.pa_energies_out(ctx, pa, 0, E, M)
    np.testing.assert_array_equal(E, ref["E"])
    np.testing.assert_array_equal(M, ref["M"])
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)


@pytest.mark.parametrize("L", [8, 4])
def test_pa_3d_ea_instances_match_oracle(ctx, L):
    I, R, S, theta, seed = 3, 500, 5, 2, 31
    lat = gbmc.lattice_init(ctx, 3, L, model=gbmc.GBMC_EA_PMJ, n_instances=I, n_replicas=R, seed=seed,
                            instance_base=10)
    betas = oracle.linear_betas(2.0, S)
    pa, stats = _run_gpu(ctx, [lat], theta, S, betas=betas)
    got = spins_out(ctx, lat).reshape(I, R, -1)
    for i in range(I):
        J = oracle.couplings(L, seed, 10 + i)
        ref = oracle.pa_run(3, L, seed, 10 + i, R, betas, theta, J=J)
        _compare_run(stats, ref, i, L ** 3)
        np.testing.assert_array_equal(got[i], ref["spins"])
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)


@pytest.mark.parametrize("mode", [gbmc.GBMC_LAUNCH_AUTO, gbmc.GBMC_LAUNCH_GRID, gbmc.GBMC_LAUNCH_PERSISTENT])
def test_pa_mixed_batch_in_one_launch_matches_oracle(ctx, mode):
    # lattices of uneven L advance together: one sweep launch covers both, as
    # one CTA per unit or as persistent CTAs claiming units largest-first
    S, theta = 4, 2
    a = gbmc.lattice_init(ctx, 2, 16, n_replicas=600, seed=3, instance_base=0)
    b = gbmc.lattice_init(ctx, 2, 32, n_replicas=300, seed=3, instance_base=1)
    gbmc.gbmc_set_sweep_launch(ctx, mode)
    try:
        pa, stats = _run_gpu(ctx, [a, b], theta, S)
    finally:
        gbmc.gbmc_set_sweep_launch(ctx, gbmc.GBMC_LAUNCH_AUTO)
    assert gbmc.pa_populations(pa) == 2
    for pop, (lat, L, R) in enumerate(((a, 16, 600), (b, 32, 300))):
        ref = oracle.pa_run(2, L, 3, pop, R, oracle.linear_betas(1.0, S), theta)
        _compare_run(stats, ref, pop, L * L)
        np.testing.assert_array_equal(spins_out(ctx, lat), ref["spins"])
    gbmc.pa_free(pa)
    gbmc.lattice_free(a)
    gbmc.lattice_free(b)


def test_pa_step_by_step_equals_run(ctx):
    L, R, S, theta = 16, 700, 5, 2
    l1 = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=9)
    l2 = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=9)
    p1, s1 = _run_gpu(ctx, [l1], theta, S)
    p2 = gbmc.pa_create(ctx, [l2], theta, S)
    rows = [gbmc.pa_step(ctx, p2) for _ in range(S)]
    with pytest.raises(gbmc.GbmcError):
        gbmc.pa_step(ctx, p2)
    for k, row in enumerate(rows):
        assert row[0]["lnZ"] == s1[k + 1, 0]["lnZ"]
        assert row[0]["sumE"] == s1[k + 1, 0]["sumE"]
    np.testing.assert_array_equal(spins_out(ctx, l1), spins_out(ctx, l2))
    for p in (p1, p2):
        gbmc.pa_free(p)
    gbmc.lattice_free(l1)
    gbmc.lattice_free(l2)


def _sampled_full_size_check(ctx, dim, L, model, I, R, theta, S, beta_f, check_steps, n_samples, seed,
                             sweep_rng=gbmc.GBMC_RNG_PHILOX):
    """Full-size population: exact check of the resampling (oracle on the whole
    energy array: every parent, ln Q) and of theta sweeps on sampled slots, at
    the annealing steps in `check_steps` (the steps in between run unchecked,
    their ln Z taken from the library's record)."""
    lat = gbmc.lattice_init(ctx, dim, L, model=model, n_instances=I, n_replicas=R, seed=seed)
    pa = gbmc.pa_create(ctx, [lat], theta, S, beta_f=beta_f, sweep_rng=sweep_rng)
    sweeps = oracle.msc_sweeps if sweep_rng == gbmc.GBMC_RNG_MSC else oracle.sweeps
    N = L ** dim
    betas = oracle.linear_betas(beta_f, S)
    E = np.empty(I * R, dtype=np.int32)
    lnZ = np.full(I, N * math.log(2.0))
    rng = np.random.default_rng(0)
    Js = [oracle.couplings(L, seed, i) if model == gbmc.GBMC_EA_PMJ else None for i in range(I)]
    done = 0
    for step in sorted(check_steps):
        while done < step - 1:
            row = gbmc.pa_step(ctx, pa)
            done += 1
            lnZ = np.array([row[i]["lnZ"] for i in range(I)])
        gbmc.pa_energies_out(ctx, pa, 0, E)
        prev = spins_out(ctx, lat).reshape(I, R, N)
        Eprev = E.reshape(I, R).astype(np.int64)
        row = gbmc.pa_step(ctx, pa)
        done += 1
        par = np.empty(I * R, dtype=np.uint32)
        gbmc.pa_parents_out(ctx, pa, 0, par)
        par = par.reshape(I, R)
        cur = spins_out(ctx, lat).reshape(I, R, N)
        gbmc.pa_energies_out(ctx, pa, 0, E)
        for i in range(I):
            counts, lnQ = oracle.resample(Eprev[i], betas[step] - betas[step - 1], seed, i, step)
            np.testing.assert_array_equal(par[i], oracle.children_order(counts))
            assert row[i]["lnQ"] == pytest.approx(lnQ, rel=RTOL, abs=1e-13)
            lnZ[i] += lnQ
            assert row[i]["lnZ"] == pytest.approx(lnZ[i], rel=RTOL)
            assert row[i]["sumE"] == int(E.reshape(I, R)[i].astype(np.int64).sum())
        for _ in range(n_samples):
            i, slot = int(rng.integers(I)), int(rng.integers(R))
            s = prev[i, par[i, slot]].copy()
            sweeps(dim, L, s, Js[i], betas[step], seed, i, slot, (step - 1) * theta, theta)
            np.testing.assert_array_equal(cur[i, slot], s)
            assert E.reshape(I, R)[i, slot] == oracle.observables(dim, L, s, Js[i])[0]
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)


def test_full_size_pa_2d_l64_r100000_sampled(ctx):
    # population annealing 2D Ising L = 64, R = 10^5, beta 0 -> 1 in 101 temperatures, theta = 10:
    # the first two steps and the last two (beta = 0.99, 1.0: energies near the ground state, the
    # weights spanning most of their range)
    _sampled_full_size_check(ctx, 2, 64, gbmc.GBMC_ISING_FM, 1, 100000, 10, 100, 1.0, (1, 2, 99, 100), 24, 1)


def test_full_size_pa_3d_ea_32x20000_sampled(ctx):
    # 3D +-J spin glass L = 8, 32 instances x 2 10^4 replicas, beta 0 -> 3 in 201 temperatures, theta = 10;
    # steps 1, 2 and 199, 200 (beta = 2.985, 3.0)
    _sampled_full_size_check(ctx, 3, 8, gbmc.GBMC_EA_PMJ, 32, 20000, 10, 200, 3.0, (1, 2, 199, 200), 24, 5)


def test_full_size_pa_mixed_2d_sampled(ctx):
    # the mixed batch in one step: (L, R) = (32, 10^5), (64, 5 10^4), (128, 2 10^4),
    # (256, 10^4), instance k for lattice k; resampling checked whole, theta sweeps
    # on sampled slots of every lattice, at steps 1, 2 and 99, 100 (beta = 0.99, 1.0)
    spec, theta, S, seed = [(32, 100000), (64, 50000), (128, 20000), (256, 10000)], 10, 100, 3
    lats = [gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=seed, instance_base=k) for k, (L, R) in enumerate(spec)]
    pa = gbmc.pa_create(ctx, lats, theta, S)
    betas = oracle.linear_betas(1.0, S)
    rng = np.random.default_rng(4)
    E = [np.empty(R, dtype=np.int32) for _, R in spec]
    lnZ = [L * L * math.log(2.0) for L, _ in spec]
    done = 0
    for step in (1, 2, 99, 100):
        while done < step - 1:
            row = gbmc.pa_step(ctx, pa)
            done += 1
            lnZ = [row[k]["lnZ"] for k in range(len(spec))]
        for k in range(len(spec)):
            gbmc.pa_energies_out(ctx, pa, k, E[k])
        prev = [spins_out(ctx, lat) for lat in lats]
        Eprev = [e.astype(np.int64) for e in E]
        row = gbmc.pa_step(ctx, pa)
        done += 1
        for k, (L, R) in enumerate(spec):
            par = np.empty(R, dtype=np.uint32)
            gbmc.pa_parents_out(ctx, pa, k, par)
            gbmc.pa_energies_out(ctx, pa, k, E[k])
            counts, lnQ = oracle.resample(Eprev[k], betas[step] - betas[step - 1], seed, k, step)
            np.testing.assert_array_equal(par, oracle.children_order(counts))
            assert row[k]["lnQ"] == pytest.approx(lnQ, rel=RTOL, abs=1e-13)
            lnZ[k] += lnQ
            assert row[k]["lnZ"] == pytest.approx(lnZ[k], rel=RTOL)
            assert row[k]["sumE"] == int(E[k].astype(np.int64).sum())
            cur = spins_out(ctx, lats[k])
            for slot in rng.integers(R, size=4):
                s = prev[k][par[slot]].copy()
                oracle.sweeps(2, L, s, None, betas[step], seed, k, int(slot), (step - 1) * theta, theta)
                np.testing.assert_array_equal(cur[slot], s)
                assert E[k][slot] == oracle.observables(2, L, s)[0]
    gbmc.pa_free(pa)
    for lat in lats:
        gbmc.lattice_free(lat)


def test_fused_and_separate_resampling_agree(ctx):
    # one cooperative launch per lattice and step vs one launch per phase
    runs = []
    for fused in (True, False):
        gbmc.gbmc_set_resample_mode(ctx, fused)
        lat = gbmc.lattice_init(ctx, 3, 8, model=gbmc.GBMC_EA_PMJ, n_instances=4, n_replicas=2500, seed=17)
        pa, stats = _run_gpu(ctx, [lat], 2, 4, beta_f=2.0)
        par = np.empty(4 * 2500, dtype=np.uint32)
        gbmc.pa_parents_out(ctx, pa, 0, par)
        runs.append((stats, spins_out(ctx, lat), par))
        gbmc.pa_free(pa)
        gbmc.lattice_free(lat)
    gbmc.gbmc_set_resample_mode(ctx, True)
    np.testing.assert_array_equal(runs[0][0]["sumE"], runs[1][0]["sumE"])
    np.testing.assert_array_equal(runs[0][0]["lnZ"], runs[1][0]["lnZ"])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    np.testing.assert_array_equal(runs[0][2], runs[1][2])


def test_graph_run_equals_stream_run_and_replays(ctx):
    # the whole fixed-schedule run as one CUDA graph, replayed after resets
    L, R, S, theta = 32, 3000, 6, 2
    a = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=12)
    b = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=12)
    pa_a, ref = _run_gpu(ctx, [a], theta, S)
    pa_b = gbmc.pa_create(ctx, [b], theta, S)
    incs = []
    for rep in range(3):
        if rep:
            gbmc.pa_reset(ctx, pa_b, True, 0)
        n0 = gbmc.gbmc_kernel_launches()
        got, n = gbmc.pa_run_graph(ctx, pa_b, capacity=S + 1)
        incs.append(gbmc.gbmc_kernel_launches() - n0)
        assert n == S
        np.testing.assert_array_equal(got["sumE"], ref["sumE"])
        np.testing.assert_array_equal(got["lnZ"], ref["lnZ"])
        np.testing.assert_array_equal(spins_out(ctx, b), spins_out(ctx, a))
        assert gbmc.lattice_info(b).sweep_counter == gbmc.lattice_info(a).sweep_counter
    # every replay counts the graph's kernel nodes (resampling phases, sweeps, records), the capture none
    assert incs[0] == incs[1] == incs[2] >= 3 * S, incs
    with pytest.raises(gbmc.GbmcError):
        gbmc.pa_run_graph(ctx, pa_b)  # not at step 0
    # a new seed is captured anew and matches the oracle
    gbmc.pa_reset(ctx, pa_b, True, 99)
    got, _ = gbmc.pa_run_graph(ctx, pa_b, capacity=S + 1)
    ref99 = oracle.pa_run(2, L, 99, 0, R, oracle.linear_betas(1.0, S), theta)
    np.testing.assert_array_equal(got[:, 0]["sumE"], ref99["sumE"])
    np.testing.assert_array_equal(spins_out(ctx, b), ref99["spins"])
    for p in (pa_a, pa_b):
        gbmc.pa_free(p)
    gbmc.lattice_free(a)
    gbmc.lattice_free(b)
