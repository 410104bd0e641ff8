"""GPU parity of the multi-spin-coded sweeps (Sec. 5.4: 32 replicas per word,
LCG uniforms re-seeded by Philox): spins bit for bit against the oracle's
replica-by-replica sweeps with the same random numbers, alone and inside
population annealing (both resampling laws)."""
import math

import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, device_i32, spins_out, torch  # noqa: F401
from tests.test_gpu_pa import RTOL, _compare_run, _sampled_full_size_check

pytestmark = pytest.mark.gpu

MSC = gbmc.GBMC_RNG_MSC


@pytest.mark.parametrize("L,I,R,n,beta", [
    (16, 1, 40, 5, 0.4406868),   # two groups, the second partial
    (64, 1, 100, 4, 0.3),
    (32, 2, 32, 3, 0.0),         # beta = 0: every spin flips
    (48, 1, 33, 3, 0.6),
    (128, 1, 70, 2, 0.5),        # 73.7 KB of words per group
    (16, 3, 130, 6, 1.0),        # 4 groups per CTA, two CTAs per instance
])
def test_msc_sweeps_match_oracle(ctx, L, I, R, n, beta):
    seed = 31 + L
    lat = gbmc.lattice_init(ctx, 2, L, n_instances=I, n_replicas=R, seed=seed, instance_base=4)
    gbmc.lattice_set_sweep_counter(lat, 9)
    gbmc.metropolis_sweeps_msc(ctx, lat, beta, n - 1)
    gbmc.metropolis_sweeps_msc(ctx, lat, beta, 1)  # counters continue across calls
    got = spins_out(ctx, lat)
    E, M = device_i32(I * R), device_i32(I * R)
    gbmc.observables(ctx, lat, E, M)
    E = E.cpu().numpy()
    for i in range(I):
        for r in range(R):
            s = oracle.init_spins(2, L, seed, 4 + i, r, True)
            oracle.msc_sweeps(2, L, s, None, beta, seed, 4 + i, r, 9, n)
            np.testing.assert_array_equal(got[i * R + r], s, err_msg="instance %d replica %d" % (i, r))
            assert E[i * R + r] == oracle.observables(2, L, s)[0]
    assert gbmc.lattice_info(lat).sweep_counter == 9 + n
    gbmc.lattice_free(lat)


@pytest.mark.parametrize("fused", [True, False])
def test_pa_msc_matches_oracle(ctx, fused):
    S, theta = 5, 2
    a = gbmc.lattice_init(ctx, 2, 16, n_replicas=600, seed=3, instance_base=0)
    b = gbmc.lattice_init(ctx, 2, 32, n_replicas=150, seed=3, instance_base=1)
    gbmc.gbmc_set_resample_mode(ctx, fused)
    try:
        pa = gbmc.pa_create(ctx, [a, b], theta, S, sweep_rng=MSC)
        stats, n = gbmc.pa_run(ctx, pa, capacity=S + 1)
    finally:
        gbmc.gbmc_set_resample_mode(ctx, True)
    assert n == S
    for pop, (lat, L, R) in enumerate(((a, 16, 600), (b, 32, 150))):
        ref = oracle.pa_run(2, L, 3, pop, R, oracle.linear_betas(1.0, S), theta, msc=True)
        _compare_run(stats, ref, pop, L * L)
        np.testing.assert_array_equal(spins_out(ctx, lat), ref["spins"])
    gbmc.pa_free(pa)
    gbmc.lattice_free(a)
    gbmc.lattice_free(b)


def test_pa_msc_with_nearest_integer_resampling(ctx):
    L, R0, cap, S, theta, seed = 16, 300, 360, 6, 2, 8
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=cap, seed=seed)
    pa = gbmc.pa_create(ctx, [lat], theta, S, sweep_rng=MSC, resample=gbmc.GBMC_RESAMPLE_NEAREST,
                        initial_replicas=R0)
    stats, _ = gbmc.pa_run(ctx, pa, capacity=S + 1)
    ref = oracle.pa_run_nearest(2, L, seed, 0, R0, cap, oracle.linear_betas(1.0, S), theta, msc=True)
    assert ref["ok"]
    np.testing.assert_array_equal(stats[:, 0]["n_replicas"], ref["nrep"])
    np.testing.assert_array_equal(stats[:, 0]["sumE"], ref["sumE"])
    np.testing.assert_allclose(stats[:, 0]["lnZ"], ref["lnZ"], rtol=RTOL, atol=0)
    n = int(ref["nrep"][-1])
    np.testing.assert_array_equal(spins_out(ctx, lat)[:n], ref["spins"])
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)


def test_full_size_pa_msc_l64_r100000_sampled(ctx):
    # the benchmark population, multi-spin-coded sweeps: exact resampling of the
    # whole population and theta sweeps on sampled slots
    _sampled_full_size_check(ctx, 2, 64, gbmc.GBMC_ISING_FM, 1, 100000, 10, 100, 1.0, (1, 2, 99, 100), 24, 5,
                             sweep_rng=MSC)


def test_msc_rejects_unsupported_lattices(ctx):
    for kw in (dict(dim=2, L=24), dict(dim=3, L=16), dict(dim=2, L=256), dict(dim=2, L=64, layout=gbmc.GBMC_BITPACK)):
        lat = gbmc.lattice_init(ctx, kw.pop("dim"), kw.pop("L"), seed=1, **kw)
        with pytest.raises(gbmc.GbmcError) as e:
            gbmc.metropolis_sweeps_msc(ctx, lat, 0.4, 1)
        assert e.value.status == gbmc.GBMC_ERR_ARG
        gbmc.lattice_free(lat)
