"""GPU parity of the bit-sliced resident sweep kernel (one bit per spin on
chip; 2D ferromagnets with L = 16, 32, 64, 128, 256 and 3D lattices with L = 8
and 16)
against the CPU oracle, element by element: spins, per-sweep energies and
magnetisations, annealing runs (multinomial and nearest-integer resampling,
mixed lattice sizes in one step), parallel tempering; and the bit-sliced and
byte-plane kernels give the same spins on populations whose copy counts leave
the last warp or block partly empty."""
import math

import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, device_i32, spins_out, torch  # noqa: F401
from tests.test_gpu_pa import _compare_run

pytestmark = pytest.mark.gpu

BITS, BYTES, AUTO = gbmc.GBMC_KERNEL_BITS, gbmc.GBMC_KERNEL_BYTES, gbmc.GBMC_KERNEL_AUTO


@pytest.fixture()
def bits(ctx):
    gbmc.gbmc_set_sweep_kernel(ctx, BITS)
    yield ctx
    gbmc.gbmc_set_sweep_kernel(ctx, AUTO)


def _kernel_ran(ctx, fn):
    gbmc.gbmc_profile(ctx, True)
    fn()
    prof = gbmc.gbmc_profile_read(ctx)
    gbmc.gbmc_profile(ctx, False)
    return prof


@pytest.mark.parametrize("dim,L,model,I,R,beta,n", [
    (2, 64, gbmc.GBMC_ISING_FM, 1, 5, 0.4406868, 7),
    (2, 16, gbmc.GBMC_ISING_FM, 2, 5, 0.4406868, 6),  # 8 copies per warp, 10 of 32 in a block
    (2, 32, gbmc.GBMC_ISING_FM, 1, 3, 0.5, 5),        # 2 copies per warp, the second warp half empty
    (2, 128, gbmc.GBMC_ISING_FM, 2, 3, 0.3, 3),
    (2, 256, gbmc.GBMC_ISING_FM, 1, 2, 0.6, 2),
    (2, 64, gbmc.GBMC_ISING_FM, 1, 3, 0.0, 2),       # beta = 0: every site flips every half-sweep
    (2, 64, gbmc.GBMC_ISING_FM, 1, 2, 20.0, 3),      # low temperature: only dE <= 0 moves
    (3, 8, gbmc.GBMC_ISING_FM, 1, 19, 0.22, 5),      # 19 copies: the last warp partly empty
    (3, 8, gbmc.GBMC_EA_PMJ, 3, 7, 1.1, 6),
    (3, 8, gbmc.GBMC_EA_PMJ, 2, 5, 0.0, 2),
    (3, 16, gbmc.GBMC_ISING_FM, 1, 5, 0.22, 4),      # one warp per copy, the last block partly empty
    (3, 16, gbmc.GBMC_EA_PMJ, 2, 3, 1.1, 4),
    (3, 16, gbmc.GBMC_EA_PMJ, 1, 2, 0.0, 2),
    (3, 16, gbmc.GBMC_ISING_FM, 1, 2, 20.0, 3),
])
def test_bits_sweeps_match_oracle(bits, dim, L, model, I, R, beta, n):
    seed = 1000 + 10 * L + dim
    lat = gbmc.lattice_init(bits, dim, L, model=model, n_instances=I, n_replicas=R, seed=seed, instance_base=4,
                            start=gbmc.GBMC_START_RANDOM)
    C = I * R
    Es, Ms = device_i32(n * C), device_i32(n * C)
    prof = _kernel_ran(bits, lambda: gbmc.metropolis_sweeps(bits, lat, beta, n, Es, Ms))
    assert "sweep_bits" in prof and "sweep_resident" not in prof
    torch.cuda.synchronize()
    got = spins_out(bits, lat)
    Es, Ms = Es.cpu().numpy().reshape(n, C), Ms.cpu().numpy().reshape(n, C)
    for c in range(C):
        i, r = divmod(c, R)
        J = oracle.couplings(L, seed, 4 + i) if model == gbmc.GBMC_EA_PMJ else None
        s = oracle.init_spins(dim, L, seed, 4 + i, r, True)
        for t in range(n):
            oracle.sweeps(dim, L, s, J, beta, seed, 4 + i, r, t, 1)
            E, M = oracle.observables(dim, L, s, J)
            assert (Es[t, c], Ms[t, c]) == (E, M), (c, t)
        np.testing.assert_array_equal(got[c], s)
    # the counters continue across calls
    gbmc.metropolis_sweeps(bits, lat, beta, 1)
    s = oracle.init_spins(dim, L, seed, 4, 0, True)
    J = oracle.couplings(L, seed, 4) if model == gbmc.GBMC_EA_PMJ else None
    oracle.sweeps(dim, L, s, J, beta, seed, 4, 0, 0, n + 1)
    np.testing.assert_array_equal(spins_out(bits, lat)[0], s)
    gbmc.lattice_free(lat)


@pytest.mark.parametrize("dim,L,model,I,R", [(2, 64, gbmc.GBMC_ISING_FM, 1, 1027),
                                             (2, 16, gbmc.GBMC_ISING_FM, 3, 45),
                                             (2, 32, gbmc.GBMC_ISING_FM, 1, 77),
                                             (2, 128, gbmc.GBMC_ISING_FM, 3, 101),
                                             (2, 256, gbmc.GBMC_ISING_FM, 1, 33),
                                             (3, 8, gbmc.GBMC_EA_PMJ, 5, 203),
                                             (3, 8, gbmc.GBMC_ISING_FM, 1, 1001),
                                             (3, 16, gbmc.GBMC_EA_PMJ, 3, 37),
                                             (3, 16, gbmc.GBMC_ISING_FM, 1, 41)])
def test_bits_equals_bytes_kernel(ctx, dim, L, model, I, R):
    out = []
    for kernel in (BITS, BYTES):
        gbmc.gbmc_set_sweep_kernel(ctx, kernel)
        lat = gbmc.lattice_init(ctx, dim, L, model=model, n_instances=I, n_replicas=R, seed=77,
                                start=gbmc.GBMC_START_RANDOM)
        E, M = device_i32(I * R), device_i32(I * R)
        gbmc.metropolis_sweeps(ctx, lat, 0.7 if dim == 3 else 0.44, 4)
        gbmc.observables(ctx, lat, E, M)
        out.append((spins_out(ctx, lat), E.cpu().numpy(), M.cpu().numpy()))
        gbmc.lattice_free(lat)
    gbmc.gbmc_set_sweep_kernel(ctx, AUTO)
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)


def test_bits_pa_mixed_lattices_match_oracle(bits):
    # one annealing step covers an L = 24 lattice (byte-plane kernel) and L = 16, 32,
    # 64, 128 lattices (bit-sliced kernel: launches for words of several rows and of
    # whole rows)
    S, theta, seed = 4, 2, 13
    spec = [(24, 200), (16, 301), (32, 150), (64, 401), (128, 37)]
    lats = [gbmc.lattice_init(bits, 2, L, n_replicas=R, seed=seed, instance_base=k) for k, (L, R) in enumerate(spec)]
    pa = gbmc.pa_create(bits, lats, theta, S, beta_f=1.0)
    prof = _kernel_ran(bits, lambda: gbmc.pa_run(bits, pa, capacity=S + 1))
    assert "sweep_bits" in prof and "sweep_resident" in prof
    gbmc.pa_reset(bits, pa, True, 0)
    stats, n = gbmc.pa_run(bits, pa, capacity=S + 1)
    for k, (L, R) in enumerate(spec):
        ref = oracle.pa_run(2, L, seed, k, R, oracle.linear_betas(1.0, S), theta)
        _compare_run(stats, ref, k, L * L)
        np.testing.assert_array_equal(spins_out(bits, lats[k]), ref["spins"])
        par = np.empty(R, dtype=np.uint32)
        gbmc.pa_parents_out(bits, pa, k, par)
        np.testing.assert_array_equal(par, ref["parents"])
    gbmc.pa_free(pa)
    for l in lats:
        gbmc.lattice_free(l)


@pytest.mark.parametrize("L,I,R", [(8, 3, 333), (16, 2, 97)])
def test_bits_pa_3d_ea_instances_match_oracle(bits, L, I, R):
    S, theta, seed = 5, 2, 31
    lat = gbmc.lattice_init(bits, 3, L, model=gbmc.GBMC_EA_PMJ, n_instances=I, n_replicas=R, seed=seed,
                            instance_base=10)
    betas = oracle.linear_betas(2.0, S)
    pa = gbmc.pa_create(bits, [lat], theta, S, schedule=gbmc.GBMC_SCHED_LIST, betas=betas)
    stats, n = gbmc.pa_run(bits, pa, capacity=S + 1)
    got = spins_out(bits, lat).reshape(I, R, -1)
    for i in range(I):
        ref = oracle.pa_run(3, L, seed, 10 + i, R, betas, theta, J=oracle.couplings(L, seed, 10 + i))
        _compare_run(stats, ref, i, L ** 3)
        np.testing.assert_array_equal(got[i], ref["spins"])
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)


def test_bits_pa_3d_mixed_sizes_match_oracle(bits):
    # one annealing step covers 3D +-J lattices with L = 6 (byte-plane kernel), L = 8
    # and L = 16 (bit-sliced kernels, one launch each)
    S, theta, seed = 3, 2, 17
    spec = [(6, 150), (8, 211), (16, 45)]
    lats = [gbmc.lattice_init(bits, 3, L, model=gbmc.GBMC_EA_PMJ, n_replicas=R, seed=seed, instance_base=3 * k)
            for k, (L, R) in enumerate(spec)]
    betas = oracle.linear_betas(1.5, S)
    pa = gbmc.pa_create(bits, lats, theta, S, schedule=gbmc.GBMC_SCHED_LIST, betas=betas)
    prof = _kernel_ran(bits, lambda: gbmc.pa_run(bits, pa, capacity=S + 1))
    assert "sweep_bits" in prof and "sweep_resident" in prof
    gbmc.pa_reset(bits, pa, True, 0)
    stats, n = gbmc.pa_run(bits, pa, capacity=S + 1)
    for k, (L, R) in enumerate(spec):
        ref = oracle.pa_run(3, L, seed, 3 * k, R, betas, theta, J=oracle.couplings(L, seed, 3 * k))
        _compare_run(stats, ref, k, L ** 3)
        np.testing.assert_array_equal(spins_out(bits, lats[k]), ref["spins"])
    gbmc.pa_free(pa)
    for l in lats:
        gbmc.lattice_free(l)


@pytest.mark.parametrize("law", [gbmc.GBMC_RESAMPLE_NEAREST, gbmc.GBMC_RESAMPLE_POISSON])
def test_bits_pa_variable_population_matches_oracle(bits, law):
    # only the live slots are swept: the population size varies from step to step
    L, R0, cap, S, theta, seed = 64, 300, 420, 5, 2, 9
    lat = gbmc.lattice_init(bits, 2, L, n_replicas=cap, seed=seed)
    pa = gbmc.pa_create(bits, [lat], theta, S, resample=law, initial_replicas=R0)
    stats, n = gbmc.pa_run(bits, pa, capacity=S + 1)
    ref = oracle.pa_run_nearest(2, L, seed, 0, R0, cap, oracle.linear_betas(1.0, S), theta,
                                poisson=law == gbmc.GBMC_RESAMPLE_POISSON)
    st = stats[:, 0]
    np.testing.assert_array_equal(st["n_replicas"], ref["nrep"])
    np.testing.assert_array_equal(st["sumE"], ref["sumE"])
    np.testing.assert_allclose(st["lnZ"], ref["lnZ"], rtol=1e-12)
    nlive = int(ref["nrep"][-1])
    np.testing.assert_array_equal(spins_out(bits, lat)[:nlive], ref["spins"])
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)


@pytest.mark.parametrize("L,I,T", [(8, 3, 8), (16, 2, 6)])
def test_bits_parallel_tempering_matches_oracle(bits, L, I, T):
    # every copy at its own temperature: per-copy thresholds in the bit-sliced kernel
    theta, steps, seed = 3, 12, 41
    betas = np.linspace(0.2, 1.4, T)
    lat = gbmc.lattice_init(bits, 3, L, model=gbmc.GBMC_EA_PMJ, n_instances=I, n_replicas=T, seed=seed,
                            instance_base=2)
    pt = gbmc.pt_create(bits, lat, betas, theta)
    gbmc.pt_step(bits, pt, steps)
    rep = np.empty(I * T, dtype=np.uint32)
    acc = np.empty(I * (T - 1), dtype=np.uint32)
    E = np.empty(I * T, dtype=np.int32)
    gbmc.pt_state_out(bits, pt, rep, acc, E)
    gbmc.pt_free(pt)
    got = spins_out(bits, lat).reshape(I, T, -1)
    for i in range(I):
        s, r, a, e = oracle.pt_run(3, L, seed, 2 + i, betas, theta, steps, J=oracle.couplings(L, seed, 2 + i))
        np.testing.assert_array_equal(got[i], s)
        np.testing.assert_array_equal(rep.reshape(I, T)[i], r)
        np.testing.assert_array_equal(acc.reshape(I, T - 1)[i], a)
        np.testing.assert_array_equal(E.reshape(I, T)[i], e)
    gbmc.lattice_free(lat)


def test_sweep_kernel_mode_checks(ctx):
    with pytest.raises(gbmc.GbmcError) as e:
        gbmc.gbmc_set_sweep_kernel(ctx, 7)
    assert e.value.status == gbmc.GBMC_ERR_ARG
    # lattices the bit-sliced kernel does not support take the byte-plane kernel in BITS mode
    gbmc.gbmc_set_sweep_kernel(ctx, BITS)
    try:
        lat = gbmc.lattice_init(ctx, 2, 24, n_replicas=3, seed=2)
        prof = _kernel_ran(ctx, lambda: gbmc.metropolis_sweeps(ctx, lat, 0.4, 2))
        assert "sweep_resident" in prof and "sweep_bits" not in prof
        s = oracle.init_spins(2, 24, 2, 0, 1, True)
        oracle.sweeps(2, 24, s, None, 0.4, 2, 0, 1, 0, 2)
        np.testing.assert_array_equal(spins_out(ctx, lat)[1], s)
        gbmc.lattice_free(lat)
    finally:
        gbmc.gbmc_set_sweep_kernel(ctx, AUTO)
    # the autotuner times the bit-sliced kernel as one more candidate for the classes it supports
    lat = gbmc.lattice_init(ctx, 2, 64, n_replicas=64, seed=1)
    try:
        t = gbmc.gbmc_autotune(ctx, lat, 0.44, 2)
        assert t.kernel in (BITS, BYTES) and math.isfinite(t.ms_per_sweep)
    finally:
        gbmc.gbmc_set_tuning(2, gbmc.GBMC_ISING_FM, 64)  # back to the untuned default
        gbmc.lattice_free(lat)
