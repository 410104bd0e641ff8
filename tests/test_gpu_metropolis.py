"""GPU parity: initial states, couplings, checkerboard sweeps and observables of
the CUDA library against the CPU oracle, element by element (bit-exact: spins,
couplings and integer energies are integers)."""
import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, device_i32, spins_out, torch  # noqa: F401

pytestmark = pytest.mark.gpu

BETA_C = 0.4406868


def _oracle_copies(dim, L, n_inst, R, seed, start_random, inst_base=0):
    return np.stack([oracle.init_spins(dim, L, seed, inst_base + i, r, start_random)
                     for i in range(n_inst) for r in range(R)])


@pytest.mark.parametrize("dim,L,n_inst,R", [(2, 64, 2, 3), (2, 6, 1, 5), (3, 8, 3, 2), (2, 2, 1, 1)])
def test_random_start_matches_oracle(ctx, dim, L, n_inst, R):
    lat = gbmc.lattice_init(ctx, dim, L, start=gbmc.GBMC_START_RANDOM, n_instances=n_inst, n_replicas=R,
                            seed=0xDEADBEEF12345, instance_base=7)
    got = spins_out(ctx, lat)
    np.testing.assert_array_equal(got, _oracle_copies(dim, L, n_inst, R, 0xDEADBEEF12345, True, 7))
    gbmc.lattice_free(lat)


def test_couplings_match_oracle(ctx):
    L, I = 8, 4
    lat = gbmc.lattice_init(ctx, 3, L, model=gbmc.GBMC_EA_PMJ, n_instances=I, n_replicas=1, seed=99,
                            instance_base=3)
    J = np.empty(I * L ** 3 * 3, dtype=np.int8)
    gbmc.lattice_couplings_out(ctx, lat, J)
    J = J.reshape(I, L ** 3, 3)
    for i in range(I):
        np.testing.assert_array_equal(J[i], oracle.couplings(L, 99, 3 + i))
    gbmc.lattice_free(lat)


def test_config_l16_series_matches_oracle(ctx):
    # 2D Ising L = 16, beta = 0.4406868, all-up, 10^4 sweeps, Philox seed 1, E and M per sweep
    L, n = 16, 10000
    lat = gbmc.lattice_init(ctx, 2, L, start=gbmc.GBMC_START_ALL_UP, seed=1)
    Es, Ms = device_i32(n), device_i32(n)
    gbmc.metropolis_sweeps(ctx, lat, BETA_C, n, Es, Ms)
    torch.cuda.synchronize()
    s = oracle.init_spins(2, L, 1, 0, 0, False)
    E_or = np.empty(n, dtype=np.int64)
    M_or = np.empty(n, dtype=np.int64)
    for t in range(n):
        oracle.sweeps(2, L, s, None, BETA_C, 1, 0, 0, t, 1)
        E_or[t], M_or[t] = oracle.observables(2, L, s)
    np.testing.assert_array_equal(Es.cpu().numpy(), E_or)
    np.testing.assert_array_equal(Ms.cpu().numpy(), M_or)
    np.testing.assert_array_equal(spins_out(ctx, lat)[0], s)
    assert gbmc.lattice_info(lat).sweep_counter == n
    gbmc.lattice_free(lat)


CASES = [
    # dim, L, model, n_inst, R, beta, sweeps   (SWAR path for L % 8 == 0, per-site otherwise)
    (2, 64, gbmc.GBMC_ISING_FM, 1, 5, BETA_C, 40),
    (2, 24, gbmc.GBMC_ISING_FM, 2, 3, 0.3, 25),
    (2, 8, gbmc.GBMC_ISING_FM, 1, 40, 0.6, 20),
    (2, 6, gbmc.GBMC_ISING_FM, 1, 7, BETA_C, 30),
    (2, 10, gbmc.GBMC_ISING_FM, 2, 2, 1.0, 30),
    (2, 2, gbmc.GBMC_ISING_FM, 1, 3, 0.2, 50),
    (2, 128, gbmc.GBMC_ISING_FM, 1, 2, 0.5, 10),
    (3, 8, gbmc.GBMC_ISING_FM, 1, 4, 0.22, 20),
    (3, 6, gbmc.GBMC_ISING_FM, 1, 3, 0.3, 20),
    (3, 8, gbmc.GBMC_EA_PMJ, 3, 2, 0.9, 20),
    (3, 4, gbmc.GBMC_EA_PMJ, 2, 3, 1.5, 20),
    (3, 16, gbmc.GBMC_EA_PMJ, 1, 2, 0.7, 10),
    (2, 64, gbmc.GBMC_ISING_FM, 1, 3, 0.0, 3),  # beta = 0: every spin flips
]


@pytest.mark.parametrize("dim,L,model,n_inst,R,beta,n", CASES)
def test_sweeps_match_oracle(ctx, dim, L, model, n_inst, R, beta, n):
    seed = 1234 + L
    lat = gbmc.lattice_init(ctx, dim, L, model=model, n_instances=n_inst, n_replicas=R, seed=seed,
                            instance_base=1)
    gbmc.lattice_set_sweep_counter(lat, 17)
    # two calls: counters continue across calls
    gbmc.metropolis_sweeps(ctx, lat, beta, n // 2)
    ncop = n_inst * R
    Es, Ms = device_i32((n - n // 2) * ncop), device_i32((n - n // 2) * ncop)
    gbmc.metropolis_sweeps(ctx, lat, beta, n - n // 2, Es, Ms)
    E, M = device_i32(ncop), device_i32(ncop)
    gbmc.observables(ctx, lat, E, M)
    got = spins_out(ctx, lat)
    Es = Es.cpu().numpy().reshape(-1, ncop)
    Ms = Ms.cpu().numpy().reshape(-1, ncop)
    for i in range(n_inst):
        J = oracle.couplings(L, seed, 1 + i) if model == gbmc.GBMC_EA_PMJ else None
        for r in range(R):
            c = i * R + r
            s = oracle.init_spins(dim, L, seed, 1 + i, r, True)
            oracle.sweeps(dim, L, s, J, beta, seed, 1 + i, r, 17, n // 2)
            for k in range(n - n // 2):
                oracle.sweeps(dim, L, s, J, beta, seed, 1 + i, r, 17 + n // 2 + k, 1)
                assert (Es[k, c], Ms[k, c]) == oracle.observables(dim, L, s, J), (c, k)
            np.testing.assert_array_equal(got[c], s, err_msg="copy %d" % c)
            assert (int(E[c]), int(M[c])) == oracle.observables(dim, L, s, J)
    gbmc.lattice_free(lat)


@pytest.mark.parametrize("mode", [gbmc.GBMC_LAUNCH_AUTO, gbmc.GBMC_LAUNCH_GRID])
@pytest.mark.parametrize("L,n,chunks", [(512, 6, (6,)), (512, 3, (1, 2)), (4096, 2, (2,)), (384, 9, (4, 5)),
                                        (768, 2, (2,)), (520, 2, (2,))])
def test_large_lattice_paths_match_oracle(ctx, L, n, chunks, mode):
    # lattices too large for shared memory, L % 128 == 0: strips of rows resident
    # in shared memory for a whole call (AUTO) or tiled sweeps (GRID: up to 4
    # sweeps per launch, any chunking); else global half-sweeps. L = 4096 is the
    # benchmark size
    lat = gbmc.lattice_init(ctx, 2, L, seed=1)
    gbmc.gbmc_set_sweep_launch(ctx, mode)
    try:
        for c in chunks:
            gbmc.metropolis_sweeps(ctx, lat, BETA_C, c)
    finally:
        gbmc.gbmc_set_sweep_launch(ctx, gbmc.GBMC_LAUNCH_AUTO)
    E, M = device_i32(1), device_i32(1)
    gbmc.observables(ctx, lat, E, M)
    got = spins_out(ctx, lat)[0]
    s = oracle.init_spins(2, L, 1, 0, 0, True)
    oracle.sweeps(2, L, s, None, BETA_C, 1, 0, 0, 0, n)
    np.testing.assert_array_equal(got, s)
    assert (int(E[0]), int(M[0])) == oracle.observables(2, L, s)
    gbmc.lattice_free(lat)


@pytest.mark.parametrize("kernel", [gbmc.GBMC_KERNEL_BYTES, gbmc.GBMC_KERNEL_AUTO])
@pytest.mark.parametrize("L,I,R,n,beta", [(1024, 1, 3, 4, 0.6), (2048, 2, 1, 3, 0.3), (4096, 1, 2, 2, 0.2)])
def test_strip_resident_sweeps_several_copies(ctx, L, I, R, n, beta, kernel):
    # every sweep of a call in one strip launch, strips of every copy side by side;
    # counters continue. BYTES: the int8 strips (one launch per call); AUTO: the
    # configuration packed to bits, the bit-packed strips, unpacked (three launches)
    lat = gbmc.lattice_init(ctx, 2, L, n_instances=I, n_replicas=R, seed=21, instance_base=5)
    gbmc.lattice_set_sweep_counter(lat, 3)
    gbmc.gbmc_set_sweep_kernel(ctx, kernel)
    try:
        n0 = gbmc.gbmc_kernel_launches()
        gbmc.metropolis_sweeps(ctx, lat, beta, n - 1)
        gbmc.metropolis_sweeps(ctx, lat, beta, 1)
        assert gbmc.gbmc_kernel_launches() - n0 == (2 if kernel == gbmc.GBMC_KERNEL_BYTES else 6)
    finally:
        gbmc.gbmc_set_sweep_kernel(ctx, gbmc.GBMC_KERNEL_AUTO)
    got = spins_out(ctx, lat)
    for i in range(I):
        for r in range(R):
            s = oracle.init_spins(2, L, 21, 5 + i, r, True)
            oracle.sweeps(2, L, s, None, beta, 21, 5 + i, r, 3, n)
            np.testing.assert_array_equal(got[i * R + r], s)
    gbmc.lattice_free(lat)


def test_tiled_path_series_and_caller_buffer(ctx):
    L, n, R = 256 + 256, 3, 2
    buf = torch.zeros(R * L * L, dtype=torch.int8, device="cuda")
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=9, instance_base=2, spins=buf)
    Es, Ms = device_i32(n * R), device_i32(n * R)
    gbmc.metropolis_sweeps(ctx, lat, 0.5, n, Es, Ms)
    torch.cuda.synchronize()
    got = buf.cpu().numpy().reshape(R, -1)  # the caller's buffer holds the result
    Es = Es.cpu().numpy().reshape(n, R)
    for r in range(R):
        s = oracle.init_spins(2, L, 9, 2, r, True)
        for k in range(n):
            oracle.sweeps(2, L, s, None, 0.5, 9, 2, r, k, 1)
            assert Es[k, r] == oracle.observables(2, L, s)[0]
        np.testing.assert_array_equal(got[r], s)
    gbmc.lattice_free(lat)


def test_caller_owned_buffer_and_copy_in(ctx):
    L, R = 16, 4
    buf = torch.zeros(R * L * L, dtype=torch.int8, device="cuda")
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=5, spins=buf)
    assert gbmc.lattice_info(lat).spins_dev == buf.data_ptr()
    host = np.where(np.random.default_rng(3).random((R, L * L)) < 0.5, 1, -1).astype(np.int8)
    gbmc.lattice_copy_in(ctx, lat, host)
    gbmc.metropolis_sweeps(ctx, lat, 0.35, 4)
    torch.cuda.synchronize()
    got = buf.cpu().numpy().reshape(R, -1)
    for r in range(R):
        s = host[r].copy()
        oracle.sweeps(2, L, s, None, 0.35, 5, 0, r, 0, 4)
        np.testing.assert_array_equal(got[r], s)
    gbmc.lattice_free(lat)


def test_invalid_arguments_are_rejected(ctx):
    with pytest.raises(gbmc.GbmcError) as e:
        gbmc.lattice_init(ctx, 2, 7)
    assert e.value.status == gbmc.GBMC_ERR_ARG
    with pytest.raises(gbmc.GbmcError):
        gbmc.lattice_init(ctx, 2, 16, n_replicas=0)
    with pytest.raises(gbmc.GbmcError):
        gbmc.lattice_init(ctx, 2, 16, model=gbmc.GBMC_EA_PMJ)
    lat = gbmc.lattice_init(ctx, 2, 16)
    with pytest.raises(gbmc.GbmcError):
        gbmc.metropolis_sweeps(ctx, lat, -0.1, 1)
    with pytest.raises(gbmc.GbmcError):
        gbmc.metropolis_sweeps(ctx, lat, 1000.0, 1)
    small = torch.zeros(10, dtype=torch.int8, device="cuda")
    with pytest.raises(gbmc.GbmcError):
        gbmc.lattice_init(ctx, 2, 16, spins=small)
    gbmc.lattice_free(lat)
