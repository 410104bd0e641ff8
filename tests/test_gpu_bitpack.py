"""GPU parity of the bit-packed layout (one bit per spin, per-colour planes):
random start, sweeps, observables and copies agree bit for bit with the oracle
and with the int8 layout (the Philox words depend only on the sites)."""
import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, device_i32, spins_out, torch  # noqa: F401

pytestmark = pytest.mark.gpu
BP = gbmc.GBMC_BITPACK


@pytest.mark.parametrize("L,I,R", [(64, 2, 2), (128, 1, 3)])
def test_packed_random_start_matches_oracle(ctx, L, I, R):
    lat = gbmc.lattice_init(ctx, 2, L, n_instances=I, n_replicas=R, seed=77, instance_base=4, layout=BP)
    assert gbmc.lattice_info(lat).spin_bytes == I * R * L * L // 8
    got = spins_out(ctx, lat)
    ref = np.stack([oracle.init_spins(2, L, 77, 4 + i, r, True) for i in range(I) for r in range(R)])
    np.testing.assert_array_equal(got, ref)
    gbmc.lattice_free(lat)


@pytest.mark.parametrize("L,I,R,n,beta", [(64, 2, 2, 7, 0.4406868), (128, 1, 2, 5, 0.6), (4096, 1, 1, 2, 0.4406868),
                                          (64, 1, 1, 3, 0.0)])
def test_packed_sweeps_match_oracle(ctx, L, I, R, n, beta):
    seed = 3 + L
    lat = gbmc.lattice_init(ctx, 2, L, n_instances=I, n_replicas=R, seed=seed, layout=BP)
    gbmc.lattice_set_sweep_counter(lat, 5)
    Es, Ms = device_i32(n * I * R), device_i32(n * I * R)
    gbmc.metropolis_sweeps(ctx, lat, beta, n, Es, Ms)
    E, M = device_i32(I * R), device_i32(I * R)
    gbmc.observables(ctx, lat, E, M)
    got = spins_out(ctx, lat)
    Es = Es.cpu().numpy().reshape(n, I * R)
    for i in range(I):
        for r in range(R):
            c = i * R + r
            s = oracle.init_spins(2, L, seed, i, r, True)
            for k in range(n):
                oracle.sweeps(2, L, s, None, beta, seed, i, r, 5 + k, 1)
                if L <= 128:
                    assert Es[k, c] == oracle.observables(2, L, s)[0]
            np.testing.assert_array_equal(got[c], s)
            assert (int(E[c]), int(M[c])) == oracle.observables(2, L, s)
    gbmc.lattice_free(lat)


@pytest.mark.parametrize("L,I,R,n,beta", [(1024, 1, 1, 5, 0.4406868), (1024, 1, 3, 3, 0.8), (2048, 2, 1, 4, 0.3),
                                          (4096, 1, 1, 3, 0.4406868), (1024, 1, 20, 2, 0.4406868)])
def test_packed_strip_resident_sweeps_match_oracle(ctx, L, I, R, n, beta):
    # no E/M series: L % 1024 == 0 runs every sweep of the call in one launch
    # (strips of rows in shared memory) when at most SMs / 8 copies; 20 copies
    # take the per-half-sweep launches
    seed = 11 + L
    lat = gbmc.lattice_init(ctx, 2, L, n_instances=I, n_replicas=R, seed=seed, instance_base=2, layout=BP)
    gbmc.lattice_set_sweep_counter(lat, 9)
    n0 = gbmc.gbmc_kernel_launches()
    gbmc.metropolis_sweeps(ctx, lat, beta, n)
    gbmc.metropolis_sweeps(ctx, lat, beta, 1)  # continues the counters
    launches = gbmc.gbmc_kernel_launches() - n0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert launches == (2 if I * R <= sms // 8 else 2 * (n + 1))
    got = spins_out(ctx, lat)
    for i in range(I):
        for r in range(R):
            s = oracle.init_spins(2, L, seed, 2 + i, r, True)
            oracle.sweeps(2, L, s, None, beta, seed, 2 + i, r, 9, n + 1)
            np.testing.assert_array_equal(got[i * R + r], s)
    gbmc.lattice_free(lat)


def test_packed_strips_equal_per_half_sweep_launches(ctx):
    L, n = 4096, 6
    a = gbmc.lattice_init(ctx, 2, L, seed=4, layout=BP)
    b = gbmc.lattice_init(ctx, 2, L, seed=4, layout=BP)
    gbmc.metropolis_sweeps(ctx, a, 0.4406868, n)
    gbmc.gbmc_set_sweep_launch(ctx, gbmc.GBMC_LAUNCH_GRID)
    try:
        gbmc.metropolis_sweeps(ctx, b, 0.4406868, n)
    finally:
        gbmc.gbmc_set_sweep_launch(ctx, gbmc.GBMC_LAUNCH_AUTO)
    np.testing.assert_array_equal(spins_out(ctx, a), spins_out(ctx, b))
    gbmc.lattice_free(a)
    gbmc.lattice_free(b)


def test_packed_equals_int8_layout(ctx):
    L, R, n = 256, 3, 12
    a = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=8, layout=BP)
    b = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=8)
    for lat in (a, b):
        gbmc.metropolis_sweeps(ctx, lat, 0.45, n)
    np.testing.assert_array_equal(spins_out(ctx, a), spins_out(ctx, b))
    gbmc.lattice_free(a)
    gbmc.lattice_free(b)


def test_packed_copy_in_round_trip_and_rejections(ctx):
    L, R = 128, 2
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=1, layout=BP)
    host = np.where(np.random.default_rng(2).random((R, L * L)) < 0.3, -1, 1).astype(np.int8)
    gbmc.lattice_copy_in(ctx, lat, host)
    np.testing.assert_array_equal(spins_out(ctx, lat), host)
    dev = torch.from_numpy(host.reshape(-1)).cuda()
    gbmc.lattice_copy_in(ctx, lat, dev)
    out = torch.zeros_like(dev)
    gbmc.lattice_copy_out(ctx, lat, out)
    np.testing.assert_array_equal(out.cpu().numpy(), host.reshape(-1))
    with pytest.raises(gbmc.GbmcError):
        gbmc.pa_create(ctx, [lat], 2, 3)
    gbmc.lattice_free(lat)
    with pytest.raises(gbmc.GbmcError):
        gbmc.lattice_init(ctx, 2, 96, layout=BP)
    with pytest.raises(gbmc.GbmcError):
        gbmc.lattice_init(ctx, 3, 64, layout=BP)
