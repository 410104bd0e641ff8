"""GPU parity of the double-checkerboard sweeps with k hits per tile
(Sec. 3.1, Fig. 5 right): spins, per-round E and M and the sweep counter
against the oracle's tile-by-tile order, bit for bit. Calls that ask for a
per-round E/M series run one launch per coarse colour and round; calls that
do not run every round in one launch with the tiles resident (64 and 128
tiles)."""
import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, device_i32, spins_out, torch  # noqa: F401

pytestmark = pytest.mark.gpu

BETA_C = 0.4406868


AUTO, BYTES = gbmc.GBMC_KERNEL_AUTO, gbmc.GBMC_KERNEL_BYTES


@pytest.fixture(params=[AUTO, BYTES], ids=["default", "bytes"])
def kernel(request, ctx):
    """Tiles of 64 and 128 sites run bit-sliced by default; BYTES forces the
    byte-plane tiles (the only kernel for 32)."""
    gbmc.gbmc_set_sweep_kernel(ctx, request.param)
    yield request.param
    gbmc.gbmc_set_sweep_kernel(ctx, AUTO)


@pytest.mark.parametrize("L,tile,k,rounds,R,beta", [
    (64, 32, 3, 2, 3, BETA_C),
    (256, 64, 1, 3, 2, 0.3),
    (256, 128, 4, 1, 1, 0.6),
    (512, 64, 10, 1, 1, BETA_C),
    (128, 32, 2, 2, 5, 0.0),        # beta = 0: every visit flips
    (128, 64, 3, 2, 2, 0.0),        # 2 x 2 tiles: both halo columns of a tile are the same tile
    (256, 128, 2, 2, 3, 0.0),
    (512, 128, 5, 2, 2, 1.2),       # cold: few flips
    (4096, 64, 10, 1, 1, BETA_C),   # the benchmark lattice, whole
])
def test_dcb_matches_oracle(ctx, kernel, L, tile, k, rounds, R, beta):
    if L >= 4096 and kernel == BYTES:
        pytest.skip("the byte-plane tiles are checked at full size by the bits-equals-bytes test")
    seed = 11 + L
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=seed, instance_base=2)
    gbmc.lattice_set_sweep_counter(lat, 5)
    Es, Ms = device_i32(rounds * R), device_i32(rounds * R)
    gbmc.metropolis_sweeps_dcb(ctx, lat, beta, rounds, k, tile, Es, Ms)
    got = spins_out(ctx, lat)
    Es = Es.cpu().numpy().reshape(rounds, R)
    Ms = Ms.cpu().numpy().reshape(rounds, R)
    for r in range(R):
        s = oracle.init_spins(2, L, seed, 2, r, True)
        for m in range(rounds):
            oracle.dcb_sweeps(L, tile, s, beta, seed, 2, r, 5 + m * k, k, 1)
            assert (Es[m, r], Ms[m, r]) == oracle.observables(2, L, s), (r, m)
        np.testing.assert_array_equal(got[r], s, err_msg="replica %d" % r)
    assert gbmc.lattice_info(lat).sweep_counter == 5 + rounds * k
    gbmc.lattice_free(lat)


def test_dcb_continues_counters_and_mixes_with_plain_sweeps(ctx):
    L, tile, seed = 128, 32, 4
    a = gbmc.lattice_init(ctx, 2, L, n_replicas=2, seed=seed)
    b = gbmc.lattice_init(ctx, 2, L, n_replicas=2, seed=seed)
    gbmc.metropolis_sweeps(ctx, a, 0.5, 3)
    gbmc.metropolis_sweeps_dcb(ctx, a, 0.5, 1, 2, tile)
    gbmc.metropolis_sweeps_dcb(ctx, a, 0.5, 1, 2, tile)
    gbmc.metropolis_sweeps(ctx, b, 0.5, 3)
    gbmc.metropolis_sweeps_dcb(ctx, b, 0.5, 2, 2, tile)
    ga, gb = spins_out(ctx, a), spins_out(ctx, b)
    np.testing.assert_array_equal(ga, gb)
    for r in range(2):
        s = oracle.init_spins(2, L, seed, 0, r, True)
        oracle.sweeps(2, L, s, None, 0.5, seed, 0, r, 0, 3)
        oracle.dcb_sweeps(L, tile, s, 0.5, seed, 0, r, 3, 2, 2)
        np.testing.assert_array_equal(ga[r], s)
        plain = oracle.init_spins(2, L, seed, 0, r, True)
        oracle.sweeps(2, L, plain, None, 0.5, seed, 0, r, 0, 7)
        assert not np.array_equal(plain, s)  # same random words, another order
    assert gbmc.lattice_info(a).sweep_counter == 7
    gbmc.lattice_free(a)
    gbmc.lattice_free(b)


def test_dcb_rejects_unsupported_lattices(ctx):
    lat = gbmc.lattice_init(ctx, 2, 96, seed=1)
    for tile in (48, 64):  # 48: no kernel; 64: 96 is not a multiple of 128
        with pytest.raises(gbmc.GbmcError) as e:
            gbmc.metropolis_sweeps_dcb(ctx, lat, 0.4, 1, 1, tile)
        assert e.value.status == gbmc.GBMC_ERR_ARG
    gbmc.lattice_free(lat)
    lat = gbmc.lattice_init(ctx, 2, 128, seed=1)
    with pytest.raises(gbmc.GbmcError):
        gbmc.metropolis_sweeps_dcb(ctx, lat, 0.4, 1, 0, 32)  # k = 0
    gbmc.lattice_free(lat)
    for kw in (dict(dim=3, L=64), dict(dim=2, L=64, layout=gbmc.GBMC_BITPACK)):
        lat = gbmc.lattice_init(ctx, kw.pop("dim"), kw.pop("L"), seed=1, **kw)
        with pytest.raises(gbmc.GbmcError):
            gbmc.metropolis_sweeps_dcb(ctx, lat, 0.4, 1, 1, 32)
        gbmc.lattice_free(lat)


def _dcb_run(ctx, kernel, L, tile, k, rounds, R, seed, beta):
    gbmc.gbmc_set_sweep_kernel(ctx, kernel)
    try:
        lat = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=seed)
        gbmc.lattice_set_sweep_counter(lat, 17)
        E, M = device_i32(rounds * R), device_i32(rounds * R)
        gbmc.gbmc_profile(ctx, True)
        gbmc.metropolis_sweeps_dcb(ctx, lat, beta, rounds, k, tile, E, M)
        prof = {name: n for name, (n, _) in gbmc.gbmc_profile_read(ctx).items()}
        gbmc.gbmc_profile(ctx, False)
        out = (spins_out(ctx, lat), E.cpu().numpy(), M.cpu().numpy())
        gbmc.lattice_free(lat)
    finally:
        gbmc.gbmc_set_sweep_kernel(ctx, AUTO)
    return out, prof


@pytest.mark.parametrize("L,tile,k,rounds,R,beta", [
    (1024, 64, 5, 3, 2, BETA_C),
    (1024, 128, 7, 2, 3, 0.35),
    (4096, 64, 10, 2, 1, BETA_C),   # the benchmark's launch configuration, two rounds
    (4096, 128, 3, 1, 1, 0.6),
])
def test_dcb_bits_equals_bytes(ctx, L, tile, k, rounds, R, beta):
    """The bit-sliced tiles (the default for 64 and 128) and the byte-plane
    tiles give the same spins and observables, bit for bit, from a random
    start; each call runs only its own kernel, two launches per round."""
    a, pa = _dcb_run(ctx, AUTO, L, tile, k, rounds, R, 5 + L, beta)
    b, pb = _dcb_run(ctx, BYTES, L, tile, k, rounds, R, 5 + L, beta)
    assert pa.get("sweep_dcb_bits") == 2 * rounds and "sweep_dcb" not in pa
    assert pb.get("sweep_dcb") == 2 * rounds and "sweep_dcb_bits" not in pb
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.fixture()
def persistent(ctx):
    """Every round of a call in one resident launch, whatever k."""
    gbmc.gbmc_set_sweep_launch(ctx, gbmc.GBMC_LAUNCH_PERSISTENT)
    yield
    gbmc.gbmc_set_sweep_launch(ctx, gbmc.GBMC_LAUNCH_AUTO)


@pytest.mark.parametrize("L,tile,k,rounds,R,beta", [
    (128, 64, 3, 2, 2, 0.0),        # 2 x 2 tiles: a CTA's two tiles are each other's left and right halo
    (256, 64, 1, 3, 2, 0.3),
    (256, 128, 4, 2, 3, 0.6),
    (512, 64, 10, 2, 1, BETA_C),
    (512, 128, 5, 2, 2, 1.2),
    (4096, 64, 10, 1, 1, BETA_C),   # the benchmark lattice, whole
])
def test_dcb_resident_matches_oracle(ctx, persistent, L, tile, k, rounds, R, beta):
    seed = 21 + L
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=seed, instance_base=1)
    gbmc.lattice_set_sweep_counter(lat, 9)
    gbmc.gbmc_profile(ctx, True)
    gbmc.metropolis_sweeps_dcb(ctx, lat, beta, rounds, k, tile)
    prof = gbmc.gbmc_profile_read(ctx)
    gbmc.gbmc_profile(ctx, False)
    assert prof["sweep_dcb_resident"][0] == 1 and "sweep_dcb_bits" not in prof
    got = spins_out(ctx, lat)
    for r in range(R):
        s = oracle.init_spins(2, L, seed, 1, r, True)
        oracle.dcb_sweeps(L, tile, s, beta, seed, 1, r, 9, k, rounds)
        np.testing.assert_array_equal(got[r], s, err_msg="replica %d" % r)
    assert gbmc.lattice_info(lat).sweep_counter == 9 + rounds * k
    gbmc.lattice_free(lat)


@pytest.mark.parametrize("L,tile,k,rounds,R", [
    (4096, 64, 10, 100, 1),   # the benchmark's call: 100 rounds of k = 10 in one launch
    (1024, 128, 3, 40, 2),
    (2048, 64, 1, 60, 3),
])
def test_dcb_resident_equals_per_round_launches(ctx, L, tile, k, rounds, R):
    """Many rounds in one resident launch (progress counters up to rounds + 1)
    against one launch per coarse colour and round, from the same random
    start: the same spins, bit for bit."""
    out = []
    for mode in (gbmc.GBMC_LAUNCH_PERSISTENT, gbmc.GBMC_LAUNCH_GRID):
        gbmc.gbmc_set_sweep_launch(ctx, mode)
        try:
            lat = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=31, instance_base=4)
            gbmc.gbmc_profile(ctx, True)
            gbmc.metropolis_sweeps_dcb(ctx, lat, BETA_C, rounds, k, tile)
            prof = gbmc.gbmc_profile_read(ctx)
            gbmc.gbmc_profile(ctx, False)
        finally:
            gbmc.gbmc_set_sweep_launch(ctx, gbmc.GBMC_LAUNCH_AUTO)
        if mode == gbmc.GBMC_LAUNCH_GRID:
            assert prof["sweep_dcb_bits"][0] == 2 * rounds and "sweep_dcb_resident" not in prof
        else:
            assert prof["sweep_dcb_resident"][0] == 1 and "sweep_dcb_bits" not in prof
        out.append(spins_out(ctx, lat))
        gbmc.lattice_free(lat)
    np.testing.assert_array_equal(out[0], out[1])


@pytest.mark.parametrize("tile,k,kind", [
    (64, 3, "sweep_dcb_resident"), (64, 4, "sweep_dcb_bits"), (64, 10, "sweep_dcb_bits"),
    (128, 7, "sweep_dcb_resident"), (128, 8, "sweep_dcb_bits"),
])
def test_dcb_auto_launch_choice(ctx, tile, k, kind):
    """AUTO: one resident launch per call for small k, per-round launches for
    larger k or when an E/M series is asked for."""
    lat = gbmc.lattice_init(ctx, 2, 512, seed=2)
    for series in (None, device_i32(2)):
        gbmc.gbmc_profile(ctx, True)
        gbmc.metropolis_sweeps_dcb(ctx, lat, BETA_C, 2, k, tile, series, None)
        prof = gbmc.gbmc_profile_read(ctx)
        gbmc.gbmc_profile(ctx, False)
        assert set(prof) & {"sweep_dcb_resident", "sweep_dcb_bits"} == \
            {kind if series is None else "sweep_dcb_bits"}
    gbmc.lattice_free(lat)


def test_dcb_resident_neighbour_wait_runs_out_and_is_reported(ctx):
    """Every neighbour wait of the resident double checkerboard is bounded: with
    one phantom round asked for, the first waits run out, the kernel returns
    without storing, the host reports GBMC_ERR_TIMEOUT and the context and
    lattice stay usable."""
    L, tile = 256, 64
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=2, seed=12)
    before = spins_out(ctx, lat)
    gbmc.gbmc_test_barrier_wait(ctx, 1, 2_000_000)  # ~1 ms budget, one phantom round
    try:
        gbmc.metropolis_sweeps_dcb(ctx, lat, 0.44, 2, 2, tile)  # k = 2: the resident launch
        with pytest.raises(gbmc.GbmcError) as e:
            gbmc.gbmc_sync(ctx)
        assert e.value.status == gbmc.GBMC_ERR_TIMEOUT
    finally:
        gbmc.gbmc_test_barrier_wait(ctx, 0, 2_000_000_000)
    gbmc.gbmc_sync(ctx)
    np.testing.assert_array_equal(spins_out(ctx, lat), before)  # no tile was stored
    gbmc.lattice_set_sweep_counter(lat, 0)
    gbmc.metropolis_sweeps_dcb(ctx, lat, 0.44, 2, 2, tile)
    got = spins_out(ctx, lat)
    for r in range(2):
        s = oracle.init_spins(2, L, 12, 0, r, True)
        oracle.dcb_sweeps(L, tile, s, 0.44, 12, 0, r, 0, 2, 2)
        np.testing.assert_array_equal(got[r], s)
    gbmc.lattice_free(lat)


def test_dcb_resident_falls_back_when_tiles_do_not_fit(ctx):
    """L = 8192 with 64 x 64 tiles has 8192 tile pairs, more than the device
    holds at once: k = 2 (a resident launch under AUTO) takes the per-round
    launches instead, with the spins of the byte-plane tiles."""
    L, tile, k, rounds = 8192, 64, 2, 1
    out = []
    for kernel in (AUTO, BYTES):
        gbmc.gbmc_set_sweep_kernel(ctx, kernel)
        try:
            lat = gbmc.lattice_init(ctx, 2, L, seed=23)
            gbmc.gbmc_profile(ctx, True)
            gbmc.metropolis_sweeps_dcb(ctx, lat, BETA_C, rounds, k, tile)
            prof = gbmc.gbmc_profile_read(ctx)
            gbmc.gbmc_profile(ctx, False)
        finally:
            gbmc.gbmc_set_sweep_kernel(ctx, AUTO)
        if kernel == AUTO:
            assert prof["sweep_dcb_bits"][0] == 2 * rounds and "sweep_dcb_resident" not in prof
        out.append(spins_out(ctx, lat))
        gbmc.lattice_free(lat)
    np.testing.assert_array_equal(out[0], out[1])
