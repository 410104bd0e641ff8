"""pa_resample_static: the resampling step for callers that must not allocate
device memory (processes whose device memory belongs to another allocator or
pool, drivers that reserve all memory at start-up, latency-critical code that
cannot take the implicit synchronisation of cudaMalloc / cudaFree). Its scratch
lives in a fixed array inside the library, so it must give exactly what the
allocating path gives: the same parent map as pa_step (bit for bit) and the
same ln Q (to the 1e-12 relative tolerance of the other tests), here on two
calls in a row; both are also checked against the oracle's resampling of the
same energies. This file runs last so that a failure here leaves the rest of
the suite already run; it also passes on its own in a fresh process."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

from paper_1709_04394_gb300 import build as gbuild  # noqa: E402
from paper_1709_04394_gb300 import gbmc  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gbuild.build()
    h = gbmc.gbmc_create(0, torch.cuda.current_stream().cuda_stream)
    yield h
    gbmc.gbmc_destroy(h)


@pytest.mark.parametrize("dim,L,model,I,R", [(2, 16, gbmc.GBMC_ISING_FM, 1, 3000),
                                             (3, 8, gbmc.GBMC_EA_PMJ, 3, 700)])
def test_static_resample_matches_pa_step_on_two_calls_in_a_row(ctx, dim, L, model, I, R):
    seed, base = 21, 5
    stream = torch.cuda.current_stream().cuda_stream
    lat = gbmc.lattice_init(ctx, dim, L, model=model, n_instances=I, n_replicas=R, seed=seed, instance_base=base)
    pa = gbmc.pa_create(ctx, [lat], 2, 6, beta_f=1.5)
    E = torch.empty(I * R, dtype=torch.int32, device="cuda")
    parent = torch.empty(I * R, dtype=torch.int32, device="cuda")
    lnQ = torch.empty(I, dtype=torch.float64, device="cuda")
    for step in (1, 2):
        gbmc.pa_energies_out(ctx, pa, 0, E)        # the population the step resamples
        row = gbmc.pa_step(ctx, pa)                 # allocating path
        ref = np.empty(I * R, dtype=np.uint32)
        gbmc.pa_parents_out(ctx, pa, 0, ref)
        parent.fill_(-1)
        gbmc.pa_resample_static(stream, 0, dim, L ** dim, I, R, base, seed, step, float(row[0]["dbeta"]),
                                E, parent, lnQ)
        torch.cuda.synchronize()
        got = parent.cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got, ref)
        np.testing.assert_allclose(lnQ.cpu().numpy(), row["lnQ"], rtol=RTOL, atol=0)
        # the oracle's multinomial resampling of the same energies
        En = E.cpu().numpy().astype(np.int64).reshape(I, R)
        for i in range(I):
            counts, lnQ_ref = oracle.resample(En[i], float(row[0]["dbeta"]), seed, base + i, step)
            np.testing.assert_array_equal(got.reshape(I, R)[i], oracle.children_order(counts))
            assert lnQ.cpu().numpy()[i] == pytest.approx(lnQ_ref, rel=RTOL)
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)


def test_static_resample_rejects_sizes_beyond_its_limit(ctx):
    stream = torch.cuda.current_stream().cuda_stream
    E = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    q = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(gbmc.GbmcError) as e:
        gbmc.pa_resample_static(stream, 0, 2, 4096, 1, 200000, 0, 1, 1, 0.01, E, out, q)
    assert e.value.status == gbmc.GBMC_ERR_ARG and "131072" in str(e.value)
    with pytest.raises(gbmc.GbmcError):
        gbmc.pa_resample_static(stream, 0, 2, 1 << 20, 1, 4, 0, 1, 1, 0.01, E, out, q)


def test_static_resample_clamps_energies_outside_the_lattice_range(ctx):
    # energies beyond [-dim N, dim N] are clamped into it: the call succeeds
    # and every parent is a valid replica index
    stream = torch.cuda.current_stream().cuda_stream
    dim, L, R = 2, 8, 500
    N = L ** dim
    rng = np.random.default_rng(3)
    E = torch.tensor(4 * rng.integers(-3 * N, 3 * N, R) + 2, dtype=torch.int32, device="cuda")
    parent = torch.full((R,), -1, dtype=torch.int32, device="cuda")
    lnQ = torch.zeros(1, dtype=torch.float64, device="cuda")
    gbmc.pa_resample_static(stream, 0, dim, N, 1, R, 0, 5, 1, 0.3, E, parent, lnQ)
    torch.cuda.synchronize()
    par = parent.cpu().numpy()
    assert par.min() >= 0 and par.max() < R
    assert np.all(np.diff(par) >= 0)  # children contiguous, parents in order
    assert np.isfinite(lnQ.cpu().numpy()).all()


def test_static_resample_allocates_no_device_memory(ctx):
    # after a first call (which may load the library's kernels), further calls
    # leave the device's free memory unchanged
    stream = torch.cuda.current_stream().cuda_stream
    I, R, N = 2, 4000, 64 * 64
    E = torch.tensor(4 * np.random.default_rng(1).integers(-N // 2, N // 2, I * R), dtype=torch.int32, device="cuda")
    parent = torch.empty(I * R, dtype=torch.int32, device="cuda")
    lnQ = torch.empty(I, dtype=torch.float64, device="cuda")
    gbmc.pa_resample_static(stream, 0, 2, N, I, R, 0, 9, 1, 0.01, E, parent, lnQ)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    for step in range(2, 6):
        gbmc.pa_resample_static(stream, 0, 2, N, I, R, 0, 9, step, 0.01, E, parent, lnQ)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(0)[0] == free0
