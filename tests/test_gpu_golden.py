"""The library against the stored fixtures of tests/golden/ (written from the
oracle by tests/golden/make_golden.py): the first 500 sweeps of the L = 16
series workload and a short annealing run, without running the oracle."""
import math
import os

import numpy as np
import pytest

from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, device_i32, torch  # noqa: F401

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_series_matches_fixture(ctx):
    rows = np.loadtxt(os.path.join(GOLDEN, "config1_L16_series.txt"), comments="#").astype(np.int64)
    n = rows.shape[0]
    lat = gbmc.lattice_init(ctx, 2, 16, start=gbmc.GBMC_START_ALL_UP, seed=1)
    Es, Ms = device_i32(n), device_i32(n)
    gbmc.metropolis_sweeps(ctx, lat, 0.4406868, n, Es, Ms)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Es.cpu().numpy(), rows[:, 1])
    np.testing.assert_array_equal(Ms.cpu().numpy(), rows[:, 2])
    gbmc.lattice_free(lat)


def test_pa_matches_fixture(ctx):
    rows = np.loadtxt(os.path.join(GOLDEN, "pa_L8_R2000.txt"), comments="#")
    lat = gbmc.lattice_init(ctx, 2, 8, n_replicas=2000, seed=6)
    pa = gbmc.pa_create(ctx, [lat], 3, 40)
    stats, n = gbmc.pa_run(ctx, pa, capacity=41)
    assert n == 40
    np.testing.assert_array_equal(stats[:, 0]["sumE"], rows[:, 2].astype(np.int64))
    np.testing.assert_allclose(stats[:, 0]["lnZ"], rows[:, 3], rtol=1e-12, atol=0)
    assert stats[0, 0]["lnZ"] == 64 * math.log(2.0)
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)
