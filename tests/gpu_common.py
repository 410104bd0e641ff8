"""Shared fixtures for the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1709_04394_gb300 import build as gbuild  # noqa: E402
from paper_1709_04394_gb300 import gbmc  # noqa: E402


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    gbuild.build()
    torch.cuda.init()
    h = gbmc.gbmc_create(0, torch.cuda.current_stream().cuda_stream)
    yield h
    gbmc.gbmc_destroy(h)


def spins_out(ctx, lat):
    info = gbmc.lattice_info(lat)
    host = np.empty((info.n_copies, info.n_sites), dtype=np.int8)
    gbmc.lattice_copy_out(ctx, lat, host)
    return host


def device_i32(n):
    return torch.zeros(int(n), dtype=torch.int32, device="cuda")
