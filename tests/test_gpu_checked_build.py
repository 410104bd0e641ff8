"""The bounds-checked build (libgbmc_check.so, kernels compiled with
GBMC_CHECK: every instrumented index is verified before its access) run over
small and uneven lattices -- L = 4, 6, 8 in 2D and 3D, copy counts that leave
thread blocks and warps partly empty, every sweep kernel, annealing with both
population laws, parallel tempering, Swendsen-Wang, the double checkerboard,
multi-spin coding and the allocation-free resampling -- must record no failed
check (gbmc_sync reports one as GBMC_ERR_STATE), and give the oracle's spins.
It runs in a child process that loads the checked library."""
import os
import subprocess
import sys

import pytest

from paper_1709_04394_gb300 import build as gbuild
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np, torch
import oracle
from paper_1709_04394_gb300 import gbmc
assert gbmc.gbmc_checked_build()
ctx = gbmc.gbmc_create(0, torch.cuda.current_stream().cuda_stream)
FM, EA = gbmc.GBMC_ISING_FM, gbmc.GBMC_EA_PMJ

def spins(lat):
    info = gbmc.lattice_info(lat)
    h = np.empty((info.n_copies, info.n_sites), dtype=np.int8)
    gbmc.lattice_copy_out(ctx, lat, h)
    return h

checked = 0
for kernel in (gbmc.GBMC_KERNEL_BYTES, gbmc.GBMC_KERNEL_BITS):
    gbmc.gbmc_set_sweep_kernel(ctx, kernel)
    for dim, L, model, I, R in [(2, 4, FM, 1, 3), (2, 6, FM, 2, 5), (2, 8, FM, 1, 7), (2, 16, FM, 2, 9),
                                (2, 32, FM, 1, 3), (2, 64, FM, 1, 5),
                                (2, 128, FM, 1, 3), (3, 4, FM, 1, 3), (3, 6, EA, 2, 3), (3, 8, EA, 3, 5),
                                (3, 8, FM, 1, 21), (3, 16, EA, 2, 3)]:
        lat = gbmc.lattice_init(ctx, dim, L, model=model, n_instances=I, n_replicas=R, seed=3, instance_base=1)
        n = 3
        Es = torch.zeros(n * I * R, dtype=torch.int32, device="cuda")
        gbmc.metropolis_sweeps(ctx, lat, 0.4, n, Es, None)
        gbmc.metropolis_sweeps(ctx, lat, 0.7, 2)
        gbmc.gbmc_sync(ctx)
        got = spins(lat)
        c = R + 1 if I > 1 else R - 1
        s = oracle.init_spins(dim, L, 3, 1 + c // R, c % R, True)
        oracle.sweeps(dim, L, s, oracle.couplings(L, 3, 1 + c // R) if model == EA else None, 0.4, 3, 1 + c // R,
                      c % R, 0, n)
        oracle.sweeps(dim, L, s, oracle.couplings(L, 3, 1 + c // R) if model == EA else None, 0.7, 3, 1 + c // R,
                      c % R, n, 2)
        assert np.array_equal(got[c], s), (dim, L, model, kernel)
        gbmc.lattice_free(lat)
        checked += 1
gbmc.gbmc_set_sweep_kernel(ctx, gbmc.GBMC_KERNEL_AUTO)

# annealing: multinomial (mixed sizes), nearest-integer and Poisson laws, 3D +-J instances
lats = [gbmc.lattice_init(ctx, 2, 4, n_replicas=37, seed=5, instance_base=0),
        gbmc.lattice_init(ctx, 2, 8, n_replicas=45, seed=5, instance_base=1),
        gbmc.lattice_init(ctx, 2, 64, n_replicas=9, seed=5, instance_base=2)]
pa = gbmc.pa_create(ctx, lats, 2, 4)
stats, _ = gbmc.pa_run(ctx, pa, capacity=5)
ref = oracle.pa_run(2, 8, 5, 1, 45, oracle.linear_betas(1.0, 4), 2)
assert np.array_equal(stats[:, 1]["sumE"], ref["sumE"])
gbmc.pa_free(pa)
for l in lats:
    gbmc.lattice_free(l)
for law in (gbmc.GBMC_RESAMPLE_NEAREST, gbmc.GBMC_RESAMPLE_POISSON):
    lat = gbmc.lattice_init(ctx, 3, 4, model=EA, n_instances=2, n_replicas=45, seed=6)
    pa = gbmc.pa_create(ctx, [lat], 2, 4, beta_f=1.5, resample=law, initial_replicas=31)
    gbmc.pa_run(ctx, pa, capacity=5)
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)
lat = gbmc.lattice_init(ctx, 3, 8, model=EA, n_instances=3, n_replicas=23, seed=6)
pa = gbmc.pa_create(ctx, [lat], 2, 3, beta_f=2.0)
gbmc.pa_run(ctx, pa, capacity=4)
gbmc.pa_free(pa)
gbmc.lattice_free(lat)
# adaptive schedule
lat = gbmc.lattice_init(ctx, 2, 6, n_replicas=200, seed=7)
pa = gbmc.pa_create(ctx, [lat], 2, 200, schedule=gbmc.GBMC_SCHED_BISECTION, beta_f=1.0, target_overlap=0.85,
                    dbeta_max=0.2)
gbmc.pa_run(ctx, pa, capacity=201)
gbmc.pa_free(pa)
gbmc.lattice_free(lat)
# parallel tempering
lat = gbmc.lattice_init(ctx, 3, 4, model=EA, n_instances=2, n_replicas=5, seed=8)
pt = gbmc.pt_create(ctx, lat, np.linspace(0.2, 1.0, 5), 2)
gbmc.pt_step(ctx, pt, 5)
gbmc.pt_free(pt)
gbmc.lattice_free(lat)
# Swendsen-Wang (untiled and tiled), double checkerboard, multi-spin coding
for dim, L in [(2, 6), (3, 4), (2, 64), (3, 16)]:
    lat = gbmc.lattice_init(ctx, dim, L, n_replicas=3, seed=9)
    gbmc.swendsen_wang(ctx, lat, 0.4, 2)
    gbmc.lattice_free(lat)
# byte-plane tiles, bit-sliced tiles one launch per round (an E series asked
# for), bit-sliced tiles resident for the whole call
for L, tile, series in [(64, 32, False), (128, 64, True), (256, 128, True), (128, 64, False), (256, 128, False)]:
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=3, seed=10)
    Es = torch.zeros(2 * 3, dtype=torch.int32, device="cuda") if series else None
    gbmc.metropolis_sweeps_dcb(ctx, lat, 0.44, 2, 2, tile, Es, None)
    got = spins(lat)
    s = oracle.init_spins(2, L, 10, 0, 2, True)
    oracle.dcb_sweeps(L, tile, s, 0.44, 10, 0, 2, 0, 2, 2)
    assert np.array_equal(got[2], s), (L, tile)
    gbmc.lattice_free(lat)
    checked += 1
lat = gbmc.lattice_init(ctx, 2, 16, n_replicas=33, seed=11)
gbmc.metropolis_sweeps_msc(ctx, lat, 0.44, 3)
gbmc.lattice_free(lat)
# the allocation-free resampling
E = torch.tensor(4 * np.random.default_rng(1).integers(-8, 8, 3 * 50), dtype=torch.int32, device="cuda")
par = torch.empty(150, dtype=torch.int32, device="cuda")
q = torch.empty(3, dtype=torch.float64, device="cuda")
gbmc.pa_resample_static(torch.cuda.current_stream().cuda_stream, 0, 2, 16, 3, 50, 0, 1, 1, 0.3, E, par, q)
gbmc.gbmc_sync(ctx)
gbmc.gbmc_destroy(ctx)
print("checked ok", checked)
'''


def test_checked_build_records_no_bounds_failure():
    require_gpu()
    gbuild.build(check=True)
    env = dict(os.environ, GBMC_LIBRARY="libgbmc_check.so")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked ok 29" in r.stdout
