"""GPU parity of parallel tempering (Sec. 5.1, Eq. (10)) on the shared sweep
kernel: configurations, temperature maps, accepted-swap counts and energies
bit for bit against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, spins_out, torch  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,L,model,I,T,theta,steps", [(3, 8, gbmc.GBMC_EA_PMJ, 3, 8, 3, 20),
                                                         (2, 16, gbmc.GBMC_ISING_FM, 1, 12, 2, 30),
                                                         (2, 6, gbmc.GBMC_ISING_FM, 2, 5, 1, 15)])
def test_pt_matches_oracle(ctx, dim, L, model, I, T, theta, steps):
    seed = 41
    betas = np.linspace(0.2, 1.4 if model == gbmc.GBMC_EA_PMJ else 0.6, T)
    lat = gbmc.lattice_init(ctx, dim, L, model=model, n_instances=I, n_replicas=T, seed=seed, instance_base=2)
    pt = gbmc.pt_create(ctx, lat, betas, theta)
    gbmc.pt_step(ctx, pt, steps // 2)
    gbmc.pt_step(ctx, pt, steps - steps // 2)
    rep = np.empty(I * T, dtype=np.uint32)
    acc = np.empty(I * (T - 1), dtype=np.uint32)
    E = np.empty(I * T, dtype=np.int32)
    gbmc.pt_state_out(ctx, pt, rep, acc, E)
    with pytest.raises(gbmc.GbmcError):
        gbmc.metropolis_sweeps(ctx, lat, 0.3, 1)  # owned by the run
    gbmc.pt_free(pt)
    got = spins_out(ctx, lat).reshape(I, T, -1)
    for i in range(I):
        J = oracle.couplings(L, seed, 2 + i) if model == gbmc.GBMC_EA_PMJ else None
        s, r, a, e = oracle.pt_run(dim, L, seed, 2 + i, betas, theta, steps, J=J)
        np.testing.assert_array_equal(got[i], s)
        np.testing.assert_array_equal(rep.reshape(I, T)[i], r)
        np.testing.assert_array_equal(acc.reshape(I, T - 1)[i], a)
        np.testing.assert_array_equal(E.reshape(I, T)[i], e)
    assert acc.sum() > 0
    gbmc.lattice_free(lat)
