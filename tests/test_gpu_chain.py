"""The GPU chain samples the right distribution: at strong coupling the plaquette follows the
character expansion <ReTr U_p / 3> = beta/18 + beta^2/216 - 25 beta^4/466560 + O(u^5) (derived and
pinned against the oracle's plain HMC in tests/test_oracle_hmc.py).  This holds at any volume, so
it checks whole mixed-precision trajectories (graphs, Philox momenta, Metropolis) at 8^4, where a
trajectory-by-trajectory comparison with the oracle would be too slow."""
import math

import numpy as np
import pytest

from gpu_util import dev
from paper_2112_04556_gb300 import inputs

pytestmark = pytest.mark.gpu

BETA = 1.0
U_SERIES = BETA / 18 + BETA ** 2 / 216 - 25 * BETA ** 4 / 466560


@pytest.mark.parametrize("mode", ["plain", "rmhmc_logdet"])
def test_strong_coupling_plaquette(mode):
    """Plain HMC (M = 1) and RMHMC with the log|M| auxiliary field (12 poles, kappa = 0.9), whose links
    are distributed as exp(-S): 10 thermalisation and 60 measured trajectories (tau = 1, 10 steps).
    The error estimate is the naive one; the bound is five of them."""
    import paper_2112_04556_gb300 as rm
    L = (8, 8, 8, 8)
    U = inputs.random_links(L, eps=1.0, seed=3)
    if mode == "plain":
        mass, logdet = {"c": 1.0, "alpha": [], "sigma": [], "kappa": 0.0}, False
    else:
        mass, logdet = rm.mass_fit(12, 0.9), True
    plaq, acc = [], 0
    with rm.Context(L) as ctx:
        Ud = dev(U)
        for n in range(70):
            p = rm.make_params(beta=BETA, mass=mass, tau=1.0, nsteps=10, tol_md=1e-6, tol_h=1e-12, fp_tol=1e-6,
                               fp_maxit=50, maxiter=400, prec=rm.MIXED, seed=29, traj_index=n, metropolis=True,
                               logdet=logdet)
            r = rm.rmhmc_trajectory(ctx, Ud, p)
            if n >= 10:
                plaq.append(r["plaq"])
                acc += r["accepted"]
    plaq = np.array(plaq)
    err = plaq.std() / math.sqrt(len(plaq))
    assert acc >= 20, acc
    assert abs(plaq.mean() - U_SERIES) < 5 * err + 2e-4, (plaq.mean(), U_SERIES, err, acc)
    assert plaq.mean() - BETA / 18 > 0.5 * BETA ** 2 / 216, (plaq.mean(), err)
