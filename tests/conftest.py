import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def site_coords(L):
    """[V,4] integer coordinates, x fastest."""
    V = int(np.prod(L))
    s = np.arange(V)
    out = np.empty((V, 4), dtype=np.int64)
    for d in range(4):
        out[:, d] = s % L[d]
        s = s // L[d]
    return out


def shift_index(L, mu, n=1):
    """index map s -> s + n*mu (periodic)."""
    c = site_coords(L)
    c[:, mu] = (c[:, mu] + n) % L[mu]
    return c[:, 0] + L[0] * (c[:, 1] + L[1] * (c[:, 2] + L[2] * c[:, 3]))


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


_CONFIG2 = {}


def config2_links():
    """16^4 links from 20 plain-HMC trajectories of the oracle (beta = 6.0, tau = 1, 20 steps, Philox
    momenta with seed 0, every trajectory accepted: thermalisation) started from the seed-0 random links
    exp(i 0.3 sum r_a T_a)."""
    if "U" not in _CONFIG2:
        import oracle
        from paper_2112_04556_gb300 import inputs
        L = (16, 16, 16, 16)
        U = inputs.random_links(L, eps=0.3, seed=0)
        U, acc = oracle.plain_hmc(L, U, 20, 6.0, seed=0, tau=1.0, nsteps=20, metropolis=False)
        _CONFIG2["U"] = U
        _CONFIG2["acc"] = acc
    return _CONFIG2["U"]
