"""GPU parity of the Wilson gradient flow and the flowed energy against the oracle (float64 and mixed
precision), and its properties at a size the oracle does not reach."""
import numpy as np
import pytest

import oracle
from gpu_util import dev, host
from paper_2112_04556_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (5, 3, 4, 7)])
def test_flow_parity(L):
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.4, seed=91)
    eps, n = 0.05, 8
    U_ref, E_ref = oracle.wilson_flow(L, U, eps, n)
    with rm.Context(L) as ctx:
        Ud = dev(U)
        E = rm.wilson_flow(ctx, Ud, eps, n, prec=rm.FP64)
        assert np.abs(host(Ud) - U_ref).max() <= 1e-12
        assert np.abs(E - E_ref).max() <= 1e-12 * E_ref[0]
        Um = dev(U)
        Em = rm.wilson_flow(ctx, Um, eps, n, prec=rm.MIXED)
        assert np.abs(host(Um) - U_ref).max() <= 1e-5
        assert np.abs(Em - E_ref).max() <= 1e-6 * E_ref[0]


def test_flow_zero_steps_and_errors():
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 4)
    U = inputs.random_links(L, eps=0.4, seed=92)
    with rm.Context(L) as ctx:
        Ud = dev(U)
        E = rm.wilson_flow(ctx, Ud, 0.05, 0)
        assert E.shape == (1,) and abs(E[0] - oracle.flow_energy(L, U)) <= 1e-12 * E[0]
        assert np.abs(host(Ud) - U).max() == 0.0
        with pytest.raises(rm.RmhmcError):
            rm.wilson_flow(ctx, Ud, float("nan"), 2)
        with pytest.raises(rm.RmhmcError):
            rm.wilson_flow(ctx, Ud, 0.05, -1)


def test_flow_16_4_to_t8():
    """16^4 oracle-HMC links (beta = 6.0) flowed to t = 8 (the paper's flow time for 16^4) in 800 steps:
    E decreases monotonically, t^2 E(t) is finite and positive, and float64 and mixed agree."""
    import paper_2112_04556_gb300 as rm
    from conftest import config2_links
    L = (16, 16, 16, 16)
    U = config2_links()
    eps, n = 0.01, 800
    with rm.Context(L) as ctx:
        E = rm.wilson_flow(ctx, dev(U), eps, n, prec=rm.FP64)
        Em = rm.wilson_flow(ctx, dev(U), eps, n, prec=rm.MIXED)
    assert np.all(np.diff(E) < 0)
    t = np.arange(n + 1) * eps
    t2E = t[-1] ** 2 * E[-1]
    assert 0.0 < t2E < 1e3
    assert np.abs(Em - E).max() <= 1e-5 * E[0]
    # the first steps against the oracle
    _, E_ref = oracle.wilson_flow(L, U, eps, 3)
    assert np.abs(E[:4] - E_ref).max() <= 1e-12 * E_ref[0]
