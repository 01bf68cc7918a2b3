"""GPU parity of gauge_force (Wilson and Iwasaki rectangles) and of the action/plaquette."""
import numpy as np
import pytest

import oracle
from gpu_util import dev, host, rel_l2, torch_cuda
from paper_2112_04556_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (5, 3, 4, 7), (3, 4, 3, 6)])
@pytest.mark.parametrize("c1", [0.0, -0.331])
def test_gauge_force_parity(L, c1):
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.6, seed=11)
    ref = oracle.gauge_force(L, U, 6.0, c1)
    S_ref, pl_ref = oracle.action(L, U, 6.0, c1)
    with rm.Context(L) as ctx:
        Ud = dev(U)
        F, S, pl = rm.gauge_force(ctx, Ud, 6.0, c1, prec=rm.FP64)
        assert rel_l2(host(F), ref) <= 1e-12
        assert abs(S - S_ref) <= 1e-12 * abs(S_ref) and abs(pl - pl_ref) <= 1e-13
        F32, S32, _ = rm.gauge_force(ctx, None, 6.0, c1, prec=rm.FP32)
        assert rel_l2(host(F32), ref) <= 1e-5
        assert abs(S32 - S_ref) <= 1e-12 * abs(S_ref)     # the action is always float64


def test_gauge_unit_links():
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 6)
    with rm.Context(L) as ctx:
        F, S, pl = rm.gauge_force(ctx, dev(inputs.unit_links(L)), 6.0, -0.331)
        assert np.abs(host(F)).max() == 0.0 and S == 0.0 and abs(pl - 1.0) < 1e-15


@pytest.mark.parametrize("L,c1", [((32, 32, 32, 32), 0.0), ((16, 16, 16, 16), -0.331)])
def test_gauge_force_full_size_sampled(L, c1):
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.3, seed=0)
    V = int(np.prod(L))
    rng = np.random.default_rng(3)
    sites = np.unique(np.concatenate([rng.integers(0, V, 600), [0, V - 1]]))
    ref = oracle.gauge_force_sites(L, U, 6.0, c1, sites)
    with rm.Context(L) as ctx:
        F, S, pl = rm.gauge_force(ctx, dev(U), 6.0, c1, prec=rm.FP64)
        assert rel_l2(host(F)[sites], ref) <= 1e-12
        F32, _, _ = rm.gauge_force(ctx, None, 6.0, c1, prec=rm.FP32)
        assert rel_l2(host(F32)[sites], ref) <= 1e-5
    if L == (16, 16, 16, 16):
        S_ref, pl_ref = oracle.action(L, U, 6.0, c1)
        assert abs(S - S_ref) <= 1e-12 * abs(S_ref) and abs(pl - pl_ref) <= 1e-13
