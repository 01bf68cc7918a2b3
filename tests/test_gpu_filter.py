"""GPU parity of the band filter applied as a vector (cheb_filter_apply) and of the momentum-injection
experiment of Sec. 4 built on it (heatbath, filter, one leapfrog step, Wilson-flowed energy), against the
oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import dev, host, rel_l2
from oracle import fit
from paper_2112_04556_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (5, 3, 4, 7)])
def test_filter_apply_parity(L):
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.5, seed=93)
    F = inputs.gaussian_fields(L, 2, seed=94)
    C = oracle.window_coeffs([0.2, 0.45], 40)[0]
    ref = np.stack([oracle.cheb_filter_apply(L, U, F[f], C) for f in range(2)])
    with rm.Context(L) as ctx:
        Y = host(rm.cheb_filter_apply(ctx, dev(U), dev(F), C, prec=rm.FP64))
        assert rel_l2(Y, ref) <= 1e-12
        Ym = host(rm.cheb_filter_apply(ctx, None, dev(F), C, prec=rm.MIXED))
        assert rel_l2(Ym, ref) <= 1e-5


def test_filter_windows_partition_identity():
    """Windows partitioning [0, 1] sum to the identity on any configuration (8^4, degree 60)."""
    import paper_2112_04556_gb300 as rm
    L = (8, 8, 8, 8)
    U = inputs.random_links(L, eps=0.4, seed=95)
    F = inputs.gaussian_fields(L, 1, seed=96)[0]
    C = rm.window_coeffs(np.linspace(0.0, 1.0, 9), 60)
    with rm.Context(L) as ctx:
        Fd = dev(F)
        for prec, tol in ((rm.FP64, 1e-12), (rm.MIXED, 1e-5)):
            total = sum(host(rm.cheb_filter_apply(ctx, dev(U), Fd, C[w], prec=prec)) for w in range(8))
            assert rel_l2(total, F) <= tol


def test_band_injection_matches_oracle():
    """The Sec. 4 experiment at 4^4: filtered heatbath momenta, one leapfrog step of 1e-4, flowed energy."""
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 4)
    U = inputs.random_links(L, eps=0.3, seed=97)
    xi = inputs.gaussian_fields(L, 1, seed=98)[0]
    m = fit.mass_term(12, 0.9)
    window, degree, md_eps, flow_t, flow_eps = (0.0, 0.25), 40, 1e-4, 0.5, 0.05
    C = oracle.window_coeffs(list(window), degree)[0]
    P = oracle.heatbath(L, U, xi, m, tol=1e-14)
    Pw = oracle.cheb_filter_apply(L, U, P, C)
    U1, _, _ = oracle.md_trajectory(L, U, Pw, md_eps, 1, 6.0, 0.0, m, tol=1e-14, fp_tol=1e-14)
    n = int(round(flow_t / flow_eps))
    E0 = oracle.wilson_flow(L, U, flow_eps, n)[1][-1]
    E1 = oracle.wilson_flow(L, U1, flow_eps, n)[1][-1]
    with rm.Context(L) as ctx:
        g1, g0, Pw_d = rm.band_injection(ctx, dev(U), dev(xi), m, window, degree=degree, md_eps=md_eps,
                                         flow_t=flow_t, flow_eps=flow_eps, prec=rm.FP64, tol=1e-13)
    assert rel_l2(host(Pw_d), Pw) <= 1e-11
    assert abs(g0 - E0) <= 1e-12 * E0 and abs(g1 - E1) <= 1e-12 * E0
    assert abs((g1 - g0) - (E1 - E0)) <= 1e-3 * abs(E1 - E0) + 1e-13 * E0
