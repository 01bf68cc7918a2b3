"""GPU parity of the batched Chebyshev moments and per-mode power spectra (Sec. 2, Eq. 4)."""
import numpy as np
import pytest

import oracle
from conftest import config2_links
from gpu_util import dev, host, rel_l2, torch_cuda
from paper_2112_04556_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_config1_spectrum_parity():
    """4^4, seed-0 links, Wilson beta = 6 force, degree 64, 16 equal windows, 16 noise fields."""
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    L = (4, 4, 4, 4)
    U = inputs.random_links(L, eps=0.3, seed=0)
    F = oracle.gauge_force(L, U, 6.0)
    noise = inputs.gaussian_fields(L, 16, seed=7)
    edges = inputs.equal_windows(16)
    s_ref, n_ref, t_ref, m_ref = oracle.power_spectrum(L, U, [F], list(noise), 64, edges)
    with rm.Context(L) as ctx:
        Fd, Nd = dev(F), dev(noise)
        spec, num, tr, mom = rm.cheb_filter_spectrum(ctx, dev(U), Fd, Nd, 64, edges, prec=rm.FP64)
        assert np.abs(mom - m_ref).max() <= 1e-12 * m_ref[:, :1].max()
        assert np.abs(spec - s_ref).max() <= 1e-10 * np.abs(s_ref).max()
        assert rel_l2(tr, t_ref) <= 1e-12
        spec32, num32, tr32, mom32 = rm.cheb_filter_spectrum(ctx, None, Fd, Nd, 64, edges, prec=rm.MIXED)
        assert np.all(np.abs(num32 - n_ref) <= 1e-4 * np.abs(n_ref) + 1e-7 * np.abs(n_ref).sum())
        assert np.all(np.abs(tr32 - t_ref) <= 1e-4 * np.abs(t_ref) + 1e-7 * np.abs(t_ref).sum())
        # no damping, odd degree, and a ragged window set
        e2 = np.array([0.0, 0.1, 0.45, 0.8, 1.0])
        s2_ref = oracle.power_spectrum(L, U, [F], list(noise[:3]), 33, e2, kernel="none")[0]
        s2 = rm.cheb_filter_spectrum(ctx, None, Fd, Nd[:3].contiguous(), 33, e2, kernel=rm.KERNEL_NONE)[0]
        assert np.abs(s2 - s2_ref).max() <= 1e-10 * np.abs(s2_ref).max()


def test_generated_noise_matches_oracle_philox():
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 6)
    U = inputs.random_links(L, eps=0.3, seed=1)
    F = inputs.gaussian_fields(L, 1, seed=2)[0]
    noise = [oracle.gauss_field(L, 99, f, 2) for f in range(4)]
    edges = inputs.equal_windows(8)
    s_ref = oracle.power_spectrum(L, U, [F], noise, 40, edges)[0]
    with rm.Context(L) as ctx:
        s = rm.cheb_filter_spectrum(ctx, dev(U), dev(F), None, 40, edges, nnoise=4, seed=99)[0]
    assert np.abs(s - s_ref).max() <= 1e-10 * np.abs(s_ref).max()


def test_config2_spectrum():
    """16^4 oracle-HMC links: degree 200 over 64 windows, Wilson and Iwasaki forces and 16 noise fields in
    one batched recurrence; float64 moments match the oracle, the float32 spectrum matches float64 to 1e-4."""
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    L = (16, 16, 16, 16)
    U = config2_links()
    Fw = oracle.gauge_force(L, U, 6.0, 0.0)
    Fi = oracle.gauge_force(L, U, 6.0, -0.331)
    noise = inputs.gaussian_fields(L, 16, seed=8)
    edges = inputs.equal_windows(64)
    m_ref = oracle.cheb_moments(L, U, Fw, 200)
    with rm.Context(L) as ctx:
        Fd = dev(np.stack([Fw, Fi]))
        Nd = dev(noise)
        spec, num, tr, mom = rm.cheb_filter_spectrum(ctx, dev(U), Fd, Nd, 200, edges, prec=rm.FP64)
        assert np.abs(mom[0] - m_ref).max() <= 1e-12 * m_ref[0]
        spec32, num32, tr32, _ = rm.cheb_filter_spectrum(ctx, None, Fd, Nd, 200, edges, prec=rm.MIXED)
    assert np.all(spec > 0)
    # float32 recurrence: per window 1e-4 of the window's value, with an absolute floor of 1e-7 of the
    # total power (the edge windows carry ~1e-7 of it; float32 moments resolve ~1e-9 of mu_0)
    for a32, a64 in ((num32, num), (tr32[None, :], tr[None, :])):
        floor = 1e-7 * np.abs(a64).sum(axis=1, keepdims=True)
        assert np.all(np.abs(a32 - a64) <= 1e-4 * np.abs(a64) + floor), np.abs(a32 / a64 - 1).max()
    bulk = (num / num.sum(axis=1, keepdims=True)) > 1e-3
    assert np.all(np.abs(spec32 - spec)[bulk] <= 1e-4 * spec[bulk])
