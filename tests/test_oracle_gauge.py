"""Pins of the oracle's gauge action and force (Sec. 2: F_G = -dS/dU with the
left-multiplication derivative; Wilson and 1x2-rectangle actions)."""
import math

import numpy as np
import pytest

import helpers as H
from conftest import shift_index
from paper_2112_04556_gb300 import inputs

ASYM = (2, 4, 6, 8)


def abelian_links(L, theta):
    V = int(np.prod(L))
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = np.exp(1j * theta)
    U[..., 1, 1] = np.exp(-1j * theta)
    U[..., 2, 2] = 1.0
    return U


@pytest.mark.parametrize("c1", [0.0, -0.331, -1.4088])
def test_abelian_closed_form(oracle_lib, c1):
    """diag(e^{i th}, e^{-i th}, 1) links: every loop is diag(e^{i Phi}, e^{-i Phi}, 1),
    ReTr = 2 cos Phi + 1, Phi the oriented sum of link angles around the loop."""
    L = ASYM
    rng = np.random.default_rng(1)
    th = rng.uniform(-math.pi, math.pi, (int(np.prod(L)), 4))
    U = abelian_links(L, th)
    beta = 5.7
    c0 = 1 - 8 * c1
    S = 0.0
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            xm = shift_index(L, mu, 1)
            xn = shift_index(L, nu, 1)
            if mu < nu:
                phi = th[:, mu] + th[xm, nu] - th[xn, mu] - th[:, nu]
                S += c0 * np.sum(1 - (2 * np.cos(phi) + 1) / 3)
            x2m = shift_index(L, mu, 2)
            xmn = shift_index(L, nu, 1)[xm]
            phi = th[:, mu] + th[xm, mu] + th[x2m, nu] - th[xmn, mu] - th[xn, mu] - th[:, nu]
            S += c1 * np.sum(1 - (2 * np.cos(phi) + 1) / 3)
    S_or, _ = oracle_lib.action(L, U, beta, c1)
    assert abs(S_or - beta * S) < 1e-10 * abs(beta * S)


@pytest.mark.parametrize("c1", [0.0, -0.331])
def test_force_finite_difference(oracle_lib, c1):
    L = (2, 4, 2, 4)
    U = inputs.random_links(L, eps=0.5, seed=21)
    beta = 6.0
    F = oracle_lib.gauge_force(L, U, beta, c1)
    rng = np.random.default_rng(22)
    h = 1e-5
    for _ in range(16):
        y, mu, a = int(rng.integers(0, np.prod(L))), int(rng.integers(0, 4)), int(rng.integers(0, 8))
        e = np.zeros(8)
        e[a] = h
        vals = []
        for sgn in (+1, -1):
            Up = U.copy()
            Up[y, mu] = H.mm(oracle_lib.exp_i(sgn * e), U[y, mu])
            vals.append(oracle_lib.action(L, Up, beta, c1)[0])
        fd = -(vals[0] - vals[1]) / (2 * h)
        assert abs(fd - F[y, mu, a]) < 2e-8 * max(1.0, abs(fd))


def test_unit_links(oracle_lib):
    L = (4, 4, 4, 4)
    U = inputs.unit_links(L)
    for c1 in (0.0, -0.331):
        F = oracle_lib.gauge_force(L, U, 6.0, c1)
        S, plaq = oracle_lib.action(L, U, 6.0, c1)
        assert np.abs(F).max() == 0.0 and S == 0.0 and abs(plaq - 1.0) < 1e-15


@pytest.mark.parametrize("c1", [0.0, -0.331])
def test_gauge_covariance(oracle_lib, c1):
    """S is invariant and F_mu(x) transforms as g(x) F g(x)^dag."""
    L = ASYM
    V = int(np.prod(L))
    U = inputs.random_links(L, eps=0.7, seed=23)
    g = inputs.random_su3(V, seed=24)
    Up = H.gauge_transform_links(L, U, g)
    S0 = oracle_lib.action(L, U, 6.0, c1)[0]
    S1 = oracle_lib.action(L, Up, 6.0, c1)[0]
    assert abs(S0 - S1) < 1e-11 * abs(S0)
    F0 = oracle_lib.gauge_force(L, U, 6.0, c1)
    F1 = oracle_lib.gauge_force(L, Up, 6.0, c1)
    assert np.abs(F1 - H.gauge_transform_field(F0, g)).max() < 1e-12


@pytest.mark.parametrize("n,e", [((1, 0, 0, 0), (0, 1, 0, 0)), ((1, 1, 0, 0), (1, -1, 0, 0)),
                                 ((0, 2, 1, 0), (1, 0, 0, 1))])
def test_weak_field_linear_response(oracle_lib, n, e):
    """Links exp(i b_mu(x) T^3) with a small transverse plane wave
    b_mu(x) = d e_mu cos(k.x + k_mu/2) (field at the link midpoint, sum_mu sin(k_mu/2) e_mu = 0):
    the Wilson force is F^3_mu = -(beta/6) khat^2 b_mu + O(d^3), khat^2 = sum 4 sin^2(k/2),
    and all other colour components vanish."""
    L = (4, 6, 4, 4)
    k = 2 * np.pi * np.asarray(n) / np.asarray(L)
    sh = np.sin(k / 2)
    e = np.asarray(e, dtype=float)
    e = e - sh * (sh @ e) / (sh @ sh)          # project onto the transverse polarisations
    assert abs(np.sum(sh * e)) < 1e-15 and np.abs(e).max() > 0.1
    d = 1e-5
    from conftest import site_coords
    c = site_coords(L)
    b = d * e[None, :] * np.cos((c @ k)[:, None] + k[None, :] / 2)
    U = abelian_links(L, b / 2)     # exp(i b T^3) = diag(e^{ib/2}, e^{-ib/2}, 1)
    beta = 6.0
    F = oracle_lib.gauge_force(L, U, beta, 0.0)
    khat2 = np.sum(4 * np.sin(k / 2) ** 2)
    expect = -(beta / 6.0) * khat2 * b
    assert np.abs(F[:, :, 2] - expect).max() < 1e-6 * np.abs(expect).max()
    others = np.delete(F, 2, axis=2)
    assert np.abs(others).max() < 1e-12


@pytest.mark.parametrize("L", [ASYM, (3, 4, 3, 6)])
@pytest.mark.parametrize("c1", [0.0, -0.331])
def test_site_sampled_force_equals_full(oracle_lib, L, c1):
    """The site-sampled gauge force (the reference of the full-size parity tests) equals the full force,
    which the pins above fix, at every site, visited in a shuffled order with repeats; the odd extent 3
    makes the rectangles' two-step reach wrap onto the starting site's neighbourhood."""
    V = int(np.prod(L))
    U = inputs.random_links(L, eps=0.8, seed=31)
    full = oracle_lib.gauge_force(L, U, 6.0, c1)
    rng = np.random.default_rng(32)
    sites = np.concatenate([rng.permutation(V), rng.integers(0, V, 13)]).astype(np.int64)
    F = oracle_lib.gauge_force_sites(L, U, 6.0, c1, sites)
    assert F.shape == (len(sites), 4, 8)
    assert np.array_equal(F, full[sites])
