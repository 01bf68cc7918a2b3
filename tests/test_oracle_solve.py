"""Pins of the oracle's rational mass term and its solves (Sec. 3, Eq. 6; Sec. 1, Eq. 2)."""
import math

import numpy as np
import pytest

import helpers as H
from conftest import site_coords
from oracle import fit
from paper_2112_04556_gb300 import inputs


@pytest.mark.parametrize("n", [2, 3])
def test_zolotarev_equioscillates(n):
    """Best approximation of type (n,n): the relative error alternates in sign at 2n+2
    points with equal magnitude (Chebyshev alternation theorem)."""
    d, a, s, err = fit.zolotarev_inv_sqrt(n, 0.1, 1.0)
    x = np.geomspace(0.1, 1.0, 400001)
    r = d + np.sum(a[None, :] / (x[:, None] + s[None, :]), axis=1)
    e = r * np.sqrt(x) - 1.0
    # local extrema (plus both end points)
    idx = [0] + [i for i in range(1, len(e) - 1) if (e[i] - e[i - 1]) * (e[i + 1] - e[i]) < 0] + [len(e) - 1]
    ext = e[idx]
    assert len(ext) == 2 * n + 2
    assert np.all(np.sign(ext[1:]) != np.sign(ext[:-1]))
    assert np.abs(np.abs(ext) - np.abs(ext).max()).max() < 1e-6 * np.abs(ext).max()


def test_twelve_pole_mass_term():
    """kappa = 0.9, 12 poles: R(lam) m(lam)^{1/2} = 1 to rounding on a 1e5-point grid of [0,1];
    poles real and negative (sigma_j > (1-kappa)/kappa), residues positive."""
    m = fit.mass_term(12, 0.9)
    lam = np.linspace(0.0, 1.0, 100001)
    err = np.abs(fit.evaluate(m, lam) * np.sqrt(0.1 + 0.9 * lam) - 1.0).max()
    assert err < 1e-14
    assert np.all(m["sigma"] > 0.1 / 0.9) and np.all(m["alpha"] > 0) and m["c"] > 0
    assert len(m["sigma"]) == 12 and len(np.unique(m["sigma"])) == 12


def test_cg_matches_dense_solve(oracle_lib):
    L = (2, 2, 2, 4)
    U = inputs.random_links(L, eps=0.8, seed=31)
    b = inputs.gaussian_fields(L, 1, seed=32)[0]
    b[:, 1:] = 0.0
    sigma = 0.2
    M = H.dense_operator(lambda X: oracle_lib.lap(L, U, X), L) + sigma * np.eye(8 * int(np.prod(L)))
    x_dense = np.linalg.solve(M, b[:, 0, :].ravel())
    x, it, res = oracle_lib.cg(lambda v: oracle_lib.lap(L, U, v) + sigma * v, b, tol=1e-13)
    assert res <= 1e-13
    assert np.abs(x[:, 0, :].ravel() - x_dense).max() < 1e-12 * np.abs(x_dense).max()
    assert np.abs(x[:, 1:]).max() == 0.0


def test_rational_apply_plane_wave(oracle_lib):
    """U = 1: R(A) (T^a cos k.x) = R(lambda_k) (T^a cos k.x)."""
    L = (4, 4, 4, 4)
    U = inputs.unit_links(L)
    m = fit.mass_term(12, 0.9)
    for n in [(0, 0, 0, 0), (1, 0, 2, 1), (2, 2, 2, 2), (1, 3, 0, 0)]:
        X = H.plane_wave(L, n, 2, 5, phase=0.3)
        Y, _ = oracle_lib.rational_apply(L, U, X, m)
        lam = H.free_eigenvalue(L, n)
        assert np.abs(Y - fit.evaluate(m, lam) * X).max() < 1e-12
        assert abs(fit.evaluate(m, lam) - (0.1 + 0.9 * lam) ** -0.5) < 1e-14


@pytest.mark.parametrize("n,e", [((1, 0, 0, 0), (0, 1, 0, 0)), ((1, 1, 0, 0), (1, -1, 0, 0)),
                                 ((0, 2, 1, 1), (1, 0, 1, 1))])
def test_u1_frequency(oracle_lib, n, e):
    """Sec. 1, Eq. (2): a small transverse abelian wave b_mu(x) T^3 moves as
    d^2 b/dtau^2 = M^{-1} F_G = -omega^2(k) b with
    omega^2(k) = (beta/6) khat^2 / [(1-kappa) + kappa khat^2/16],
    the paper's k^2/(1 - kappa + kappa k^2) in the normalisation of -Delta/16."""
    L = (4, 6, 4, 4)
    k = 2 * np.pi * np.asarray(n) / np.asarray(L)
    sh = np.sin(k / 2)
    e = np.asarray(e, float)
    e = e - sh * (sh @ e) / (sh @ sh)
    d = 1e-5
    b = d * e[None, :] * np.cos((site_coords(L) @ k)[:, None] + k[None, :] / 2)
    V = int(np.prod(L))
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = np.exp(0.5j * b)
    U[..., 1, 1] = np.exp(-0.5j * b)
    U[..., 2, 2] = 1.0
    beta, kappa = 6.0, 0.9
    m = fit.mass_term(12, kappa)
    F = oracle_lib.gauge_force(L, U, beta, 0.0)
    Y, _ = oracle_lib.rational_apply(L, U, F, m)
    Minv_F, _ = oracle_lib.rational_apply(L, U, Y, m)
    khat2 = np.sum(4 * sh ** 2)
    omega2 = (beta / 6.0) * khat2 / ((1 - kappa) + kappa * khat2 / 16.0)
    acc = Minv_F[:, :, 2]
    assert np.abs(acc + omega2 * b).max() < 1e-5 * omega2 * np.abs(b).max()
    # kappa -> 1: every mode moves at the same frequency (beta/6)*16
    m1 = fit.mass_term(12, 0.999)
    Y, _ = oracle_lib.rational_apply(L, U, F, m1)
    acc1, _ = oracle_lib.rational_apply(L, U, Y, m1)
    w1 = (beta / 6.0) * khat2 / (0.001 + 0.999 * khat2 / 16.0)
    assert abs(w1 - 16.0) < 0.05 * 16.0
    assert np.abs(acc1[:, :, 2] + w1 * b).max() < 1e-5 * w1 * np.abs(b).max()


def test_spectrum_fit_recovers_exact_rational():
    """A spectrum generated from R* = c* + sum alpha*_j/(lam + sigma_j) on the fit's own pole grid
    (alpha* >= 0) is fitted exactly: M = R*^{-2} up to the normalisation M = 1 at the largest power."""
    sigma = np.geomspace(1e-3, 10.0, 8)
    rng = np.random.default_rng(11)
    alpha = rng.uniform(0.0, 0.05, 8) * (rng.uniform(size=8) > 0.3)
    Rstar = {"c": 0.3, "alpha": alpha, "sigma": sigma}
    lam = (np.arange(64) + 0.5) / 64
    spec = 5.0 * fit.evaluate(Rstar, lam) ** -2
    m = fit.spectrum_mass_term(lam, spec, 8)
    g = (spec / spec.max()) ** -0.5
    assert np.abs(fit.evaluate(m, lam) / g - 1).max() < 1e-10
    assert m["err"] < 1e-10 and m["kappa"] == 0.0 and m["c"] >= 0 and np.all(m["alpha"] >= 0)


def test_spectrum_fit_linear_power():
    """The near-linear power of Sec. 2 (s = 0.1 + lam): 12 poles fit M = s / max s to better than 1e-3,
    and the fitted M increases with lam."""
    lam = (np.arange(64) + 0.5) / 64
    m = fit.spectrum_mass_term(lam, 0.1 + lam, 12)
    assert m["err"] < 1e-3
    M = fit.evaluate(m, np.linspace(0, 1, 201)) ** -2
    assert np.all(np.diff(M) > 0)


@pytest.mark.parametrize("c", [0.7, 0.0])
def test_inverse_partial_fraction(c):
    """(p0 + p1 lam + sum beta_j/(lam + zeta_j)) R(lam) = 1 on [0, 1] and beyond, with and without c."""
    mass = {"c": c, "alpha": np.array([0.02, 0.3, 0.0, 1.5, 0.7]), "sigma": np.array([0.01, 0.2, 0.5, 1.3, 4.0])}
    inv = fit.inverse_partial_fraction(mass)
    lam = np.linspace(0.0, 3.0, 301)
    r = inv["p0"] + inv["p1"] * lam + sum(b / (lam + z) for b, z in zip(inv["beta"], inv["zeta"]))
    assert np.abs(r * fit.evaluate(mass, lam) - 1).max() < 1e-11
    assert np.all(inv["zeta"] > 0)


def test_general_heatbath_plane_wave(oracle_lib):
    """U = 1: a plane wave of eigenvalue lam_k goes to X / R(lam_k) under the heatbath of a general
    rational mass (kappa = 0)."""
    L = (4, 4, 4, 4)
    U = inputs.unit_links(L)
    X = H.plane_wave(L, (1, 0, 2, 1), 3, 4, 0.1)
    lam = H.free_eigenvalue(L, (1, 0, 2, 1))
    mass = {"c": 0.4, "alpha": np.array([0.05, 0.2, 0.6]), "sigma": np.array([0.02, 0.3, 2.0]), "kappa": 0.0}
    P = oracle_lib.heatbath(L, U, X, mass, tol=1e-13)
    assert np.abs(P - X / fit.evaluate(mass, lam)).max() < 1e-11


def test_general_heatbath_kinetic_identity(oracle_lib):
    """T(P) = 1/2 |R P|^2 = 1/2 |xi|^2 for P = R^{-1} xi on random links."""
    L = (2, 2, 2, 4)
    U = inputs.random_links(L, eps=0.6, seed=12)
    xi = inputs.gaussian_fields(L, 1, seed=13)[0]
    mass = {"c": 0.4, "alpha": np.array([0.05, 0.2, 0.6]), "sigma": np.array([0.02, 0.3, 2.0]), "kappa": 0.0}
    P = oracle_lib.heatbath(L, U, xi, mass, tol=1e-13)
    T, _, _ = oracle_lib.kinetic(L, U, P, mass, tol=1e-14)
    assert abs(T - 0.5 * np.sum(xi * xi)) < 1e-11 * T


@pytest.mark.parametrize("symplectic", [False, True])
def test_linearised_md_follows_the_discrete_oscillator(oracle_lib, symplectic):
    """A weak transverse abelian wave b_mu(x) T^3 (amplitude 1e-6, P = 0) under the implicit leapfrog:
    to first order in b the step is the plain leapfrog of the oscillator d^2 b/dtau^2 = -omega^2 b with
    omega^2 = (beta/6) khat^2 R(lambda_k)^2 (M^{-1} = R^2 exactly, lambda_k = khat^2/16), whose
    discrete solution from rest is b_n = b_0 cos(n theta), cos theta = 1 - (omega eps)^2 / 2.  Both
    forms of the step (the dexp factors act at O(b^2))."""
    L = (4, 4, 4, 4)
    k = 2 * np.pi * np.array([1, 0, 0, 0]) / np.asarray(L)
    sh = np.sin(k / 2)
    e = np.array([0.0, 1.0, 0.0, 0.0])
    b0 = 1e-6 * e[None, :] * np.cos((site_coords(L) @ k)[:, None] + k[None, :] / 2)
    V = int(np.prod(L))
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = np.exp(0.5j * b0)
    U[..., 1, 1] = np.exp(-0.5j * b0)
    U[..., 2, 2] = 1.0
    P = np.zeros((V, 4, 8))
    beta = 6.0
    m = fit.mass_term(4, 0.9)
    khat2 = np.sum(4 * sh ** 2)
    omega = math.sqrt(beta / 6.0 * khat2) * float(fit.evaluate(m, khat2 / 16.0))
    eps, n = 0.05, 12
    theta = math.acos(1.0 - 0.5 * (omega * eps) ** 2)
    U1, _, _ = oracle_lib.md_trajectory(L, U, P, eps * n, n, beta, 0.0, m, tol=1e-13, fp_tol=1e-16,
                                        symplectic=symplectic)
    b1 = np.angle(U1[..., 0, 0] / U1[..., 1, 1])
    expect = b0 * math.cos(n * theta)
    assert abs(math.cos(n * theta) - math.cos(n * eps * omega)) > 1e-3    # the discrete phase is resolved
    assert np.abs(b1 - expect).max() < 1e-8 * np.abs(b0).max()
