"""Pins of the oracle's Chebyshev band-pass filters and per-mode power spectrum
(Sec. 2, Eq. 4; B(lambda) = sum_i c_i T_i[-Delta_G/16])."""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from scipy.integrate import quad

import helpers as H
from conftest import site_coords
from paper_2112_04556_gb300 import inputs


def test_moments_match_dense_spectral_sum(oracle_lib):
    """mu_k(F) = sum_c sum_i <v_i, F_c>^2 T_k(2 lambda_i - 1) from numpy's eigh."""
    L = (2, 2, 2, 4)
    U = inputs.random_links(L, eps=0.8, seed=41)
    F = inputs.gaussian_fields(L, 1, seed=42)[0]
    M = H.dense_operator(lambda X: oracle_lib.lap(L, U, X), L)
    lam, vec = np.linalg.eigh(M)
    N = 40
    mu = oracle_lib.cheb_moments(L, U, F, N)
    ref = np.zeros(N + 1)
    for c in range(4):
        w = (vec.T @ F[:, c, :].ravel()) ** 2
        for k in range(N + 1):
            ref[k] += np.sum(w * npcheb.chebval(2 * lam - 1, np.eye(N + 1)[k]))
    assert np.abs(mu - ref).max() < 1e-11 * mu[0]


def test_moments_free_field_fft(oracle_lib):
    """U = 1: mu_k(F) = (1/V) sum_k |F~(k)|^2 T_k(2 lambda_k - 1) per coefficient."""
    L = (6, 4, 6, 4)
    U = inputs.unit_links(L)
    F = inputs.gaussian_fields(L, 1, seed=43)[0]
    N = 30
    mu = oracle_lib.cheb_moments(L, U, F, N)
    V = int(np.prod(L))
    shape = (L[3], L[2], L[1], L[0])
    power = np.zeros(shape)
    for c in range(4):
        for a in range(8):
            power += np.abs(np.fft.fftn(F[:, c, a].reshape(shape))) ** 2
    power /= V
    ks = [2 * np.pi * np.fft.fftfreq(l) for l in (L[3], L[2], L[1], L[0])]
    KT, KZ, KY, KX = np.meshgrid(*ks, indexing="ij")
    lam = (np.sin(KX / 2) ** 2 + np.sin(KY / 2) ** 2 + np.sin(KZ / 2) ** 2 + np.sin(KT / 2) ** 2) / 4
    ref = np.array([np.sum(power * np.cos(k * np.arccos(np.clip(2 * lam - 1, -1, 1)))) for k in range(N + 1)])
    assert np.abs(mu - ref).max() < 1e-11 * mu[0]


def test_window_coefficients_quadrature(oracle_lib):
    """c_k = (2 - delta_k0)/pi * int_0^pi 1_w(cos th) cos(k th) d th, by adaptive quadrature."""
    edges = np.array([0.0, 0.13, 0.5, 0.77, 1.0])
    N = 25
    C = oracle_lib.window_coeffs(edges, N, kernel="none")
    for w in range(4):
        xa, xb = 2 * edges[w] - 1, 2 * edges[w + 1] - 1
        for k in range(N + 1):
            val, _ = quad(lambda th: math.cos(k * th) if xa <= math.cos(th) <= xb else 0.0, 0, math.pi,
                          points=[math.acos(xa), math.acos(xb)], limit=200)
            ref = (1.0 if k == 0 else 2.0) / math.pi * val
            assert abs(C[w, k] - ref) < 1e-10


def test_windows_partition_unity_and_jackson_positive(oracle_lib):
    edges = inputs.equal_windows(16)
    N = 64
    C = oracle_lib.window_coeffs(edges, N, kernel="none")
    s = C.sum(axis=0)
    assert abs(s[0] - 1.0) < 1e-14 and np.abs(s[1:]).max() < 1e-13
    CJ = oracle_lib.window_coeffs(edges, N, kernel="jackson")
    x = np.linspace(-1, 1, 20001)
    vals = np.array([npcheb.chebval(x, CJ[w]) for w in range(16)])
    assert vals.min() > -1e-12                      # Jackson-damped filters are non-negative
    assert np.abs(vals.sum(axis=0) - 1.0).max() < 1e-12


def test_free_field_window_projector(oracle_lib):
    """U = 1, windows whose edges avoid every lambda_k: the degree-200 Jackson filter
    reproduces the ideal projector sum_{lambda_k in w} |F~(k)|^2 to < 1%."""
    L = (6, 6, 6, 6)
    U = inputs.unit_links(L)
    F = inputs.gaussian_fields(L, 1, seed=44)[0]
    edges = np.concatenate([[0.0], np.arange(1, 16) / 16.0 + 1.0 / 32.0, [1.0]])
    N = 200
    spec, num, tr, mom = oracle_lib.power_spectrum(L, U, [F], [F], N, edges)
    V = int(np.prod(L))
    shape = (6, 6, 6, 6)
    power = np.zeros(shape)
    for c in range(4):
        for a in range(8):
            power += np.abs(np.fft.fftn(F[:, c, a].reshape(shape))) ** 2
    power /= V
    k1 = 2 * np.pi * np.fft.fftfreq(6)
    K = np.meshgrid(k1, k1, k1, k1, indexing="ij")
    lam = sum(np.sin(kk / 2) ** 2 for kk in K) / 4
    for w in range(16):
        sel = (lam >= edges[w]) & (lam <= edges[w + 1])
        ideal = power[sel].sum()
        if ideal > 0:
            assert abs(num[0, w] - ideal) < 1e-2 * ideal


def test_white_noise_spectrum_is_flat(oracle_lib):
    """A white-noise 'force' has spectrum 1 per mode (the normalisation of Eq. 4)."""
    L = (6, 6, 6, 6)
    U = inputs.random_links(L, eps=0.3, seed=45)
    fields = inputs.gaussian_fields(L, 9, seed=46)
    spec, num, tr, _ = oracle_lib.power_spectrum(L, U, [fields[0]], list(fields[1:]), 48, inputs.equal_windows(8))
    assert np.all(tr > 0)
    assert abs(spec.mean() - 1.0) < 0.05
    assert np.abs(spec - 1.0).max() < 0.3


def test_spectrum_gauge_invariant(oracle_lib):
    L = (4, 4, 4, 4)
    V = int(np.prod(L))
    U = inputs.random_links(L, eps=0.5, seed=47)
    F = oracle_lib.gauge_force(L, U, 6.0)
    eta = inputs.gaussian_fields(L, 2, seed=48)
    g = inputs.random_su3(V, seed=49)
    Up = H.gauge_transform_links(L, U, g)
    Fp = H.gauge_transform_field(F, g)
    etap = [H.gauge_transform_field(e, g) for e in eta]
    s0 = oracle_lib.power_spectrum(L, U, [F], list(eta), 32, inputs.equal_windows(8))[0]
    s1 = oracle_lib.power_spectrum(L, Up, [Fp], etap, 32, inputs.equal_windows(8))[0]
    assert np.abs(s0 - s1).max() < 1e-10 * np.abs(s0).max()


def test_filter_apply_dense(oracle_lib):
    """B F = sum_i v_i g(lambda_i) <v_i, F> with g(lambda) = sum_k c_k T_k(2 lambda - 1), from numpy's eigh
    of the dense operator, per component."""
    L = (2, 2, 2, 4)
    U = inputs.random_links(L, eps=0.8, seed=45)
    F = inputs.gaussian_fields(L, 1, seed=46)[0]
    M = H.dense_operator(lambda X: oracle_lib.lap(L, U, X), L)
    lam, vec = np.linalg.eigh(M)
    coef = oracle_lib.window_coeffs([0.1, 0.35], 30)[0]
    Y = oracle_lib.cheb_filter_apply(L, U, F, coef)
    g = npcheb.chebval(2 * lam - 1, coef)
    for c in range(4):
        ref = vec @ (g * (vec.T @ F[:, c, :].ravel()))
        assert np.abs(Y[:, c, :].ravel() - ref).max() < 1e-12 * np.abs(ref).max()


def test_filter_apply_free_plane_wave_and_partition(oracle_lib):
    """U = 1: a plane wave is an eigenvector, B X = g(lambda_k) X; and windows that partition [0, 1]
    sum to the identity (their coefficients add up to delta_k0)."""
    L = (4, 4, 6, 4)
    U = inputs.unit_links(L)
    X = H.plane_wave(L, (1, 2, 3, 0), 2, 5, 0.3)
    lam = H.free_eigenvalue(L, (1, 2, 3, 0))
    N = 60
    edges = np.linspace(0.0, 1.0, 9)
    C = oracle_lib.window_coeffs(edges, N)
    total = np.zeros_like(X)
    for w in range(8):
        Y = oracle_lib.cheb_filter_apply(L, U, X, C[w])
        assert np.abs(Y - npcheb.chebval(2 * lam - 1, C[w]) * X).max() < 1e-12
        total += Y
    assert np.abs(total - X).max() < 1e-12


def test_heatbath_momenta_spectrum_is_the_mass(oracle_lib):
    """The per-mode spectrum of heatbath momenta P = M^{1/2} xi is M itself: on random links, with the
    Zolotarev mass m(lam) = (1-kappa) + kappa lam, the window spectra of P follow m at the window centres
    (Eq. 4 normalisation; Hutchinson noise and the momenta from independent Gaussians)."""
    from oracle import fit
    L = (4, 4, 4, 4)
    U = inputs.random_links(L, eps=0.3, seed=60)
    m = fit.mass_term(12, 0.9)
    xis = inputs.gaussian_fields(L, 4, seed=61)
    P = [oracle_lib.heatbath(L, U, xi, m, tol=1e-12) for xi in xis]
    noise = list(inputs.gaussian_fields(L, 8, seed=62))
    edges = np.linspace(0.0, 1.0, 9)
    spec, num, tr, _ = oracle_lib.power_spectrum(L, U, P, noise, 64, edges)
    centres = 0.5 * (edges[:-1] + edges[1:])
    mean = spec.mean(axis=0)
    # windows that hold a good share of the modes (the spectrum of A is concentrated in the middle)
    ok = tr > 0.05 * tr.sum()
    target = (1 - 0.9) + 0.9 * centres
    assert np.all(np.abs(mean[ok] / target[ok] - 1) < 0.08), (mean, target, tr)
