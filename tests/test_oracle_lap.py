"""Pins of the oracle's normalised covariant Laplacian A = -Delta_G/16 (Sec. 2, Eq. 3)
against what the mathematics fixes: free plane-wave eigenvalues, the dense free
spectrum, gauge covariance, symmetry and bounds, the bipartite spectral mirror, and
finite differences for the link derivative."""
import numpy as np
import pytest

import helpers as H
from paper_2112_04556_gb300 import inputs

ASYM = (2, 4, 6, 8)


@pytest.mark.parametrize("L", [(4, 4, 4, 4), ASYM])
def test_free_plane_waves(oracle_lib, L):
    """U = 1: A (T^a cos k.x) = lambda_k (T^a cos k.x), lambda_k = sum_nu sin^2(k_nu/2)/4
    (= Sum 4 sin^2(k_nu/2), the free -Delta eigenvalue, divided by 16)."""
    U = inputs.unit_links(L)
    rng = np.random.default_rng(5)
    for trial in range(12):
        n = [int(rng.integers(0, l)) for l in L]
        comp, a = int(rng.integers(0, 4)), int(rng.integers(0, 8))
        X = H.plane_wave(L, n, comp, a, phase=float(rng.uniform(0, 6.3)))
        Y = oracle_lib.lap(L, U, X)
        lam = H.free_eigenvalue(L, n)
        assert np.abs(Y - lam * X).max() < 1e-14


def test_free_dense_spectrum(oracle_lib):
    """On U = 1 the dense spectrum of A on one component is {lambda_k}, each 8-fold."""
    L = (2, 2, 4, 4)
    U = inputs.unit_links(L)
    M = H.dense_operator(lambda X: oracle_lib.lap(L, U, X), L)
    ev = np.sort(np.linalg.eigvalsh(M))
    grid = np.array(np.meshgrid(*[np.arange(l) for l in L], indexing="ij")).reshape(4, -1).T
    lam = np.sort(np.repeat([H.free_eigenvalue(L, n) for n in grid], 8))
    assert np.abs(ev - lam).max() < 1e-13


@pytest.mark.parametrize("L", [(4, 4, 4, 4), ASYM])
def test_gauge_covariance(oracle_lib, L):
    """U'_nu(x) = g(x) U_nu(x) g(x+nu)^dag, X' = g X g^dag  =>  A' X' = g (A X) g^dag."""
    V = int(np.prod(L))
    U = inputs.random_links(L, eps=0.6, seed=3)
    X = inputs.gaussian_fields(L, 1, seed=4)[0]
    g = inputs.random_su3(V, seed=6)
    Up = H.gauge_transform_links(L, U, g)
    Xp = H.gauge_transform_field(X, g)
    lhs = oracle_lib.lap(L, Up, Xp)
    rhs = H.gauge_transform_field(oracle_lib.lap(L, U, X), g)
    assert np.abs(lhs - rhs).max() < 1e-13


def test_pure_gauge_has_free_spectrum(oracle_lib):
    L = (2, 2, 2, 4)
    V = int(np.prod(L))
    g = inputs.random_su3(V, seed=8)
    U = H.pure_gauge_links(L, g)
    M = H.dense_operator(lambda X: oracle_lib.lap(L, U, X), L)
    ev = np.sort(np.linalg.eigvalsh(0.5 * (M + M.T)))
    grid = np.array(np.meshgrid(*[np.arange(l) for l in L], indexing="ij")).reshape(4, -1).T
    lam = np.sort(np.repeat([H.free_eigenvalue(L, n) for n in grid], 8))
    assert np.abs(ev - lam).max() < 1e-12


def test_symmetric_and_bounded(oracle_lib):
    """<Y, A X> = <A Y, X>, and 0 <= spec(A) <= 1 for random links (Delta is negative
    semi-definite with norm at most 16); the spectrum is mirrored about 1/2 for even L."""
    L = (2, 2, 4, 4)
    U = inputs.random_links(L, eps=1.0, seed=9)
    X, Y = inputs.gaussian_fields(L, 2, seed=10)
    assert abs(oracle_lib.inner(Y, oracle_lib.lap(L, U, X)) - oracle_lib.inner(oracle_lib.lap(L, U, Y), X)) < 1e-12
    M = H.dense_operator(lambda Z: oracle_lib.lap(L, U, Z), L)
    assert np.abs(M - M.T).max() < 1e-14
    ev = np.sort(np.linalg.eigvalsh(M))
    assert ev[0] > -1e-13 and ev[-1] < 1 + 1e-13
    # checkerboard sign flips the hopping part: A = 1/2 - K with eps K eps = -K
    assert np.abs(np.sort(1.0 - ev) - ev).max() < 1e-12
    # odd Chebyshev traces vanish exactly
    Hm = 2 * M - np.eye(len(M))
    T1, T3 = Hm, 4 * Hm @ Hm @ Hm - 3 * Hm
    assert abs(np.trace(T1)) < 1e-10 and abs(np.trace(T3)) < 1e-9


def test_garbled_form_is_not_covariant(oracle_lib):
    """The backward hop with U^dag on both sides (as printed) breaks covariance, which the
    oracle's form passes; checked here on the hop itself with numpy."""
    rng = np.random.default_rng(0)
    U = inputs.random_su3(1, seed=11)[0]
    g0, g1 = inputs.random_su3(2, seed=12)
    X = H.to_mat(rng.standard_normal(8))
    # backward hop to x from x-nu: link U(x-nu), field at x-nu transforms with g1 (at x-nu),
    # U' = g1 U g0^dag; covariant result must transform with g0.
    Up, Xp = g1 @ U @ H.dag(g0), g1 @ X @ H.dag(g1)
    good = H.dag(Up) @ Xp @ Up
    bad = H.dag(Up) @ Xp @ H.dag(Up)
    assert np.abs(good - g0 @ (H.dag(U) @ X @ U) @ H.dag(g0)).max() < 1e-13
    assert np.abs(bad - g0 @ (H.dag(U) @ X @ H.dag(U)) @ H.dag(g0)).max() > 1e-3


def test_link_gradient_finite_difference(oracle_lib):
    """d<Z, A X>/dw^a for U_nu(y) -> exp(i w^a T^a) U_nu(y), against central differences."""
    L = (2, 4, 2, 4)
    U = inputs.random_links(L, eps=0.5, seed=13)
    X, Z = inputs.gaussian_fields(L, 2, seed=14)
    G = oracle_lib.lap_link_grad(L, U, X, Z, [1.0])
    rng = np.random.default_rng(15)
    h = 1e-5
    for _ in range(12):
        y, nu, a = int(rng.integers(0, np.prod(L))), int(rng.integers(0, 4)), int(rng.integers(0, 8))
        e = np.zeros(8)
        e[a] = h
        vals = []
        for sgn in (+1, -1):
            Up = U.copy()
            Up[y, nu] = H.mm(oracle_lib.exp_i(sgn * e), U[y, nu])
            vals.append(oracle_lib.inner(Z, oracle_lib.lap(L, Up, X)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - G[y, nu, a]) < 1e-8 * max(1.0, abs(fd))
    # two weighted pairs = weighted sum of single pairs
    X2, Z2 = inputs.gaussian_fields(L, 2, seed=16)
    G2 = oracle_lib.lap_link_grad(L, U, np.stack([X, X2]), np.stack([Z, Z2]), [0.3, -1.7])
    ref = 0.3 * G - 1.7 * oracle_lib.lap_link_grad(L, U, X2, Z2, [1.0])
    assert np.abs(G2 - ref).max() < 1e-12


@pytest.mark.parametrize("L", [ASYM, (3, 4, 3, 6)])
def test_site_sampled_form_equals_full(oracle_lib, L):
    """The site-sampled A X (the reference of the full-size parity tests) equals the full application,
    which the pins above fix, at every site of the lattice, visited in a shuffled order with repeats;
    odd extents exercise the periodic wrap at both ends."""
    V = int(np.prod(L))
    U = inputs.random_links(L, eps=0.7, seed=21)
    X = inputs.gaussian_fields(L, 1, seed=22)[0]
    full = oracle_lib.lap(L, U, X)
    rng = np.random.default_rng(23)
    sites = np.concatenate([rng.permutation(V), rng.integers(0, V, 17)]).astype(np.int64)
    Y = oracle_lib.lap_sites(L, U, X, sites)
    assert Y.shape == (len(sites), 4, 8)
    assert np.array_equal(Y, full[sites])
