"""Pins of the oracle's kinetic force and implicit leapfrog (Sec. 3, Eqs. 5-6)."""
import math

import numpy as np
import pytest

import helpers as H
from oracle import fit
from paper_2112_04556_gb300 import inputs

L2 = (2, 2, 2, 2)


def test_kinetic_force_finite_difference(oracle_lib):
    """F_K = -dT/dw, T = 1/2 |R(A(U)) P|^2, against central differences (h = 1e-5)
    along random single-link directions."""
    L = L2
    U = inputs.random_links(L, eps=0.5, seed=51)
    P = inputs.gaussian_fields(L, 1, seed=52)[0]
    m = fit.mass_term(12, 0.9)
    T, FK, Vel = oracle_lib.kinetic(L, U, P, m, tol=1e-14)
    rng = np.random.default_rng(53)
    h = 1e-5
    for _ in range(8):
        y, nu = int(rng.integers(0, 16)), int(rng.integers(0, 4))
        d = rng.standard_normal(8)
        vals = []
        for sgn in (+1, -1):
            Up = U.copy()
            Up[y, nu] = H.mm(oracle_lib.exp_i(sgn * h * d), U[y, nu])
            vals.append(oracle_lib.kinetic(L, Up, P, m, tol=1e-14)[0])
        fd = -(vals[0] - vals[1]) / (2 * h)
        an = float(FK[y, nu] @ d)
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_kinetic_identity_mass(oracle_lib):
    L = L2
    U = inputs.random_links(L, eps=0.5, seed=54)
    P = inputs.gaussian_fields(L, 1, seed=55)[0]
    T, FK, Vel = oracle_lib.kinetic(L, U, P, oracle_lib.identity_mass())
    assert abs(T - 0.5 * np.sum(P * P)) < 1e-12 and np.abs(FK).max() == 0 and np.abs(Vel - P).max() == 0


def test_kinetic_force_covariant(oracle_lib):
    L = (2, 2, 2, 4)
    V = 32
    U = inputs.random_links(L, eps=0.5, seed=56)
    P = inputs.gaussian_fields(L, 1, seed=57)[0]
    g = inputs.random_su3(V, seed=58)
    m = fit.mass_term(6, 0.9)
    T0, F0, V0 = oracle_lib.kinetic(L, U, P, m)
    T1, F1, V1 = oracle_lib.kinetic(L, H.gauge_transform_links(L, U, g), H.gauge_transform_field(P, g), m)
    assert abs(T0 - T1) < 1e-11 * T0
    assert np.abs(F1 - H.gauge_transform_field(F0, g)).max() < 1e-11
    assert np.abs(V1 - H.gauge_transform_field(V0, g)).max() < 1e-11


def test_heatbath_covariance_plane_wave(oracle_lib):
    """U = 1: P = m(A) R(A) xi acts on a plane wave as m(lam) R(lam) = m^{1/2}(lam)."""
    L = (4, 4, 4, 4)
    U = inputs.unit_links(L)
    m = fit.mass_term(12, 0.9)
    xi = H.plane_wave(L, (1, 2, 0, 3), 1, 4)
    P = oracle_lib.heatbath(L, U, xi, m)
    lam = H.free_eigenvalue(L, (1, 2, 0, 3))
    assert np.abs(P - math.sqrt(0.1 + 0.9 * lam) * xi).max() < 1e-12


def test_reversibility(oracle_lib):
    """Forward trajectory, momentum flip, forward again returns to the start."""
    L = L2
    U = inputs.random_links(L, eps=0.3, seed=61)
    P = inputs.gaussian_fields(L, 1, seed=62)[0]
    m = fit.mass_term(12, 0.9)
    U1, P1, _ = oracle_lib.md_trajectory(L, U, P, 0.4, 4, 6.0, 0.0, m, tol=1e-14)
    U2, P2, _ = oracle_lib.md_trajectory(L, U1, -P1, 0.4, 4, 6.0, 0.0, m, tol=1e-14)
    assert np.abs(U2 - U).max() < 1e-11
    assert np.abs(P2 + P).max() < 1e-10


def test_energy_error_scales_as_step_squared(oracle_lib):
    L = L2
    U = inputs.random_links(L, eps=0.3, seed=63)
    P = inputs.gaussian_fields(L, 1, seed=64)[0]
    m = fit.mass_term(8, 0.9)
    dH = []
    for n in (5, 10):
        H0 = oracle_lib.hamiltonian(L, U, P, 6.0, 0.0, m)[0]
        U1, P1, _ = oracle_lib.md_trajectory(L, U, P, 0.5, n, 6.0, 0.0, m)
        dH.append(oracle_lib.hamiltonian(L, U1, P1, 6.0, 0.0, m)[0] - H0)
    ratio = dH[0] / dH[1]
    assert 3.0 < ratio < 5.0, dH


def test_identity_mass_is_plain_leapfrog(oracle_lib):
    """M = 1: the implicit scheme reduces to the explicit leapfrog
    P' = P + eps/2 F(U), U' = exp(i eps P') U, P'' = P' + eps/2 F(U')."""
    L = (2, 2, 2, 4)
    U = inputs.random_links(L, eps=0.3, seed=65)
    P = inputs.gaussian_fields(L, 1, seed=66)[0]
    eps, n = 0.1, 5
    Ua, Pa, _ = oracle_lib.md_trajectory(L, U, P, eps * n, n, 6.0, -0.331, oracle_lib.identity_mass())
    Ub, Pb = U, P
    for _ in range(n):
        Ph = Pb + 0.5 * eps * oracle_lib.gauge_force(L, Ub, 6.0, -0.331)
        Ub = H.mm(oracle_lib.exp_i(eps * Ph), Ub)
        Pb = Ph + 0.5 * eps * oracle_lib.gauge_force(L, Ub, 6.0, -0.331)
    assert np.abs(Ua - Ub).max() < 1e-13 and np.abs(Pa - Pb).max() < 1e-12


@pytest.mark.slow
def test_plain_hmc_exp_minus_dH(oracle_lib):
    """<exp(-dH)> = 1 for an area-preserving reversible integrator (plain HMC, 2^4)."""
    L = L2
    U = inputs.random_links(L, eps=0.3, seed=0)
    U, _ = oracle_lib.plain_hmc(L, U, 20, 6.0, seed=5, tau=1.0, nsteps=10)
    vals = []
    for n in range(300):
        xi = oracle_lib.gauss_field(L, 9, n, 0)
        r = oracle_lib.trajectory(L, U, xi, oracle_lib.uniform(9, n), 1.0, 6, 6.0, 0.0,
                                  oracle_lib.identity_mass())
        U = r["U"]
        vals.append(math.exp(-r["dH"]))
    vals = np.array(vals)
    assert abs(vals.mean() - 1.0) < 4 * vals.std() / math.sqrt(len(vals)) + 1e-3


def test_aux_action_is_half_eta_squared(oracle_lib):
    """phi = R(A) eta gives S_aux = 1/2 <phi, M phi> = 1/2 |eta|^2 (M = R^{-2})."""
    L = L2
    U = inputs.random_links(L, eps=0.5, seed=71)
    eta = inputs.gaussian_fields(L, 1, seed=72)[0]
    m = fit.mass_term(12, 0.9)
    phi = oracle_lib.rational_apply(L, U, eta, m, 1e-14)[0]
    S = oracle_lib.aux_action(L, U, phi, m, 1e-14)
    assert abs(S - 0.5 * np.sum(eta * eta)) < 1e-11 * S


def test_aux_force_finite_difference(oracle_lib):
    """The auxiliary-field force is -dS_aux/dw (central differences along random single-link directions)."""
    L = L2
    U = inputs.random_links(L, eps=0.5, seed=73)
    phi = inputs.gaussian_fields(L, 1, seed=74)[0]
    m = fit.mass_term(8, 0.9)
    F = oracle_lib.potential_force(L, U, 6.0, 0.0, m, phi, 1e-14) - oracle_lib.gauge_force(L, U, 6.0, 0.0)
    rng = np.random.default_rng(75)
    h = 1e-5
    for _ in range(6):
        y, nu = int(rng.integers(0, 16)), int(rng.integers(0, 4))
        d = rng.standard_normal(8)
        vals = []
        for sgn in (+1, -1):
            Up = U.copy()
            Up[y, nu] = H.mm(oracle_lib.exp_i(sgn * h * d), U[y, nu])
            vals.append(oracle_lib.aux_action(L, Up, phi, m, 1e-14))
        fd = -(vals[0] - vals[1]) / (2 * h)
        an = float(F[y, nu] @ d)
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_aux_energy_error_scales_as_step_squared(oracle_lib):
    """With the auxiliary field in H and its force in the MD, dH still falls as the step size squared."""
    L = L2
    U = inputs.random_links(L, eps=0.3, seed=76)
    P = inputs.gaussian_fields(L, 1, seed=77)[0]
    eta = inputs.gaussian_fields(L, 1, seed=78)[0]
    m = fit.mass_term(8, 0.9)
    phi = oracle_lib.rational_apply(L, U, eta, m, 1e-14)[0]
    H = lambda U_, P_: (oracle_lib.hamiltonian(L, U_, P_, 6.0, 0.0, m)[0] + oracle_lib.aux_action(L, U_, phi, m))
    dH = []
    for n in (5, 10):
        H0 = H(U, P)
        U1, P1, _ = oracle_lib.md_trajectory(L, U, P, 0.5, n, 6.0, 0.0, m, phi=phi)
        dH.append(H(U1, P1) - H0)
    assert 3.0 < dH[0] / dH[1] < 5.0, dH


def _log_near_identity(W):
    """-i log W for a unitary W within ~1e-4 of the identity (series of log(1 + E) to E^4)."""
    E = W - np.eye(3)
    E2 = H.mm(E, E)
    return -1j * (E - E2 / 2 + H.mm(E2, E) / 3 - H.mm(E2, E2) / 4)


def _step_jacobian(oracle_lib, L, U0, P0, eps, m, symplectic=False, d=1e-5):
    """Jacobian of one step (U, P) -> (U'', P'') in right-trivialised coordinates, by central
    differences: links are moved as exp(i w) U and read back as w'' = -i log(U''(w) U''(0)^dagger), so
    at w = 0 the coordinate volume is the Haar volume.  Returns (J, P'')."""
    def step(U, P):
        r = oracle_lib.md_trajectory(L, U, P, eps, 1, 6.0, 0.0, m, tol=1e-14, fp_tol=1e-14, fp_maxit=200,
                                     symplectic=symplectic)
        return r[0], r[1]

    U1, P1 = step(U0, P0)
    U1d = H.dag(U1)
    n = P0.size
    J = np.empty((2 * n, 2 * n))
    for k in range(2 * n):
        outs = []
        for s in (+1, -1):
            e = np.zeros(n)
            e[k % n] = s * d
            e = e.reshape(P0.shape)
            if k < n:
                Ua, Pa = step(H.mm(oracle_lib.exp_i(e), U0), P0)
            else:
                Ua, Pa = step(U0, P0 + e)
            w = H.to_coef(_log_near_identity(H.mm(Ua, U1d)))
            outs.append(np.concatenate([w.ravel(), Pa.ravel()]))
        J[:, k] = (outs[0] - outs[1]) / (2 * d)
    return J, P1


def _step_log_jacobian(oracle_lib, L, U0, P0, eps, m, symplectic=False):
    """log |det| of the step's Jacobian with respect to Haar x Lebesgue measure."""
    sign, logdet = np.linalg.slogdet(_step_jacobian(oracle_lib, L, U0, P0, eps, m, symplectic)[0])
    assert sign > 0
    return logdet


def test_leapfrog_volume_identity_mass(oracle_lib):
    """M = 1: every sub-step is a shear (P by a force of U alone, U by a left translation
    exp(i eps P') U), so one step preserves the phase-space volume exactly."""
    L = (1, 1, 1, 2)
    U = inputs.random_links(L, eps=0.5, seed=67)
    P = inputs.gaussian_fields(L, 1, seed=68)[0]
    assert abs(_step_log_jacobian(oracle_lib, L, U, P, 0.2, oracle_lib.identity_mass())) < 1e-8


@pytest.mark.slow
def test_leapfrog_volume_error_is_third_order(oracle_lib):
    """A link-dependent mass: the generalised leapfrog of Sec. 3 written with group exponentials
    keeps the flat-space cancellation of the sub-step Jacobians up to the non-commuting terms of
    d exp, so log det J is not zero but, the step being symmetric (its inverse is the step with
    -eps), it is odd in eps and starts at eps^3: halving eps divides it by ~8.  A scheme that
    evaluated the velocity or the force at the wrong end of a sub-step would start at eps^2
    (ratio ~4)."""
    L = (1, 1, 1, 1)
    U = inputs.random_links(L, eps=0.5, seed=69)
    P = inputs.gaussian_fields(L, 1, seed=70)[0]
    m = fit.mass_term(4, 0.5)
    a = _step_log_jacobian(oracle_lib, L, U, P, 0.05, m)
    b = _step_log_jacobian(oracle_lib, L, U, P, 0.025, m)
    assert abs(b) > 1e-6, b
    assert 6.5 < a / b < 17.0, (a, b)


@pytest.mark.slow
def test_plain_hmc_strong_coupling_plaquette(oracle_lib):
    """The chain samples exp(-S) with the action normalised as in Sec. 2: at small beta the
    plaquette follows the strong-coupling (character) expansion.  One plaquette with weight
    exp(beta/3 ReTr U) under Haar measure has log Z = (beta/3)^2 <(ReTr U)^2>/2
    + (beta/3)^3 <(ReTr U)^3>/6 + ..., with the SU(3) Haar moments <|Tr U|^2> = 1,
    <(Tr U)^2> = 0, <(Tr U)^3> = 1 (so <(ReTr U)^2> = 1/2, <(ReTr U)^3> = 1/4), a vanishing fourth
    cumulant (<|Tr U|^4> = 2) and a fifth cumulant of -5/16; d log Z / d beta gives
    <ReTr U_p / 3> = beta/18 + beta^2/216 - 25 beta^4/466560 + ...  On the lattice the first
    correction comes from closed cubes, O(u^5) ~ 1e-6 at beta = 1.  100 trajectories on 4^4 resolve
    the beta^2 term at several standard deviations."""
    L = (4, 4, 4, 4)
    beta = 1.0
    U = inputs.random_links(L, eps=1.0, seed=3)
    U, _ = oracle_lib.plain_hmc(L, U, 5, beta, seed=11)
    plaq = []
    for n in range(100):
        U, _ = oracle_lib.plain_hmc(L, U, 1, beta, seed=1000 + n)
        plaq.append(oracle_lib.action(L, U, beta)[1])
    plaq = np.array(plaq)
    err = plaq.std() / math.sqrt(len(plaq))
    u = beta / 18 + beta ** 2 / 216 - 25 * beta ** 4 / 466560
    assert abs(plaq.mean() - u) < 4 * err, (plaq.mean(), u, err)
    assert plaq.mean() - beta / 18 > 0.5 * beta ** 2 / 216, (plaq.mean(), err)


def _structure_constants():
    """f^{abc} of su(3) from [T^a, T^b] = i f^{abc} T^c with the Gell-Mann matrices of the helpers."""
    T = H.TGEN
    f = np.empty((8, 8, 8))
    for a in range(8):
        for b in range(8):
            C = H.mm(T[a], T[b]) - H.mm(T[b], T[a])
            for c in range(8):
                f[a, b, c] = np.real(-2j * np.trace(H.mm(C, T[c])))
    return f


def _canonical_form(P):
    """Matrix of the canonical symplectic form of T*SU(3)^links at momenta P in right-trivialised
    coordinates (w, P): with the Liouville form theta = P.w and right-invariant fields, whose bracket is
    [X_a, X_b] = f^{abc} X_c, d theta((w1, P1), (w2, P2)) = P1.w2 - P2.w1 - f^{abc} w1^a w2^b P^c."""
    f = _structure_constants()
    Pl = P.reshape(-1, 8)
    n = Pl.size
    K = np.zeros((n, n))
    for l in range(len(Pl)):
        K[8 * l:8 * l + 8, 8 * l:8 * l + 8] = -np.einsum("abc,c->ab", f, Pl[l])
    return np.block([[K, -np.eye(n)], [np.eye(n), np.zeros((n, n))]])


def test_dexp_against_finite_differences(oracle_lib):
    """dexp_X Y = -i log(exp(i(X + tY).T) exp(-iX.T)) / t as t -> 0 (scipy's expm and logm), and
    dexp_inv inverts it; for Y parallel to X, dexp_X Y = Y."""
    import scipy.linalg as sl
    rng = np.random.default_rng(71)
    X = rng.standard_normal((3, 8)) * np.array([[0.1], [0.7], [2.0]])
    Y = rng.standard_normal((3, 8))
    D = oracle_lib.dexp(X, Y)
    t = 1e-6
    for l in range(3):
        Ep = sl.expm(1j * H.to_mat(X[l] + t * Y[l]))
        Em = sl.expm(1j * H.to_mat(X[l] - t * Y[l]))
        E0 = sl.expm(-1j * H.to_mat(X[l]))
        fd = H.to_coef(-1j * (sl.logm(Ep @ E0) - sl.logm(Em @ E0))) / (2 * t)
        assert np.abs(fd - D[l]).max() < 1e-8 * max(1.0, np.abs(D[l]).max())
    assert np.abs(oracle_lib.dexp_inv(X, D) - Y).max() < 1e-12
    assert np.abs(oracle_lib.dexp(X, 0.3 * X) - 0.3 * X).max() < 1e-14


@pytest.mark.slow
def test_symplectic_step_preserves_the_canonical_form(oracle_lib):
    """The Lie-group variational form of the implicit leapfrog is a symplectic map of T*SU(3):
    J^T Omega(P'') J = Omega(P) for the canonical form, so det J = 1; the form with the opposite sign
    of its structure-constant term is not preserved (the check sees that term), and the plain
    group-exponential leapfrog preserves neither."""
    L = (1, 1, 1, 1)
    U = inputs.random_links(L, eps=0.5, seed=69)
    P = inputs.gaussian_fields(L, 1, seed=70)[0]
    m = fit.mass_term(4, 0.5)
    J, P1 = _step_jacobian(oracle_lib, L, U, P, 0.1, m, symplectic=True)
    assert np.abs(J.T @ _canonical_form(P1) @ J - _canonical_form(P)).max() < 1e-8
    assert abs(np.linalg.slogdet(J)[1]) < 1e-8
    assert np.abs(J.T @ _canonical_form(-P1) @ J - _canonical_form(-P)).max() > 1e-2
    J0, P10 = _step_jacobian(oracle_lib, L, U, P, 0.1, m, symplectic=False)
    assert np.abs(J0.T @ _canonical_form(P10) @ J0 - _canonical_form(P)).max() > 1e-3


def test_symplectic_step_reversible_and_plain_for_identity_mass(oracle_lib):
    """Forward, momentum flip, forward returns to the start; with M = 1 (V = P, ad_P P = 0) the dexp
    factors drop out and the step is the group-exponential leapfrog."""
    L = L2
    U = inputs.random_links(L, eps=0.3, seed=72)
    P = inputs.gaussian_fields(L, 1, seed=73)[0]
    m = fit.mass_term(8, 0.9)
    U1, P1, _ = oracle_lib.md_trajectory(L, U, P, 0.2, 2, 6.0, 0.0, m, tol=1e-14, symplectic=True)
    U2, P2, _ = oracle_lib.md_trajectory(L, U1, -P1, 0.2, 2, 6.0, 0.0, m, tol=1e-14, symplectic=True)
    assert np.abs(U2 - U).max() < 1e-11 and np.abs(P2 + P).max() < 1e-10
    I = oracle_lib.identity_mass()
    Ua, Pa, _ = oracle_lib.md_trajectory(L, U, P, 0.3, 3, 6.0, -0.331, I, symplectic=True)
    Ub, Pb, _ = oracle_lib.md_trajectory(L, U, P, 0.3, 3, 6.0, -0.331, I, symplectic=False)
    assert np.abs(Ua - Ub).max() < 1e-12 and np.abs(Pa - Pb).max() < 1e-11


@pytest.mark.slow
def test_symplectic_energy_error_scales_as_step_squared(oracle_lib):
    L = L2
    U = inputs.random_links(L, eps=0.3, seed=63)
    P = inputs.gaussian_fields(L, 1, seed=64)[0]
    m = fit.mass_term(8, 0.9)
    H0 = oracle_lib.hamiltonian(L, U, P, 6.0, 0.0, m)[0]
    dH = []
    for n in (5, 10):
        U1, P1, _ = oracle_lib.md_trajectory(L, U, P, 0.5, n, 6.0, 0.0, m, symplectic=True)
        dH.append(oracle_lib.hamiltonian(L, U1, P1, 6.0, 0.0, m)[0] - H0)
    assert 3.0 < dH[0] / dH[1] < 5.0, dH
