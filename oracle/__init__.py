"""FP64 CPU oracle for the RMHMC hot path — TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline legs of
`bench.py` may import this package.  It shares no code with the CUDA library
(`paper_2112_04556_gb300`); the two meet only through the seeded inputs of
`paper_2112_04556_gb300.inputs`, which hold none of the method's arithmetic.

The per-site primitives (Laplacian, its link derivative, gauge loops, the
exponential, Philox) are plain C in `oracle.c`; the algorithms built on them
(CG, Chebyshev moments and windows, rational mass term, kinetic force,
implicit leapfrog, Metropolis) are written below in numpy, step by step in the
order the method states them.  Everything is float64.

Paper: Nguyen, Boyle, Christ, Jang, Jung, "Riemannian manifold hybrid Monte
Carlo in lattice QCD", LATTICE2021 (arXiv:2112.04556).
  Sec. 2, Eq. (3): adjoint covariant Laplacian, normalised -Delta_G/16.
  Sec. 2, Eq. (4): per-mode power spectrum <F|B(lambda)|F> / Tr B(lambda),
                   B(lambda) = sum_i c_i T_i[-Delta_G/16].
  Sec. 3, Eq. (5): H = 1/2 Tr P^dag M^{-1} P + S[U]; the log|M| term through an
                   auxiliary field (aux_mass, aux_action, potential_force).
  Sec. 3, Eq. (6): M = [c + rational function of -Delta_G/16]^{-2}.
  Sec. 3: implicit (generalised) leapfrog of Girolami & Calderhead with group
          exponentials (leapfrog_step), and its exactly symplectic form on
          T*SU(3) (symplectic_step, with ad, dexp_matrix, dexp, dexp_inv).
  Sec. 4: Wilson flow and flowed energy (wilson_flow, flow_energy), band filters
          as vectors (cheb_filter_apply), the mass fitted to a spectrum (fit.py).

Parity pins: every function here is checked in tests/test_oracle_*.py against
closed forms, invariants, dense linear algebra or finite differences.
"""
import ctypes
import math
import os
import subprocess

import numpy as np

from . import fit

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP over sites)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-fPIC", "-shared",
                           src, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        I4 = ctypes.POINTER(ctypes.c_int)
        d = ctypes.c_double
        L.orc_lap.argtypes = [I4, P, P, P, ctypes.c_int]
        L.orc_lap_sites.argtypes = [I4, P, P, P, P, ctypes.c_long]
        L.orc_lap_link_grad.argtypes = [I4, P, P, P, ctypes.c_int, P, P]
        L.orc_action_density.argtypes = [I4, P, d, d, P, P]
        L.orc_gauge_force.argtypes = [I4, P, d, d, P]
        L.orc_gauge_force_sites.argtypes = [I4, P, d, d, P, ctypes.c_long, P]
        L.orc_link_update.argtypes = [I4, P, d, P, P]
        L.orc_exp_i.argtypes = [ctypes.c_long, P, P]
        L.orc_mat_mul.argtypes = [ctypes.c_long, P, P, P]
        L.orc_coef_to_mat.argtypes = [ctypes.c_long, P, P]
        L.orc_mat_to_coef.argtypes = [ctypes.c_long, P, P]
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_gauss_field.argtypes = [I4, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, P]
        L.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_uniform.restype = d
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dims(L):
    return (ctypes.c_int * 4)(*[int(v) for v in L])


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads():
    return lib().orc_num_threads()


def volume(L):
    return int(np.prod(L))


# --------------------------------------------------------------------------
# Sec. 2, Eq. (3): A = -Delta_G/16 and its link derivative
# --------------------------------------------------------------------------

def lap(L, U, X):
    """A X with A = -Delta_G/16 (Eq. 3), X of shape [V,4,8] or [n,V,4,8]."""
    U = _c(U, np.complex128)
    X = _c(X, np.float64)
    single = X.ndim == 3
    Xs = X[None] if single else X
    Y = np.empty_like(Xs)
    lib().orc_lap(_dims(L), _p(U), _p(Xs), _p(Y), Xs.shape[0])
    return Y[0] if single else Y


def lap_sites(L, U, X, sites):
    """(A X) at the listed sites only: returns [len(sites), 4, 8]."""
    U = _c(U, np.complex128)
    X = _c(X, np.float64)
    sites = _c(sites, np.int64)
    Y = np.empty((len(sites), 4, 8))
    lib().orc_lap_sites(_dims(L), _p(U), _p(X), _p(Y), _p(sites), len(sites))
    return Y


def lap_link_grad(L, U, X, Z, w):
    """G^a(y,nu) = sum_f w_f d<Z_f, A X_f>/dw^a for U_nu(y) -> exp(i w^a T^a) U_nu(y)."""
    U = _c(U, np.complex128)
    X = _c(X, np.float64)
    Z = _c(Z, np.float64)
    if X.ndim == 3:
        X, Z = X[None], Z[None]
    w = _c(np.atleast_1d(w), np.float64)
    G = np.empty(X.shape[1:], dtype=np.float64)
    lib().orc_lap_link_grad(_dims(L), _p(U), _p(X), _p(Z), X.shape[0], _p(w), _p(G))
    return G


def inner(X, Y):
    """<X,Y> = sum_{x,mu,a} X^a Y^a (= 2 sum Tr XY)."""
    return float(np.dot(np.ravel(X), np.ravel(Y)))


# --------------------------------------------------------------------------
# gauge action and force (Sec. 2: F_G = -dS/dU with left multiplication)
# --------------------------------------------------------------------------

def action_density(L, U, beta, c1=0.0):
    U = _c(U, np.complex128)
    V = volume(L)
    s = np.empty(V)
    p = np.empty(V)
    lib().orc_action_density(_dims(L), _p(U), float(beta), float(c1), _p(s), _p(p))
    return s, p


def action(L, U, beta, c1=0.0):
    """S = beta sum [c0 sum_plaq (1 - ReTr/3) + c1 sum_rect (1 - ReTr/3)], c0 = 1 - 8 c1;
    returns (S, plaquette average), both summed exactly (math.fsum)."""
    s, p = action_density(L, U, beta, c1)
    return math.fsum(s), math.fsum(p) / len(p)


def gauge_force(L, U, beta, c1=0.0):
    """F^a_mu(x) = -dS/dw^a, U_mu(x) -> exp(i w^a T^a) U_mu(x); shape [V,4,8]."""
    U = _c(U, np.complex128)
    F = np.empty((volume(L), 4, 8))
    lib().orc_gauge_force(_dims(L), _p(U), float(beta), float(c1), _p(F))
    return F


def gauge_force_sites(L, U, beta, c1, sites):
    """The gauge force at the listed sites only: [len(sites), 4, 8]."""
    U = _c(U, np.complex128)
    sites = _c(sites, np.int64)
    F = np.empty((len(sites), 4, 8))
    lib().orc_gauge_force_sites(_dims(L), _p(U), float(beta), float(c1), _p(sites), len(sites), _p(F))
    return F


def link_update(L, U, V, eps):
    """U <- exp(i eps V) U per link (Taylor series with scaling and squaring)."""
    U = _c(U, np.complex128)
    V = _c(V, np.float64)
    out = np.empty_like(U)
    lib().orc_link_update(_dims(L), _p(V), float(eps), _p(U), _p(out))
    return out


def exp_i(h):
    """exp(i sum_a h^a T^a) for h of shape [..., 8]."""
    h = _c(h, np.float64)
    n = h.size // 8
    out = np.empty(h.shape[:-1] + (3, 3), dtype=np.complex128)
    lib().orc_exp_i(n, _p(h), _p(out))
    return out


def coef_to_mat(p):
    p = _c(p, np.float64)
    out = np.empty(p.shape[:-1] + (3, 3), dtype=np.complex128)
    lib().orc_coef_to_mat(p.size // 8, _p(p), _p(out))
    return out


def mat_to_coef(m):
    m = _c(m, np.complex128)
    out = np.empty(m.shape[:-2] + (8,))
    lib().orc_mat_to_coef(m.size // 9, _p(m), _p(out))
    return out


# --------------------------------------------------------------------------
# counter-based random numbers (Philox4x32-10, Salmon et al. SC'11)
# --------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    c = _c(np.asarray(ctr, dtype=np.uint32), np.uint32)
    k = _c(np.asarray(key, dtype=np.uint32), np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def gauss_field(L, seed, stream, tag=0):
    """Gaussian su(3) field [V,4,8] from Philox block (n/2, site, stream, tag), key = seed."""
    out = np.empty((volume(L), 4, 8))
    lib().orc_gauss_field(_dims(L), int(seed), int(stream), int(tag), _p(out))
    return out


def uniform(seed, stream, tag=1):
    return lib().orc_uniform(int(seed), int(stream), int(tag))


# --------------------------------------------------------------------------
# Krylov solves: plain CG, one shift at a time (definition of (A+sigma)^{-1} b)
# --------------------------------------------------------------------------

def cg(apply, b, tol=1e-13, maxiter=10000):
    """Textbook conjugate gradients for a symmetric positive definite operator.
    Stops when the true relative residual |b - A x| / |b| <= tol."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = inner(r, r)
    bb = inner(b, b)
    if bb == 0.0:
        return x, 0, 0.0
    it = 0
    while it < maxiter:
        q = apply(p)
        alpha = rr / inner(p, q)
        x += alpha * p
        r -= alpha * q
        rr_new = inner(r, r)
        it += 1
        if math.sqrt(rr_new / bb) <= 0.5 * tol:
            true_r = b - apply(x)
            res = math.sqrt(inner(true_r, true_r) / bb)
            if res <= tol:
                return x, it, res
            r = true_r
            rr_new = inner(r, r)
            p = r.copy()
            rr = rr_new
            continue
        p = r + (rr_new / rr) * p
        rr = rr_new
    true_r = b - apply(x)
    raise RuntimeError("oracle CG did not converge: residual %g" % math.sqrt(inner(true_r, true_r) / bb))


def shifted_solves(L, U, b, sigma, tol=1e-13):
    """x_j = (A + sigma_j)^{-1} b for every shift, each by its own CG."""
    xs = []
    for s in sigma:
        x, _, _ = cg(lambda v, s=s: lap(L, U, v) + s * v, b, tol)
        xs.append(x)
    return np.array(xs)


def rational_apply(L, U, b, mass, tol=1e-13):
    """R(A) b = c b + sum_j alpha_j (A + sigma_j)^{-1} b (Eq. 6 in partial fractions).
    Returns (R b, [x_j])."""
    xs = shifted_solves(L, U, b, mass["sigma"], tol)
    y = mass["c"] * b
    for a, x in zip(mass["alpha"], xs):
        y = y + a * x
    return y, xs


# --------------------------------------------------------------------------
# Sec. 2, Eq. (4): Chebyshev band-pass filters and the per-mode spectrum
# --------------------------------------------------------------------------

def cheb_moments(L, U, F, N):
    """mu_k = <F, T_k(2A - 1) F>, k = 0..N, by the plain three-term recurrence
    v_0 = F, v_1 = (2A-1) F, v_{k+1} = 2 (2A-1) v_k - v_{k-1}."""
    H = lambda v: 2.0 * lap(L, U, v) - v
    mu = np.zeros(N + 1)
    v_prev = F
    mu[0] = inner(F, F)
    if N == 0:
        return mu
    v = H(F)
    mu[1] = inner(F, v)
    for k in range(2, N + 1):
        v_prev, v = v, 2.0 * H(v) - v_prev
        mu[k] = inner(F, v)
    return mu


def cheb_filter_apply(L, U, F, coef):
    """Y = sum_k coef[k] T_k(2A - 1) F: the filter applied as a vector (band-filtered fields of Sec. 4),
    by the same plain three-term recurrence, accumulating every term."""
    H = lambda v: 2.0 * lap(L, U, v) - v
    N = len(coef) - 1
    Y = coef[0] * F
    if N == 0:
        return Y
    v_prev, v = F, H(F)
    Y = Y + coef[1] * v
    for k in range(2, N + 1):
        v_prev, v = v, 2.0 * H(v) - v_prev
        Y = Y + coef[k] * v
    return Y


def jackson(N):
    """Jackson damping g_k, k = 0..N (kernel polynomial method)."""
    k = np.arange(N + 1)
    q = math.pi / (N + 1)
    return ((N - k + 1) * np.cos(q * k) + np.sin(q * k) / math.tan(q)) / (N + 1)


def window_coeffs(edges, N, kernel="jackson"):
    """C[w,k]: Chebyshev coefficients (in x = 2 lambda - 1) of the indicator of the
    window [edges[w], edges[w+1]] of eigenvalues of A, times the damping g_k."""
    edges = np.asarray(edges, dtype=np.float64)
    theta = np.arccos(np.clip(2.0 * edges - 1.0, -1.0, 1.0))
    k = np.arange(1, N + 1)
    C = np.zeros((len(edges) - 1, N + 1))
    for w in range(len(edges) - 1):
        ta, tb = theta[w], theta[w + 1]
        C[w, 0] = (ta - tb) / math.pi
        C[w, 1:] = 2.0 * (np.sin(k * ta) - np.sin(k * tb)) / (k * math.pi)
    if kernel == "jackson":
        C *= jackson(N)[None, :]
    return C


def power_spectrum(L, U, forces, noises, N, edges, kernel="jackson"):
    """Eq. (4): spec[f,w] = <F_f|B_w|F_f> / Tr B_w, with B_w = sum_k C[w,k] T_k(2A-1) and
    Tr B_w over the full [V,4,8] space estimated as the mean of <eta|B_w|eta> over the
    supplied noise fields (Hutchinson).  Returns (spec, num, tr, moments)."""
    C = window_coeffs(edges, N, kernel)
    mf = np.array([cheb_moments(L, U, F, N) for F in forces])
    mn = np.array([cheb_moments(L, U, e, N) for e in noises])
    num = mf @ C.T
    tr = (mn @ C.T).mean(axis=0)
    return num / tr[None, :], num, tr, np.concatenate([mf, mn])


# --------------------------------------------------------------------------
# Sec. 3, Eqs. (5)-(6): mass term, kinetic energy and force
# --------------------------------------------------------------------------

def identity_mass():
    return {"c": 1.0, "alpha": np.zeros(0), "sigma": np.zeros(0), "kappa": 0.0}


def kinetic(L, U, P, mass, tol=1e-13):
    """T = 1/2 <P, M^{-1} P> with M = R(A)^{-2}: T = 1/2 |R P|^2.
    Also the velocity V = M^{-1} P = R(R P) and the kinetic force
    F_K = -dT/dw = sum_j alpha_j <Z_j, (dA/dw) X_j>,
    X_j = (A+sigma_j)^{-1} P, Z_j = (A+sigma_j)^{-1} R P."""
    Y, X = rational_apply(L, U, P, mass, tol)
    Vel, Z = rational_apply(L, U, Y, mass, tol)
    T = 0.5 * math.fsum((Y * Y).ravel())
    if len(mass["sigma"]):
        FK = lap_link_grad(L, U, X, Z, mass["alpha"])
    else:
        FK = np.zeros_like(P)
    return T, FK, Vel


def heatbath(L, U, xi, mass, tol=1e-13):
    """Momentum refresh P = M^{1/2} xi, taken as m(A) R(A) xi with m(A) = (1-kappa) + kappa A
    (R ~ m^{-1/2}, so m R ~ m^{1/2} = M^{1/2} to the accuracy of the rational fit).  A general rational
    mass (kappa = 0 with poles, e.g. fitted to a spectrum) has P = R(A)^{-1} xi exactly, here by CG on
    the symmetric positive operator R(A), each application one set of shifted solves."""
    if mass.get("kappa", 0.0) == 0.0 and len(mass["sigma"]) > 0:
        P, _, _ = cg(lambda v: rational_apply(L, U, v, mass, 1e-2 * tol)[0], xi, tol=tol)
        return P
    y, _ = rational_apply(L, U, xi, mass, tol)
    k = mass.get("kappa", 0.0)
    return (1.0 - k) * y + k * lap(L, U, y)


def hamiltonian(L, U, P, beta, c1, mass, tol=1e-13):
    """H = 1/2 <P, M^{-1} P> + S[U] (Eq. 5 without the log|M| term)."""
    T, _, _ = kinetic(L, U, P, mass, tol)
    S, plaq = action(L, U, beta, c1)
    return T + S, T, S, plaq


def _maxabs(a):
    return float(np.max(np.abs(a))) if a.size else 0.0


# --------------------------------------------------------------------------
# Sec. 3: the log|M| term realised by an auxiliary field.  Integrating the momenta out of
# exp(-1/2 P M^{-1} P) leaves det M^{1/2}; an auxiliary field phi with action S_aux = 1/2 <phi, M phi>
# contributes det M^{-1/2}, so the links are distributed as exp(-S).  With M = R^{-2},
# S_aux = 1/2 |Q phi|^2 with Q = 1/R (partial fraction p0 + sum_j beta_j/(A + zeta_j), c > 0), which
# has the form of the kinetic energy with the mass term Q: its force is the kinetic force of phi
# under Q.  phi is drawn once per trajectory, phi = M^{-1/2} eta = R(A) eta, and held fixed in the MD.
# --------------------------------------------------------------------------

def aux_mass(mass):
    """The inverse mass term Q = 1/R as a partial fraction {c: p0, alpha: beta, sigma: zeta}."""
    inv = fit.inverse_partial_fraction(mass)
    if inv["p1"] != 0.0:
        raise ValueError("the auxiliary field needs c > 0 (1/R without a linear term)")
    return {"c": inv["p0"], "alpha": inv["beta"], "sigma": inv["zeta"], "kappa": 0.0}


def aux_action(L, U, phi, mass, tol=1e-13):
    """S_aux = 1/2 <phi, M phi> = 1/2 |Q phi|^2."""
    T, _, _ = kinetic(L, U, phi, aux_mass(mass), tol)
    return T


def potential_force(L, U, beta, c1, mass=None, phi=None, tol=1e-13):
    """F_G(U), plus the auxiliary-field force -d S_aux/dw when phi is given."""
    F = gauge_force(L, U, beta, c1)
    if phi is not None:
        _, FA, _ = kinetic(L, U, phi, aux_mass(mass), tol)
        F = F + FA
    return F


def leapfrog_step(L, U, P, eps, beta, c1, mass, Q0, tol=1e-13, fp_tol=1e-13, fp_maxit=100, FG=None, phi=None):
    """One generalised-leapfrog step (Sec. 3; Girolami & Calderhead) on SU(3):
      (1) P' = P + eps/2 F(U, P')                      [fixed point]
      (2) U' = exp(i eps/2 V(U',P')) exp(i eps/2 V(U,P')) U   [fixed point]
      (3) P'' = P' + eps/2 F(U', P')
    with F = F_G + F_K and V = M^{-1} P.  Iteration rules: step (1) starts from Q0 and,
    at iterate Q_i, evaluates F_K and V at (U, Q_i); it stops when max|Q_{i+1}-Q_i| <= fp_tol
    and keeps V(U, Q_i).  Step (2) starts from exp(i eps V(U,P')) U, evaluates V and F_K at
    (W_i, P') and stops when max|W_{i+1}-W_i| <= fp_tol, keeping F_K(W_i, P') for step (3).
    The Lie-Poisson term of the group flow is not included (it changes neither H nor the
    phase-space volume of the continuous flow).  Phase-space volume: exact for a link-independent
    mass; with a link-dependent mass the group exponentials leave log det J = O(eps^3) per step
    (finite-difference Jacobians in tests/test_oracle_hmc.py).
    FG (optional) is F_G(U) if the caller has it.  With an auxiliary field phi, F_G stands for the whole
    potential force F_G + F_aux (both depend on U only).
    Returns (U'', P'', next initial guess, iteration counts, F_G(U''))."""
    if FG is None:
        FG = potential_force(L, U, beta, c1, mass, phi, tol)
    Q = Q0
    for i1 in range(1, fp_maxit + 1):
        _, FK, V0 = kinetic(L, U, Q, mass, tol)
        Qn = P + 0.5 * eps * (FG + FK)
        done = _maxabs(Qn - Q) <= fp_tol
        Q = Qn
        if done:
            break
    else:
        raise RuntimeError("oracle: momentum fixed point did not converge")
    Ph = Q
    E0U = np.matmul(exp_i(0.5 * eps * V0), U)
    W = link_update(L, U, V0, eps)
    for i2 in range(1, fp_maxit + 1):
        _, FK1, V1 = kinetic(L, W, Ph, mass, tol)
        Wn = np.matmul(exp_i(0.5 * eps * V1), E0U)
        done = _maxabs(Wn - W) <= fp_tol
        W = Wn
        if done:
            break
    else:
        raise RuntimeError("oracle: link fixed point did not converge")
    FG1 = potential_force(L, W, beta, c1, mass, phi, tol)
    P2 = Ph + 0.5 * eps * (FG1 + FK1)
    Qnext = P2 + 0.5 * eps * (FG1 + FK1)
    return W, P2, Qnext, (i1, i2), FG1


# --------------------------------------------------------------------------
# Sec. 3's implicit leapfrog written as a Lie-group variational integrator (exactly symplectic on
# T*SU(3)).  The generalised leapfrog is the composition of the two symplectic Euler methods; on the
# group, symplectic Euler comes from the discrete Lagrangian h L(U, xi) with exp(i h xi) = U_{k+1} U_k^-1,
# whose discrete Legendre transforms carry the right-trivialised derivative of the exponential.
# --------------------------------------------------------------------------

def ad(X, Y):
    """ad_X Y: coefficients of i [X^a T^a, Y^b T^b] (the bracket of the generators i X.T and i Y.T)."""
    A = coef_to_mat(X)
    B = coef_to_mat(Y)
    return mat_to_coef(1j * (np.matmul(A, B) - np.matmul(B, A)))


def ad_matrix(X):
    """8x8 matrix (per link) of Y -> ad_X Y."""
    X = _c(X, np.float64)
    cols = []
    for b in range(8):
        e = np.zeros(X.shape)
        e[..., b] = 1.0
        cols.append(ad(X, e))
    return np.stack(cols, axis=-1)


def dexp_matrix(X, nterms=40):
    """8x8 matrix (per link) of dexp_X = sum_n ad_X^n / (n+1)!, the right-trivialised derivative of the
    exponential: d/dt exp(i (X + t Y).T) exp(-i X.T) = i (dexp_X Y).T.  The series is entire."""
    A = ad_matrix(X)
    term = np.broadcast_to(np.eye(8), A.shape).copy()
    acc = term.copy()
    fact = 1.0
    for n in range(1, nterms):
        term = np.matmul(A, term)
        fact *= n + 1
        acc = acc + term / fact
    return acc


def dexp(X, Y):
    return np.einsum("...ab,...b->...a", dexp_matrix(X), Y)


def dexp_inv(X, Y):
    """Z with dexp_X Z = Y, by a linear solve per link."""
    return np.linalg.solve(dexp_matrix(X), _c(Y, np.float64)[..., None])[..., 0]


def symplectic_step(L, U, P, eps, beta, c1, mass, Q0, tol=1e-13, fp_tol=1e-13, fp_maxit=100, FG=None, phi=None):
    """One step of the implicit leapfrog as the composition of the two Lie-group symplectic Euler maps
    of half a step, h = eps/2 (F = F_G + F_K, V = M^{-1} P as in `leapfrog_step`):
      (A) mu:  dexp^{-1}_{X1} mu = P + h F(U, mu),  X1 = h V(U, mu);  B = exp(i X1) U;
          P_h = dexp^{-1}_{-X1} mu
      (B) (mu2, U'):  dexp^{-1}_{X2} mu2 = P_h,  X2 = h V(U', mu2),  U' = exp(i X2) B;
          P'' = dexp^{-1}_{-X2} mu2 + h F(U', mu2).
    Each half is the discrete Legendre transform of the discrete Lagrangian h L(U_k, xi) (A) or
    h L(U_{k+1}, xi) (B) with L = 1/2 xi.M xi - S; each is symplectic and B is the adjoint of A, so the
    step preserves the phase-space volume exactly and is reversible.  With dexp = 1 it is
    `leapfrog_step`; to first order in h the dexp terms add the Lie-Poisson term ad_V P to dP/dt.
    Iteration rules as in `leapfrog_step`: (A) starts from Q0 and, at iterate mu_i, evaluates F_K and V
    at (U, mu_i), sets mu_{i+1} = dexp_{h V}(P + h F) and stops when max|mu_{i+1} - mu_i| <= fp_tol,
    keeping X1 = h V(U, mu_i).  (B) starts from mu2 = mu_{i+1} and W = exp(2 i X1) U; at (W_j, mu2_j) it
    evaluates F_K and V, sets X2 = h V, mu2_{j+1} = dexp_{X2} P_h, W_{j+1} = exp(i X2) B, and stops when
    the larger of max|W_{j+1} - W_j| and max|mu2_{j+1} - mu2_j| is <= fp_tol, keeping F_K and X2 of
    (W_j, mu2_j).
    Returns (U'', P'', next initial guess, iteration counts, F_G(U''))."""
    h = 0.5 * eps
    if FG is None:
        FG = potential_force(L, U, beta, c1, mass, phi, tol)
    mu = Q0
    for i1 in range(1, fp_maxit + 1):
        _, FK, V = kinetic(L, U, mu, mass, tol)
        mun = dexp(h * V, P + h * (FG + FK))
        done = _maxabs(mun - mu) <= fp_tol
        mu = mun
        if done:
            break
    else:
        raise RuntimeError("oracle: momentum fixed point did not converge")
    X1 = h * V
    B = np.matmul(exp_i(X1), U)
    Ph = dexp_inv(-X1, mu)
    mu2 = mu
    W = np.matmul(exp_i(2.0 * X1), U)
    for i2 in range(1, fp_maxit + 1):
        _, FK1, V1 = kinetic(L, W, mu2, mass, tol)
        X2 = h * V1
        mu2n = dexp(X2, Ph)
        Wn = np.matmul(exp_i(X2), B)
        done = max(_maxabs(Wn - W), _maxabs(mu2n - mu2)) <= fp_tol
        W, mu2 = Wn, mu2n
        if done:
            break
    else:
        raise RuntimeError("oracle: link fixed point did not converge")
    FG1 = potential_force(L, W, beta, c1, mass, phi, tol)
    P2 = dexp_inv(-X2, mu2) + h * (FG1 + FK1)
    Qnext = P2 + h * (FG1 + FK1)
    return W, P2, Qnext, (i1, i2), FG1


def md_trajectory(L, U, P, tau, nsteps, beta, c1, mass, tol=1e-13, fp_tol=1e-13, fp_maxit=100, phi=None,
                  symplectic=False):
    """nsteps generalised-leapfrog steps of size tau/nsteps; the first momentum
    fixed point starts from P + eps/2 F_G(U) (F_G + F_aux with an auxiliary field phi).
    symplectic=True takes `symplectic_step` instead of `leapfrog_step`."""
    eps = tau / nsteps
    FG = potential_force(L, U, beta, c1, mass, phi, tol)
    Q0 = P + 0.5 * eps * FG
    iters = []
    step = symplectic_step if symplectic else leapfrog_step
    for _ in range(nsteps):
        U, P, Q0, it, FG = step(L, U, P, eps, beta, c1, mass, Q0, tol, fp_tol, fp_maxit, FG, phi)
        iters.append(it)
    return U, P, iters


def trajectory(L, U, xi, u, tau, nsteps, beta, c1, mass, tol_md=1e-13, tol_h=1e-13,
               fp_tol=1e-13, fp_maxit=100, metropolis=True, eta=None, symplectic=False):
    """One RMHMC trajectory: heatbath P = M^{1/2} xi, H0, MD, H1, accept if u <= exp(-dH).
    With eta (a Gaussian field), the log|M| term is included through the auxiliary field
    phi = R(A) eta, held fixed in the MD, and H = T + S + S_aux."""
    phi = rational_apply(L, U, eta, mass, tol_h)[0] if eta is not None else None
    P0 = heatbath(L, U, xi, mass, tol_h)
    H0, T0, S0, _ = hamiltonian(L, U, P0, beta, c1, mass, tol_h)
    A0 = aux_action(L, U, phi, mass, tol_h) if phi is not None else 0.0
    U1, P1, iters = md_trajectory(L, U, P0, tau, nsteps, beta, c1, mass, tol_md, fp_tol, fp_maxit, phi, symplectic)
    H1, T1, S1, plaq1 = hamiltonian(L, U1, P1, beta, c1, mass, tol_h)
    A1 = aux_action(L, U1, phi, mass, tol_h) if phi is not None else 0.0
    H0 += A0
    H1 += A1
    dH = H1 - H0
    accept = (not metropolis) or (u <= math.exp(-dH) if dH > 0 else True)
    Uout = U1 if accept else U
    return {"U": Uout, "U1": U1, "P0": P0, "P1": P1, "H0": H0, "H1": H1, "dH": dH,
            "T0": T0, "S0": S0, "T1": T1, "S1": S1, "A0": A0, "A1": A1, "accepted": bool(accept),
            "plaq": action(L, Uout, beta, c1)[1], "iters": iters}


def plain_hmc(L, U, ntraj, beta, seed, tau=1.0, nsteps=20, c1=0.0, metropolis=True):
    """Plain HMC (M = 1) with Philox momenta (stream = trajectory index).  metropolis=False accepts
    every trajectory (thermalisation from an ordered start, where dH is far from O(1))."""
    m = identity_mass()
    acc = 0
    for n in range(ntraj):
        xi = gauss_field(L, seed, n, 0)
        r = trajectory(L, U, xi, uniform(seed, n), tau, nsteps, beta, c1, m, metropolis=metropolis)
        U = r["U"]
        acc += r["accepted"]
    return U, acc


# --------------------------------------------------------------------------
# Wilson gradient flow and the flowed energy (the observable of Sec. 4, defined by Luscher,
# JHEP 08 (2010) 071, which the paper cites for it)
# --------------------------------------------------------------------------

def flow_energy(L, U):
    """Plaquette definition of the energy density, averaged over sites:
    E = (1/V) sum_x 2 sum_{mu<nu} Re Tr(1 - P_mu,nu(x)) = 36 (1 - <Re Tr P / 3>)."""
    _, plaq = action(L, U, 1.0)
    return 36.0 * (1.0 - plaq)


def wilson_flow(L, U, eps, nsteps):
    """Luscher's third-order Runge-Kutta scheme for dV/dt = -g0^2 (dS_W) V, nsteps steps of size eps:
        W1 = exp(Z0/4) W0,  W2 = exp(8/9 Z1 - 17/36 Z0) W1,  W3 = exp(3/4 Z2 - 8/9 Z1 + 17/36 Z0) W2,
    Z_i = eps Z(W_i).  With U -> exp(i w^a T^a) U and F = -dS/dw (gauge_force), the flow velocity is
    i g0^2 F^a T^a; g0^2 = 6/beta and F is proportional to beta, so g0^2 F = 6 F(beta = 1) and the
    flow does not depend on beta.  Returns the flowed links and E(t) at t = 0, eps, ..., nsteps eps."""
    U = np.array(U, dtype=np.complex128, copy=True)
    E = [flow_energy(L, U)]
    for _ in range(nsteps):
        Z0 = 6.0 * gauge_force(L, U, 1.0)
        W1 = link_update(L, U, Z0, 0.25 * eps)
        Z1 = 6.0 * gauge_force(L, W1, 1.0)
        W2 = link_update(L, W1, (8.0 / 9.0) * Z1 - (17.0 / 36.0) * Z0, eps)
        Z2 = 6.0 * gauge_force(L, W2, 1.0)
        U = link_update(L, W2, 0.75 * Z2 - (8.0 / 9.0) * Z1 + (17.0 / 36.0) * Z0, eps)
        E.append(flow_energy(L, U))
    return U, np.array(E)
