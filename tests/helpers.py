"""Test-side helpers written independently of the oracle and of the CUDA library:
Gell-Mann basis, coefficient <-> matrix maps, gauge transforms, plane waves."""
import numpy as np

from conftest import shift_index, site_coords

LAMBDA = np.zeros((8, 3, 3), dtype=np.complex128)
LAMBDA[0][0, 1] = LAMBDA[0][1, 0] = 1
LAMBDA[1][0, 1] = -1j
LAMBDA[1][1, 0] = 1j
LAMBDA[2][0, 0] = 1
LAMBDA[2][1, 1] = -1
LAMBDA[3][0, 2] = LAMBDA[3][2, 0] = 1
LAMBDA[4][0, 2] = -1j
LAMBDA[4][2, 0] = 1j
LAMBDA[5][1, 2] = LAMBDA[5][2, 1] = 1
LAMBDA[6][1, 2] = -1j
LAMBDA[6][2, 1] = 1j
LAMBDA[7] = np.diag([1, 1, -2]) / np.sqrt(3)
TGEN = LAMBDA / 2


def to_mat(p):
    return np.einsum("...a,aij->...ij", p, TGEN)


def to_coef(m):
    # x^a = Tr(lambda^a X) for Hermitian traceless X
    return np.real(np.einsum("aij,...ji->...a", LAMBDA, m))


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def mm(a, b):
    return np.einsum("...ij,...jk->...ik", a, b)


def gauge_transform_links(L, U, g):
    """U'_nu(x) = g(x) U_nu(x) g(x+nu)^dag."""
    out = np.empty_like(U)
    for nu in range(4):
        gp = g[shift_index(L, nu, +1)]
        out[:, nu] = mm(mm(g, U[:, nu]), dag(gp))
    return out


def gauge_transform_field(X, g):
    """X'_mu(x) = g(x) X_mu(x) g(x)^dag on coefficient fields [V,4,8]."""
    M = to_mat(X)
    return to_coef(mm(mm(g[:, None], M), dag(g)[:, None]))


def pure_gauge_links(L, g):
    """U_nu(x) = g(x) g(x+nu)^dag."""
    V = int(np.prod(L))
    U = np.empty((V, 4, 3, 3), dtype=np.complex128)
    for nu in range(4):
        U[:, nu] = mm(g, dag(g[shift_index(L, nu, +1)]))
    return U


def free_eigenvalue(L, n):
    """lambda_k of A = -Delta/16 on U = 1 for k_nu = 2 pi n_nu / L_nu."""
    k = 2 * np.pi * np.asarray(n) / np.asarray(L)
    return float(np.sum(np.sin(k / 2) ** 2) / 4.0)


def plane_wave(L, n, comp, a, phase=0.0):
    """X_comp^a(x) = cos(k.x + phase), all other coefficients zero."""
    V = int(np.prod(L))
    k = 2 * np.pi * np.asarray(n) / np.asarray(L)
    X = np.zeros((V, 4, 8))
    X[:, comp, a] = np.cos(site_coords(L) @ k + phase)
    return X


def dense_operator(apply, L, ncomp_dim=8):
    """Dense matrix of an operator acting on component 0 of [V,4,8] fields (8V x 8V)."""
    V = int(np.prod(L))
    n = 8 * V
    basis = np.zeros((n, V, 4, 8))
    idx = np.arange(n)
    basis[idx, idx // 8, 0, idx % 8] = 1.0
    Y = apply(basis)
    return Y[:, :, 0, :].reshape(n, n).T
