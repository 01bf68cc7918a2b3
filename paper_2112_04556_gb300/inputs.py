"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the benchmark.

This module holds none of the method's arithmetic: it only draws random
numbers and packs them into the library's canonical layouts.

Layouts (canonical, used at the C ABI):
  links   U: complex128 [V][4][3][3], site s = x + Lx*(y + Ly*(z + Lz*t))
  fields  X: float64 [nfield][V][4][8], coefficients in the basis T^a = lambda^a/2

Link recipe: U_mu(x) = exp(i * eps * sum_a r_a T_a) with r_a ~ N(0,1) drawn by
numpy's PCG64 from `seed` (eps = 0.3 and seed 0 for the 4^4 workload).  The
matrix exponential of the Hermitian argument is taken through numpy's batched
Hermitian eigensolver, so no part of the library's own exponential is used.
"""
import numpy as np

SQRT3 = np.sqrt(3.0)


def volume(dims):
    v = 1
    for d in dims:
        v *= int(d)
    return v


def _hermitian_from_coefficients(r):
    """H = sum_a r_a lambda_a / 2 for r of shape [..., 8] (Gell-Mann basis)."""
    h = np.zeros(r.shape[:-1] + (3, 3), dtype=np.complex128)
    h[..., 0, 1] = r[..., 0] - 1j * r[..., 1]
    h[..., 0, 2] = r[..., 3] - 1j * r[..., 4]
    h[..., 1, 2] = r[..., 5] - 1j * r[..., 6]
    h[..., 1, 0] = np.conj(h[..., 0, 1])
    h[..., 2, 0] = np.conj(h[..., 0, 2])
    h[..., 2, 1] = np.conj(h[..., 1, 2])
    h[..., 0, 0] = r[..., 2] + r[..., 7] / SQRT3
    h[..., 1, 1] = -r[..., 2] + r[..., 7] / SQRT3
    h[..., 2, 2] = -2.0 * r[..., 7] / SQRT3
    return 0.5 * h


def _expi_hermitian(h):
    """exp(i h) for Hermitian h [..., 3, 3] via eigen-decomposition."""
    w, v = np.linalg.eigh(h)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), np.conj(v))


def random_links(dims, eps=0.3, seed=0, chunk=1 << 18):
    """Random SU(3) links U = exp(i eps sum_a r_a T_a), r_a ~ N(0,1) (PCG64(seed))."""
    V = volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.standard_normal((V, 4, 8))
    U = np.empty((V, 4, 3, 3), dtype=np.complex128)
    flat_r = r.reshape(-1, 8)
    flat_u = U.reshape(-1, 3, 3)
    for i in range(0, flat_r.shape[0], chunk):
        flat_u[i:i + chunk] = _expi_hermitian(eps * _hermitian_from_coefficients(flat_r[i:i + chunk]))
    return U


def unit_links(dims):
    V = volume(dims)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def gaussian_fields(dims, nfield=1, seed=1):
    """nfield su(3) link fields with N(0,1) coefficients, shape [nfield][V][4][8]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((nfield, volume(dims), 4, 8))


def random_su3(n, seed=2, eps=1.0):
    """n random SU(3) matrices exp(i eps sum_a r_a T_a) (used as gauge transforms)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return _expi_hermitian(eps * _hermitian_from_coefficients(rng.standard_normal((n, 8))))


def equal_windows(nwin, offset=0.0):
    """nwin+1 window edges splitting [0,1] evenly, optionally shifted inward by `offset`."""
    e = np.linspace(0.0, 1.0, nwin + 1)
    if offset:
        e[1:-1] += offset
    return e
