"""Host logic of the library that needs no GPU: the Zolotarev mass-term fit (rmhmc_mass_fit, C++ with its
own AGM elliptic functions) against the oracle's scipy-based fit, its error bound, and argument checks."""
import ctypes

import numpy as np
import pytest

from oracle import fit


def _lib():
    import __graft_entry__ as ge
    return ctypes.CDLL(ge.build_library())


def _fit(L, n, kappa):
    c = ctypes.c_double()
    a = np.zeros(max(n, 1))
    s = np.zeros(max(n, 1))
    e = ctypes.c_double()
    code = L.rmhmc_mass_fit(ctypes.c_int(n), ctypes.c_double(kappa), ctypes.byref(c),
                            a.ctypes.data_as(ctypes.c_void_p), s.ctypes.data_as(ctypes.c_void_p), ctypes.byref(e))
    return code, c.value, a[:n], s[:n], e.value


@pytest.mark.parametrize("n,kappa", [(12, 0.9), (6, 0.9), (3, 0.5), (12, 0.99), (2, 0.9)])
def test_fit_matches_oracle(n, kappa):
    code, c, a, s, e = _fit(_lib(), n, kappa)
    assert code == 0
    m = fit.mass_term(n, kappa)
    assert abs(c / m["c"] - 1) < 1e-12
    assert np.abs(a / m["alpha"] - 1).max() < 1e-11
    assert np.abs(s / m["sigma"] - 1).max() < 1e-11
    lam = np.linspace(0, 1, 10001)
    r = c + np.sum(a[None, :] / (lam[:, None] + s[None, :]), axis=1)
    err = np.abs(r * np.sqrt((1 - kappa) + kappa * lam) - 1).max()
    assert err <= max(2 * m["err"], 1e-14) and e <= max(2 * m["err"], 1e-14)


def test_fit_arguments():
    L = _lib()
    assert _fit(L, -1, 0.9)[0] == -1
    assert _fit(L, 12, 1.0)[0] == -1
    assert _fit(L, 25, 0.9)[0] == -1
    code, c, _, _, e = _fit(L, 0, 0.0)
    assert code == 0 and c == 1.0 and e == 0.0


@pytest.mark.parametrize("kernel", [0, 1])
def test_window_coefficients_match_oracle(kernel):
    """cheb_window_coeffs (host C++) against the oracle's numpy expansion of the window indicators."""
    import oracle
    lib = _lib()
    edges = np.array([0.0, 0.05, 0.2, 0.5, 0.51, 1.0])
    N = 150
    C = np.zeros((len(edges) - 1, N + 1))
    P = ctypes.POINTER(ctypes.c_double)
    rc = lib.cheb_window_coeffs(ctypes.c_int(len(edges) - 1), edges.ctypes.data_as(P), ctypes.c_int(N),
                                ctypes.c_int(kernel), C.ctypes.data_as(P))
    assert rc == 0
    ref = oracle.window_coeffs(edges, N, kernel="jackson" if kernel == 1 else "none")
    assert np.abs(C - ref).max() < 1e-14
    bad = np.array([0.0, 0.5, 0.4])
    assert lib.cheb_window_coeffs(ctypes.c_int(2), bad.ctypes.data_as(P), ctypes.c_int(N), ctypes.c_int(1),
                                  C.ctypes.data_as(P)) == -1


def _spec_fit(lam, spec, npole, smin=1e-3, smax=10.0):
    lib = _lib()
    P = ctypes.POINTER(ctypes.c_double)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    spec = np.ascontiguousarray(spec, dtype=np.float64)
    c = ctypes.c_double()
    err = ctypes.c_double()
    alpha = np.zeros(npole)
    sigma = np.zeros(npole)
    rc = lib.rmhmc_mass_fit_spectrum(ctypes.c_int(len(lam)), lam.ctypes.data_as(P), spec.ctypes.data_as(P),
                                     ctypes.c_int(npole), ctypes.c_double(smin), ctypes.c_double(smax),
                                     ctypes.byref(c), alpha.ctypes.data_as(P), sigma.ctypes.data_as(P),
                                     ctypes.byref(err))
    return rc, {"c": c.value, "alpha": alpha, "sigma": sigma, "kappa": 0.0}, err.value


@pytest.mark.parametrize("shape", ["rational", "linear", "curved"])
def test_spectrum_fit_matches_oracle(shape):
    """rmhmc_mass_fit_spectrum (host C++, its own Lawson-Hanson NNLS) against the oracle's scipy NNLS fit:
    the fitted R agrees at the windows and on [0, 1]."""
    lam = (np.arange(64) + 0.5) / 64
    if shape == "rational":
        s = 5.0 * fit.evaluate({"c": 0.3, "alpha": np.array([0.01, 0.0, 0.2, 0.05, 0.0, 0.3, 0.0, 0.4]),
                                "sigma": np.geomspace(1e-3, 10.0, 8)}, lam) ** -2
    elif shape == "linear":
        s = 0.1 + lam
    else:
        s = 0.05 + lam ** 1.3 + 0.2 * np.sin(3 * lam) ** 2
    rc, m, err = _spec_fit(lam, s, 8)
    assert rc == 0
    ref = fit.spectrum_mass_term(lam, s, 8)
    assert np.abs(m["sigma"] - ref["sigma"]).max() < 1e-14 * 10
    grid = np.linspace(0.0, 1.0, 101)
    assert np.abs(fit.evaluate(m, grid) / fit.evaluate(ref, grid) - 1).max() < 1e-8
    assert abs(err - ref["err"]) < 1e-8 + 1e-6 * ref["err"]
    assert m["c"] >= 0 and np.all(m["alpha"] >= 0)


def test_spectrum_fit_arguments():
    lam = np.array([0.1, 0.5, 0.9])
    assert _spec_fit(lam, np.array([1.0, -1.0, 2.0]), 4)[0] == -1
    assert _spec_fit(np.array([0.1, 1.5, 0.9]), np.ones(3), 4)[0] == -1
    assert _spec_fit(lam, np.ones(3), 25)[0] == -1
    assert _spec_fit(lam, np.ones(3), 4, smin=0.0)[0] == -1
