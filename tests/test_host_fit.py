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
