"""Oracle rational mass term (Sec. 3, Eq. 6) — TEST INFRASTRUCTURE ONLY.

Eq. (6) writes the mass term as M = [c + sum_i (a_0i + a_1i lam)/(b_0i + b_1i lam + lam^2)]^{-2},
lam the eigenvalue of -Delta_G/16, i.e. the rational function R(lam) in brackets equals
M^{-1/2}.  Each quadratic denominator splits into two simple poles, so
    R(lam) = c + sum_{j=1}^{n} alpha_j / (lam + sigma_j).
The target mass shape is the linear Duane form m(lam) = (1 - kappa) + kappa lam
(config: kappa = 0.9, twelve poles), so R is the best rational approximation of
m^{-1/2}.  It is built as Zolotarev's optimal relative approximation of x^{-1/2}
on x in [1-kappa, 1] (Zolotarev 1877; e.g. Chiu et al. 2002 for the closed form),
with the elliptic functions taken from scipy, and then shifted to lam by
x = (1-kappa) + kappa lam.
"""
import numpy as np
from scipy.special import ellipj, ellipk


def zolotarev_inv_sqrt(n, xmin, xmax):
    """Best relative approximation of x^{-1/2} on [xmin, xmax] of type (n, n):
    r(x) = d + sum_l a_l / (x + s_l).  Returns (d, a[n], s[n], max relative error on a grid)."""
    ratio = xmax / xmin
    m = 1.0 - 1.0 / ratio                       # parameter k'^2 of the complementary modulus
    K = ellipk(m)
    l = np.arange(1, 2 * n + 1)
    sn, _, _, _ = ellipj(l * K / (2 * n + 1), m)
    c = sn ** 2 / (1.0 - sn ** 2)               # c_1 .. c_2n; odd ones are poles, even ones zeros
    poles = c[0::2]
    zeros = c[1::2]
    # unnormalised product form f(y) = prod (y + c_2l)/(y + c_2l-1) on y = x/xmin in [1, ratio];
    # the optimal scale equioscillates: d0 = 2 / (max sqrt(y) f + min sqrt(y) f)
    y = np.geomspace(1.0, ratio, 200001)
    f = np.sqrt(y) * np.prod((y[:, None] + zeros[None, :]) / (y[:, None] + poles[None, :]), axis=1)
    d0 = 2.0 / (f.max() + f.min())
    # partial fractions in y: d0 [1 + sum_l b_l / (y + p_l)]
    b = np.empty(n)
    for i in range(n):
        num = np.prod(zeros - poles[i])
        den = np.prod(np.delete(poles, i) - poles[i])
        b[i] = num / den
    # back to x = xmin y:  x^{-1/2} = xmin^{-1/2} (xmin/x)^{...}:  r(x) = xmin^{-1/2} R_y(x / xmin)
    d = d0 / np.sqrt(xmin)
    a = d0 * np.sqrt(xmin) * b
    s = xmin * poles
    err = np.abs(d0 * f - 1.0).max()
    return d, a, s, err


def mass_term(npole=12, kappa=0.9):
    """R(lam) = c + sum_j alpha_j/(lam + sigma_j) ~ m(lam)^{-1/2}, m = (1-kappa) + kappa lam."""
    if kappa == 0.0:
        return {"c": 1.0, "alpha": np.zeros(0), "sigma": np.zeros(0), "kappa": 0.0, "err": 0.0}
    d, a, s, err = zolotarev_inv_sqrt(npole, 1.0 - kappa, 1.0)
    sigma = (1.0 - kappa + s) / kappa
    alpha = a / kappa
    return {"c": float(d), "alpha": alpha, "sigma": sigma, "kappa": float(kappa), "err": float(err)}


def evaluate(mass, lam):
    lam = np.asarray(lam, dtype=np.float64)
    r = np.full_like(lam, mass["c"])
    for a, s in zip(mass["alpha"], mass["sigma"]):
        r = r + a / (lam + s)
    return r
