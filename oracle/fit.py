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


def spectrum_mass_term(lam, spec, npole, sigma_min=1e-3, sigma_max=10.0):
    """Mass term fitted to a measured force power spectrum per mode (Sec. 4: the mass term "fitted to
    match the spectral dependence of the gauge force").  A harmonic mode of stiffness k has force power k
    and moves with frequency^2 = k / M, so every mode moves at the same rate when M(lam) is proportional
    to the power s(lam); M is normalised to 1 at the largest measured power.  With R = M^{-1/2} the
    target is g_w = (s_w / max s)^{-1/2} at the window centres lam_w.  The poles sigma_j are fixed on a
    geometric grid in [sigma_min, sigma_max]; c >= 0 and alpha_j >= 0 solve the non-negative least-squares
    problem min sum_w (R(lam_w) / g_w - 1)^2, so R is positive and decreasing and M = R^{-2} positive and
    increasing.  kappa = 0 marks a general rational mass (heatbath P = R(A)^{-1} xi)."""
    from scipy.optimize import nnls
    lam = np.asarray(lam, dtype=np.float64)
    spec = np.asarray(spec, dtype=np.float64)
    g = (spec / spec.max()) ** -0.5
    sigma = np.geomspace(sigma_min, sigma_max, npole)
    cols = [np.ones_like(lam)] + [1.0 / (lam + s) for s in sigma]
    A = np.column_stack(cols) / g[:, None]
    x, _ = nnls(A, np.ones_like(lam))
    mass = {"c": float(x[0]), "alpha": x[1:].copy(), "sigma": sigma, "kappa": 0.0}
    mass["err"] = float(np.abs(evaluate(mass, lam) / g - 1.0).max())
    return mass


def inverse_partial_fraction(mass):
    """1/R(lam) = p0 + p1 lam + sum_j beta_j / (lam + zeta_j) for R = c + sum_j alpha_j/(lam + sigma_j) with
    c >= 0, alpha_j > 0: R has one zero between consecutive poles (and one below the smallest -sigma when
    c > 0), found here with Brent's method; beta_j = 1 / R'(-zeta_j); p1 = 0 and p0 = 1/c when c > 0,
    else 1/R ~ lam / sum(alpha) + sum(alpha sigma) / sum(alpha)^2 at infinity."""
    from scipy.optimize import brentq
    keep = np.asarray(mass["alpha"]) > 0
    alpha = np.asarray(mass["alpha"], dtype=np.float64)[keep]
    sigma = np.asarray(mass["sigma"], dtype=np.float64)[keep]
    order = np.argsort(sigma)
    alpha, sigma = alpha[order], sigma[order]
    c = float(mass["c"])
    m = {"c": c, "alpha": alpha, "sigma": sigma}
    R = lambda x: evaluate(m, x)
    zeros = []
    for j in range(len(sigma) - 1):
        a, b = -sigma[j + 1], -sigma[j]
        w = b - a
        zeros.append(brentq(R, a + 1e-14 * w, b - 1e-14 * w, xtol=1e-300, rtol=1e-15, maxiter=500))
    if c > 0 and len(sigma):
        b = -sigma[-1]
        a = b - 1.0
        while R(a) < 0:
            a = b - 2.0 * (b - a)
        zeros.append(brentq(R, a, b - 1e-14 * max(1.0, abs(b)), xtol=1e-300, rtol=1e-15, maxiter=500))
    zeros = np.array(zeros)
    dR = lambda x: -np.sum(alpha / (x + sigma) ** 2)
    beta = np.array([1.0 / dR(z) for z in zeros])
    if c > 0:
        p0, p1 = 1.0 / c, 0.0
    else:
        sa = alpha.sum()
        p0, p1 = float(np.sum(alpha * sigma) / sa ** 2), 1.0 / sa
    return {"p0": p0, "p1": p1, "beta": beta, "zeta": -zeros}
