// Rational mass term of Sec. 3, Eq. (6) for the linear target m(lam) = (1-kappa) + kappa lam:
// R(lam) = c + sum_j alpha_j / (lam + sigma_j) ~ m(lam)^{-1/2}, Zolotarev's best relative
// approximation of x^{-1/2} on [1-kappa, 1] mapped to lam in [0, 1].
//
// Zolotarev (1877): on y in [1, K] the best relative approximation of type (n, n) of y^{-1/2} is
//   d prod_{l=1..n} (y + c_{2l}) / (y + c_{2l-1}),  c_l = sn^2(l K'/(2n+1); k') / cn^2(l K'/(2n+1); k'),
// with complementary parameter k'^2 = 1 - 1/K and K' the complete elliptic integral at k'^2; d makes the
// relative error equioscillate.  The elliptic functions are computed here with the arithmetic-geometric
// mean (descending Landen transformation), in long double.
#include <math.h>

#include <algorithm>
#include <vector>

#include "../../include/rmhmc.h"

namespace {

typedef long double ld;

// complete elliptic integral of the first kind K(m), m = k^2, by the AGM: K = pi / (2 AGM(1, sqrt(1-m)))
ld ellip_K(ld m) {
    ld a = 1.0L, b = sqrtl(1.0L - m);
    for (int i = 0; i < 64 && fabsl(a - b) > 1e-21L * a; i++) {
        const ld an = 0.5L * (a + b);
        b = sqrtl(a * b);
        a = an;
    }
    return (ld)M_PI / (2.0L * a);
}

// sn and cn of (u | m) by the AGM scale with backward amplitude recursion
void ellip_sncn(ld u, ld m, ld& sn, ld& cn) {
    ld a[64], c[64];
    a[0] = 1.0L;
    ld b = sqrtl(1.0L - m);
    c[0] = sqrtl(m);
    int N = 0;
    while (N < 62 && fabsl(c[N]) > 1e-21L) {
        a[N + 1] = 0.5L * (a[N] + b);
        c[N + 1] = 0.5L * (a[N] - b);
        b = sqrtl(a[N] * b);
        N++;
    }
    ld phi = ldexpl(a[N] * u, N);
    for (int n = N; n > 0; n--) phi = 0.5L * (phi + asinl(c[n] * sinl(phi) / a[n]));
    sn = sinl(phi);
    cn = cosl(phi);
}

}  // namespace

extern "C" int rmhmc_mass_fit(int npole, double kappa, double* c, double* alpha, double* sigma, double* max_rel_err) {
    if (!c || npole < 0 || npole > 24 || (npole > 0 && (!alpha || !sigma))) return RMHMC_EINVAL;
    if (!(kappa >= 0.0 && kappa < 1.0)) return RMHMC_EINVAL;
    if (npole == 0 || kappa == 0.0) {
        if (npole != 0) return RMHMC_EINVAL;   // kappa = 0 is the identity mass: no poles
        *c = 1.0;
        if (max_rel_err) *max_rel_err = 0.0;
        return RMHMC_OK;
    }
    const int n = npole;
    const ld xmin = 1.0L - (ld)kappa, ratio = 1.0L / xmin;
    const ld mprime = 1.0L - 1.0L / ratio;
    const ld Kp = ellip_K(mprime);
    std::vector<ld> cl(2 * n + 1);
    for (int l = 1; l <= 2 * n; l++) {
        ld sn, cn;
        ellip_sncn((ld)l * Kp / (ld)(2 * n + 1), mprime, sn, cn);
        cl[l] = (sn * sn) / (cn * cn);
    }
    // d0 from equioscillation of sqrt(y) * prod on [1, ratio]
    auto f = [&](ld y) {
        ld p = sqrtl(y);
        for (int l = 1; l <= n; l++) p *= (y + cl[2 * l]) / (y + cl[2 * l - 1]);
        return p;
    };
    ld fmax = 0.0L, fmin = 1e300L;
    const int G = 20000;
    for (int i = 0; i <= G; i++) {
        const ld y = expl(logl(ratio) * (ld)i / (ld)G);
        const ld v = f(y);
        fmax = std::max(fmax, v);
        fmin = std::min(fmin, v);
    }
    const ld d0 = 2.0L / (fmax + fmin);
    // partial fractions in y: d0 [1 + sum_l b_l / (y + c_{2l-1})]
    const ld sx = sqrtl(xmin);
    for (int l = 1; l <= n; l++) {
        const ld p = cl[2 * l - 1];
        ld num = 1.0L, den = 1.0L;
        for (int m = 1; m <= n; m++) {
            num *= cl[2 * m] - p;
            if (m != l) den *= cl[2 * m - 1] - p;
        }
        const ld bl = num / den;
        // x = xmin y:  a_l / (x + s_l) with a_l = d0 sqrt(xmin) b_l, s_l = xmin c_{2l-1}; then lam: x = (1-k) + k lam
        const ld al = d0 * sx * bl, sl = xmin * p;
        alpha[l - 1] = (double)(al / (ld)kappa);
        sigma[l - 1] = (double)((xmin + sl) / (ld)kappa);
    }
    *c = (double)(d0 / sx);
    if (max_rel_err) {
        double e = 0.0;
        for (int i = 0; i <= 4096; i++) {
            const double lam = i / 4096.0;
            double r = *c;
            for (int j = 0; j < n; j++) r += alpha[j] / (lam + sigma[j]);
            e = std::max(e, fabs(r * sqrt((1.0 - kappa) + kappa * lam) - 1.0));
        }
        *max_rel_err = e;
    }
    return RMHMC_OK;
}

// ------------------------------------------------------------------------------------------------
// Mass term fitted to a measured force spectrum (Sec. 4: a mass term "fitted to match the spectral
// dependence of the gauge force").  Equal MD rates for every mode need M(lam) proportional to the force
// power per mode s(lam) (a harmonic mode of stiffness k has force power k and frequency^2 k / M);
// M = 1 at the largest measured power.  R = M^{-1/2} = c + sum_j alpha_j / (lam + sigma_j) with the poles on
// a fixed geometric grid and c, alpha_j >= 0 from non-negative least squares on the relative error.
// ------------------------------------------------------------------------------------------------
namespace {

// least squares min |A_P z - b| over the passive columns P (column-major A, m rows) by Householder QR;
// z receives the solution on P and 0 elsewhere
void ls_passive(int m, int n, const std::vector<double>& A, const std::vector<double>& b,
                const std::vector<char>& P, std::vector<double>& z) {
    std::vector<int> cols;
    for (int j = 0; j < n; j++)
        if (P[j]) cols.push_back(j);
    const int k = (int)cols.size();
    std::vector<double> Q((size_t)m * k), y(b);
    for (int c = 0; c < k; c++)
        for (int i = 0; i < m; i++) Q[(size_t)c * m + i] = A[(size_t)cols[c] * m + i];
    std::vector<double> diag(k, 0.0);
    for (int c = 0; c < k && c < m; c++) {
        double* v = &Q[(size_t)c * m];
        double nrm = 0.0;
        for (int i = c; i < m; i++) nrm += v[i] * v[i];
        nrm = sqrt(nrm);
        const double alpha = v[c] > 0 ? -nrm : nrm;
        diag[c] = alpha;
        if (nrm == 0.0) continue;
        v[c] -= alpha;   // Householder vector in v[c..m)
        double vv = 0.0;
        for (int i = c; i < m; i++) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        for (int c2 = c + 1; c2 < k; c2++) {
            double* u = &Q[(size_t)c2 * m];
            double d = 0.0;
            for (int i = c; i < m; i++) d += v[i] * u[i];
            d = 2.0 * d / vv;
            for (int i = c; i < m; i++) u[i] -= d * v[i];
        }
        double d = 0.0;
        for (int i = c; i < m; i++) d += v[i] * y[i];
        d = 2.0 * d / vv;
        for (int i = c; i < m; i++) y[i] -= d * v[i];
    }
    // back substitution R z = (Q^T b)[0..k)
    std::vector<double> zc(k, 0.0);
    for (int c = k - 1; c >= 0; c--) {
        double s = y[c];
        for (int c2 = c + 1; c2 < k; c2++) s -= Q[(size_t)c2 * m + c] * zc[c2];
        zc[c] = diag[c] != 0.0 ? s / diag[c] : 0.0;
    }
    z.assign(n, 0.0);
    for (int c = 0; c < k; c++) z[cols[c]] = zc[c];
}

// non-negative least squares min |A x - b|, x >= 0: the active-set method of Lawson and Hanson
// (Solving Least Squares Problems, 1974, Ch. 23)
void nnls(int m, int n, const std::vector<double>& A, const std::vector<double>& b, std::vector<double>& x) {
    x.assign(n, 0.0);
    std::vector<char> P(n, 0);
    std::vector<double> r(m), w(n), z;
    double anorm = 0.0;
    for (double a : A) anorm = std::max(anorm, fabs(a));
    const double tol = 1e-13 * anorm * m;
    for (int outer = 0; outer < 4 * n + 10; outer++) {
        for (int i = 0; i < m; i++) {
            double s = b[i];
            for (int j = 0; j < n; j++) s -= A[(size_t)j * m + i] * x[j];
            r[i] = s;
        }
        int t = -1;
        double wmax = tol;
        for (int j = 0; j < n; j++) {
            double s = 0.0;
            for (int i = 0; i < m; i++) s += A[(size_t)j * m + i] * r[i];
            w[j] = s;
            if (!P[j] && s > wmax) { wmax = s; t = j; }
        }
        if (t < 0) break;
        P[t] = 1;
        for (int inner = 0; inner < 4 * n + 10; inner++) {
            ls_passive(m, n, A, b, P, z);
            bool feasible = true;
            for (int j = 0; j < n; j++)
                if (P[j] && z[j] <= 0.0) feasible = false;
            if (feasible) { x = z; break; }
            double step = 1.0;
            for (int j = 0; j < n; j++)
                if (P[j] && z[j] <= 0.0) step = std::min(step, x[j] / (x[j] - z[j]));
            for (int j = 0; j < n; j++) {
                if (!P[j]) continue;
                x[j] += step * (z[j] - x[j]);
                if (x[j] <= 1e-300) { x[j] = 0.0; P[j] = 0; }
            }
        }
    }
}

}  // namespace

extern "C" int rmhmc_mass_fit_spectrum(int nwin, const double* lam, const double* spec, int npole, double sigma_min,
                                       double sigma_max, double* c, double* alpha, double* sigma, double* max_rel_err) {
    if (nwin < 1 || !lam || !spec || !c || npole < 0 || npole > 24 || (npole > 0 && (!alpha || !sigma)))
        return RMHMC_EINVAL;
    if (npole > 0 && !(sigma_min > 0.0 && sigma_max >= sigma_min && isfinite(sigma_max))) return RMHMC_EINVAL;
    double smax = 0.0;
    for (int w = 0; w < nwin; w++) {
        if (!(spec[w] > 0.0) || !isfinite(spec[w]) || !(lam[w] >= 0.0 && lam[w] <= 1.0)) return RMHMC_EINVAL;
        smax = std::max(smax, spec[w]);
    }
    std::vector<double> g(nwin);
    for (int w = 0; w < nwin; w++) g[w] = 1.0 / sqrt(spec[w] / smax);
    for (int j = 0; j < npole; j++)
        sigma[j] = npole == 1 ? sigma_min : sigma_min * pow(sigma_max / sigma_min, (double)j / (double)(npole - 1));
    const int n = npole + 1;
    std::vector<double> A((size_t)nwin * n), b(nwin, 1.0), x;
    for (int w = 0; w < nwin; w++) {
        A[w] = 1.0 / g[w];
        for (int j = 0; j < npole; j++) A[(size_t)(j + 1) * nwin + w] = 1.0 / ((lam[w] + sigma[j]) * g[w]);
    }
    nnls(nwin, n, A, b, x);
    *c = x[0];
    for (int j = 0; j < npole; j++) alpha[j] = x[j + 1];
    if (max_rel_err) {
        double e = 0.0;
        for (int w = 0; w < nwin; w++) {
            double r = *c;
            for (int j = 0; j < npole; j++) r += alpha[j] / (lam[w] + sigma[j]);
            e = std::max(e, fabs(r / g[w] - 1.0));
        }
        *max_rel_err = e;
    }
    return RMHMC_OK;
}
