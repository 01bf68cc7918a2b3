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
