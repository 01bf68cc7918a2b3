/*
 * FP64 CPU oracle for the RMHMC hot path (Nguyen, Boyle, Christ, Jang, Jung,
 * "Riemannian manifold hybrid Monte Carlo in lattice QCD", LATTICE2021).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of what the method computes.  It shares no code with the CUDA
 * library; only the tests, the package smoke check and the CPU-baseline leg
 * of the benchmark load it.  Every routine works on 3x3 complex matrices in
 * double precision with plain loops over sites; the only optimisation is an
 * OpenMP "parallel for" over independent sites, which does not change any
 * result (every site is written by exactly one iteration, no reductions).
 *
 * Conventions (fixed once for the whole project):
 *   site s = x + Lx*(y + Ly*(z + Lz*t)), periodic in all four directions;
 *   links U[s][mu][i][j], complex128;
 *   su(3) fields as coefficients p^a (a = 1..8 stored at 0..7) in the basis
 *   T^a = lambda^a / 2 (Gell-Mann), P = sum_a p^a T^a, layout [V][4][8];
 *   left-multiplication derivative: U -> exp(i w^a T^a) U (Sec. 2, below Eq. 3).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef double complex cplx;
typedef struct { cplx e[3][3]; } mat3;

/* ------------------------------------------------------------------ */
/* lattice geometry                                                     */
/* ------------------------------------------------------------------ */

static long volume(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords(const int L[4], long s, int c[4]) {
    for (int d = 0; d < 4; d++) { c[d] = (int)(s % L[d]); s /= L[d]; }
}

static long index_of(const int L[4], const int c[4]) {
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

/* site reached from s by n steps along direction mu (n may be negative) */
static long shift_site(const int L[4], long s, int mu, int n) {
    int c[4];
    coords(L, s, c);
    c[mu] = ((c[mu] + n) % L[mu] + L[mu]) % L[mu];
    return index_of(L, c);
}

/* ------------------------------------------------------------------ */
/* 3x3 complex algebra                                                  */
/* ------------------------------------------------------------------ */

static mat3 m_zero(void) { mat3 r; memset(&r, 0, sizeof r); return r; }
static mat3 m_unit(void) { mat3 r = m_zero(); for (int i = 0; i < 3; i++) r.e[i][i] = 1.0; return r; }

static mat3 m_mul(mat3 a, mat3 b) {
    mat3 r = m_zero();
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) r.e[i][j] += a.e[i][k] * b.e[k][j];
    return r;
}

static mat3 m_dag(mat3 a) {
    mat3 r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) r.e[i][j] = conj(a.e[j][i]);
    return r;
}

static mat3 m_add(mat3 a, mat3 b) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) a.e[i][j] += b.e[i][j];
    return a;
}

static mat3 m_scale(mat3 a, cplx z) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) a.e[i][j] *= z;
    return a;
}

static cplx m_trace(mat3 a) { return a.e[0][0] + a.e[1][1] + a.e[2][2]; }

static double m_maxabs(mat3 a) {
    double m = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) if (cabs(a.e[i][j]) > m) m = cabs(a.e[i][j]);
    return m;
}

static mat3 m_load(const double *p) {          /* 9 complex numbers, row major */
    mat3 r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) r.e[i][j] = p[2 * (3 * i + j)] + I * p[2 * (3 * i + j) + 1];
    return r;
}

static void m_store(double *p, mat3 a) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            p[2 * (3 * i + j)] = creal(a.e[i][j]);
            p[2 * (3 * i + j) + 1] = cimag(a.e[i][j]);
        }
}

/* Gell-Mann generators T^a = lambda^a / 2, a = 1..8 stored at 0..7 */
static mat3 T[8];
static int T_ready = 0;

static void init_generators(void) {
    if (T_ready) return;
    for (int a = 0; a < 8; a++) T[a] = m_zero();
    T[0].e[0][1] = 1;   T[0].e[1][0] = 1;             /* lambda_1 */
    T[1].e[0][1] = -I;  T[1].e[1][0] = I;             /* lambda_2 */
    T[2].e[0][0] = 1;   T[2].e[1][1] = -1;            /* lambda_3 */
    T[3].e[0][2] = 1;   T[3].e[2][0] = 1;             /* lambda_4 */
    T[4].e[0][2] = -I;  T[4].e[2][0] = I;             /* lambda_5 */
    T[5].e[1][2] = 1;   T[5].e[2][1] = 1;             /* lambda_6 */
    T[6].e[1][2] = -I;  T[6].e[2][1] = I;             /* lambda_7 */
    T[7].e[0][0] = 1.0 / sqrt(3.0); T[7].e[1][1] = 1.0 / sqrt(3.0);
    T[7].e[2][2] = -2.0 / sqrt(3.0);                  /* lambda_8 */
    for (int a = 0; a < 8; a++) T[a] = m_scale(T[a], 0.5);
    T_ready = 1;
}

/* P = sum_a p^a T^a */
static mat3 from_coef(const double *p) {
    mat3 r = m_zero();
    for (int a = 0; a < 8; a++) r = m_add(r, m_scale(T[a], p[a]));
    return r;
}

/* p^a = 2 Re Tr(T^a P): the coefficients of the traceless Hermitian part */
static void to_coef(mat3 m, double *p) {
    for (int a = 0; a < 8; a++) p[a] = 2.0 * creal(m_trace(m_mul(T[a], m)));
}

/* Re Tr(i T^a M) for a = 1..8: the left-multiplication derivative of Re Tr(M) */
static void deriv_coef(mat3 m, double *g) {
    for (int a = 0; a < 8; a++) g[a] = creal(I * m_trace(m_mul(T[a], m)));
}

/* exp(M) by Taylor series with scaling and squaring (no closed form used) */
static mat3 m_exp(mat3 m) {
    int s = 0;
    double nrm = m_maxabs(m) * 3.0;
    while (nrm > 0.25) { nrm *= 0.5; s++; }
    mat3 a = m_scale(m, ldexp(1.0, -s));
    mat3 term = m_unit(), sum = m_unit();
    for (int k = 1; k <= 30; k++) {
        term = m_scale(m_mul(term, a), 1.0 / k);
        sum = m_add(sum, term);
        if (m_maxabs(term) < 1e-19) break;
    }
    for (int k = 0; k < s; k++) sum = m_mul(sum, sum);
    return sum;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition */
/* ------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    memcpy(out, c, sizeof c);
}

/* Two uniforms in (0,1] (53 bits each) from one Philox block, then the
 * Box-Muller transform: g0 = r cos(2 pi u1), g1 = r sin(2 pi u1), r = sqrt(-2 ln u0). */
static void gauss_pair(const uint32_t w[4], double *g0, double *g1) {
    uint64_t k0 = ((uint64_t)(w[0] >> 5) << 26) | (w[1] >> 6);
    uint64_t k1 = ((uint64_t)(w[2] >> 5) << 26) | (w[3] >> 6);
    double u0 = ((double)k0 + 1.0) * 0x1p-53;
    double u1 = ((double)k1 + 1.0) * 0x1p-53;
    double r = sqrt(-2.0 * log(u0));
    *g0 = r * cos(2.0 * M_PI * u1);
    *g1 = r * sin(2.0 * M_PI * u1);
}

/* Gaussian su(3) field [V][4][8]: coefficient n = 8*mu + a of site s comes from
 * block counter (n/2, s, stream, tag), key (seed_lo, seed_hi); even n takes g0. */
void orc_gauss_field(const int L[4], uint64_t seed, uint32_t stream, uint32_t tag, double *out) {
    long V = volume(L);
    #pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        for (int k = 0; k < 16; k++) {
            uint32_t ctr[4] = {(uint32_t)k, (uint32_t)s, stream, tag};
            uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
            uint32_t w[4];
            orc_philox4x32_10(ctr, key, w);
            gauss_pair(w, &out[32 * s + 2 * k], &out[32 * s + 2 * k + 1]);
        }
    }
}

/* uniform in (0,1] for the Metropolis test: block (0, 0xFFFFFFFF, stream, tag) */
double orc_uniform(uint64_t seed, uint32_t stream, uint32_t tag) {
    uint32_t ctr[4] = {0u, 0xFFFFFFFFu, stream, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint64_t k0 = ((uint64_t)(w[0] >> 5) << 26) | (w[1] >> 6);
    return ((double)k0 + 1.0) * 0x1p-53;
}

/* ------------------------------------------------------------------ */
/* normalised covariant Laplacian, Sec. 2 Eq. (3), A = -Delta_G / 16      */
/* ------------------------------------------------------------------ */

/* Y = A X for nfield fields of layout [V][4][8]; each of the 4 components
 * P_mu of a field is an independent adjoint-valued operand.
 * Delta X(x) = sum_nu [ U_nu(x) X(x+nu) U_nu(x)^dag
 *                     + U_nu(x-nu)^dag X(x-nu) U_nu(x-nu) - 2 X(x) ].
 * (The second term is taken as U^dag X U: the form printed with U^dag on both
 *  sides is not gauge covariant; the covariance test decides.) */
void orc_lap(const int L[4], const double *U, const double *X, double *Y, int nfield) {
    init_generators();
    long V = volume(L);
    for (int f = 0; f < nfield; f++) {
        const double *Xf = X + (long)f * V * 32;
        double *Yf = Y + (long)f * V * 32;
        #pragma omp parallel for schedule(static)
        for (long s = 0; s < V; s++) {
            for (int c = 0; c < 4; c++) {
                mat3 xc = from_coef(Xf + 32 * s + 8 * c);
                mat3 acc = m_zero();
                for (int nu = 0; nu < 4; nu++) {
                    long sp = shift_site(L, s, nu, +1), sm = shift_site(L, s, nu, -1);
                    mat3 uf = m_load(U + 18 * (4 * s + nu));
                    mat3 ub = m_load(U + 18 * (4 * sm + nu));
                    mat3 xp = from_coef(Xf + 32 * sp + 8 * c);
                    mat3 xm = from_coef(Xf + 32 * sm + 8 * c);
                    acc = m_add(acc, m_mul(m_mul(uf, xp), m_dag(uf)));
                    acc = m_add(acc, m_mul(m_mul(m_dag(ub), xm), ub));
                    acc = m_add(acc, m_scale(xc, -2.0));
                }
                to_coef(m_scale(acc, -1.0 / 16.0), Yf + 32 * s + 8 * c);
            }
        }
    }
}

/* A X at a list of sites only (same arithmetic as orc_lap; used to sample large lattices) */
void orc_lap_sites(const int L[4], const double *U, const double *X, double *Y, const long *sites, long nsites) {
    init_generators();
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < nsites; i++) {
        long s = sites[i];
        for (int c = 0; c < 4; c++) {
            mat3 xc = from_coef(X + 32 * s + 8 * c);
            mat3 acc = m_zero();
            for (int nu = 0; nu < 4; nu++) {
                long sp = shift_site(L, s, nu, +1), sm = shift_site(L, s, nu, -1);
                mat3 uf = m_load(U + 18 * (4 * s + nu));
                mat3 ub = m_load(U + 18 * (4 * sm + nu));
                acc = m_add(acc, m_mul(m_mul(uf, from_coef(X + 32 * sp + 8 * c)), m_dag(uf)));
                acc = m_add(acc, m_mul(m_mul(m_dag(ub), from_coef(X + 32 * sm + 8 * c)), ub));
                acc = m_add(acc, m_scale(xc, -2.0));
            }
            to_coef(m_scale(acc, -1.0 / 16.0), Y + 32 * i + 8 * c);
        }
    }
}

/* Link derivative of the bilinear form:  G^a(y,nu) = sum_f w_f d<Z_f, A X_f>/dw^a
 * with U_nu(y) -> exp(i w^a T^a) U_nu(y), <X,Y> = sum_{x,mu,a} X^a Y^a.
 * Only two terms of Delta contain U = U_nu(y): the forward hop at y and the
 * backward hop at y+nu.  Writing W1 = U X(y+nu) U^dag and W2 = U Z(y+nu) U^dag,
 *   d<Z, Delta X>/dw^a = 2 i sum_mu { Tr(T^a [W1, Z(y)]) - Tr(T^a [X(y), W2]) },
 * and A = -Delta/16 multiplies this by -1/16. */
void orc_lap_link_grad(const int L[4], const double *U, const double *X, const double *Z,
                       int nfield, const double *w, double *G) {
    init_generators();
    long V = volume(L);
    #pragma omp parallel for schedule(static)
    for (long y = 0; y < V; y++) {
        for (int nu = 0; nu < 4; nu++) {
            long yp = shift_site(L, y, nu, +1);
            mat3 u = m_load(U + 18 * (4 * y + nu));
            double g[8] = {0};
            for (int f = 0; f < nfield; f++) {
                const double *Xf = X + (long)f * V * 32, *Zf = Z + (long)f * V * 32;
                for (int c = 0; c < 4; c++) {
                    mat3 w1 = m_mul(m_mul(u, from_coef(Xf + 32 * yp + 8 * c)), m_dag(u));
                    mat3 w2 = m_mul(m_mul(u, from_coef(Zf + 32 * yp + 8 * c)), m_dag(u));
                    mat3 zy = from_coef(Zf + 32 * y + 8 * c);
                    mat3 xy = from_coef(Xf + 32 * y + 8 * c);
                    mat3 c1 = m_add(m_mul(w1, zy), m_scale(m_mul(zy, w1), -1.0));
                    mat3 c2 = m_add(m_mul(xy, w2), m_scale(m_mul(w2, xy), -1.0));
                    mat3 d = m_add(c1, m_scale(c2, -1.0));
                    for (int a = 0; a < 8; a++)
                        g[a] += w[f] * (-1.0 / 16.0) * creal(2.0 * I * m_trace(m_mul(T[a], d)));
                }
            }
            for (int a = 0; a < 8; a++) G[32 * y + 8 * nu + a] = g[a];
        }
    }
}

/* ------------------------------------------------------------------ */
/* gauge action and force from closed loops (Sec. 2, below Eq. 3)       */
/* ------------------------------------------------------------------ */

/* A loop shape is a list of steps; step code = +(d+1) for a move along +d
 * (multiply by U_d(pos)), -(d+1) for a move along -d (multiply by U_d(pos-d)^dag).
 * The action is  S = beta * sum_shapes w_shape * sum_x (1 - Re Tr W(x)/3). */
#define MAXSTEP 8
typedef struct { int n; int step[MAXSTEP]; double w; } shape_t;

static int make_shapes(double c1, shape_t *sh) {
    int n = 0;
    double c0 = 1.0 - 8.0 * c1;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++) {
            shape_t s = {4, {mu + 1, nu + 1, -(mu + 1), -(nu + 1)}, c0};
            sh[n++] = s;
        }
    if (c1 != 0.0)
        for (int mu = 0; mu < 4; mu++)
            for (int nu = 0; nu < 4; nu++) {
                if (mu == nu) continue;
                shape_t s = {6, {mu + 1, mu + 1, nu + 1, -(mu + 1), -(mu + 1), -(nu + 1)}, c1};
                sh[n++] = s;
            }
    return n;
}

static mat3 link_step(const int L[4], const double *U, long *pos, int code) {
    int d = (code > 0 ? code : -code) - 1;
    if (code > 0) {
        mat3 u = m_load(U + 18 * (4 * (*pos) + d));
        *pos = shift_site(L, *pos, d, +1);
        return u;
    }
    *pos = shift_site(L, *pos, d, -1);
    return m_dag(m_load(U + 18 * (4 * (*pos) + d)));
}

/* per-site action density s(x) = beta sum_shapes w (1 - ReTr W/3), and the
 * per-site plaquette average (1/6) sum_{mu<nu} ReTr P_{mu nu}(x)/3 */
void orc_action_density(const int L[4], const double *U, double beta, double c1,
                        double *sdens, double *plaq) {
    shape_t sh[64];
    int ns = make_shapes(c1, sh);
    long V = volume(L);
    #pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) {
        double sx = 0.0, px = 0.0;
        for (int k = 0; k < ns; k++) {
            long pos = x;
            mat3 w = m_unit();
            for (int i = 0; i < sh[k].n; i++) w = m_mul(w, link_step(L, U, &pos, sh[k].step[i]));
            double rt = creal(m_trace(w)) / 3.0;
            sx += beta * sh[k].w * (1.0 - rt);
            if (sh[k].n == 4) px += rt / 6.0;
        }
        sdens[x] = sx;
        plaq[x] = px;
    }
}

/* F^a_mu(y) = -dS/dw^a for U_mu(y) -> exp(i w^a T^a) U_mu(y).  For every loop
 * through the link: if it passes forward, W = A U B and d ReTr W = ReTr(i T U B A);
 * if backward, W = A U^dag B and d ReTr W = ReTr(-i T B A U^dag).
 * Hence F = (beta w / 3) * sum over occurrences of those derivatives. */
static void gauge_force_link(const int L[4], const double *U, const shape_t *sh, int ns, double beta,
                             long y, int mu, double *out) {
    double f[8] = {0};
    mat3 u = m_load(U + 18 * (4 * y + mu));
    for (int k = 0; k < ns; k++) {
        for (int i = 0; i < sh[k].n; i++) {
            int code = sh[k].step[i];
            int d = (code > 0 ? code : -code) - 1;
            if (d != mu) continue;
            /* displacement of steps 0..i-1 */
            int disp[4] = {0, 0, 0, 0};
            for (int j = 0; j < i; j++) {
                int cj = sh[k].step[j];
                disp[(cj > 0 ? cj : -cj) - 1] += (cj > 0 ? 1 : -1);
            }
            /* start site: forward step i starts at y; backward step i ends at y */
            long x = (code > 0) ? y : shift_site(L, y, mu, +1);
            for (int e = 0; e < 4; e++) x = shift_site(L, x, e, -disp[e]);
            long pos = x;
            mat3 A = m_unit(), B = m_unit();
            for (int j = 0; j < i; j++) A = m_mul(A, link_step(L, U, &pos, sh[k].step[j]));
            (void)link_step(L, U, &pos, code);
            for (int j = i + 1; j < sh[k].n; j++) B = m_mul(B, link_step(L, U, &pos, sh[k].step[j]));
            double g[8];
            if (code > 0) deriv_coef(m_mul(m_mul(u, B), A), g);
            else deriv_coef(m_scale(m_mul(m_mul(B, A), m_dag(u)), -1.0), g);
            for (int a = 0; a < 8; a++) f[a] += beta * sh[k].w / 3.0 * g[a];
        }
    }
    for (int a = 0; a < 8; a++) out[a] = f[a];
}

void orc_gauge_force(const int L[4], const double *U, double beta, double c1, double *F) {
    init_generators();
    shape_t sh[64];
    int ns = make_shapes(c1, sh);
    long V = volume(L);
    #pragma omp parallel for schedule(static)
    for (long y = 0; y < V; y++)
        for (int mu = 0; mu < 4; mu++) gauge_force_link(L, U, sh, ns, beta, y, mu, F + 32 * y + 8 * mu);
}

/* the force at a list of sites only (all four directions): F[i][mu][8] */
void orc_gauge_force_sites(const int L[4], const double *U, double beta, double c1, const long *sites, long nsites,
                           double *F) {
    init_generators();
    shape_t sh[64];
    int ns = make_shapes(c1, sh);
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < nsites; i++)
        for (int mu = 0; mu < 4; mu++) gauge_force_link(L, U, sh, ns, beta, sites[i], mu, F + 32 * i + 8 * mu);
}

/* ------------------------------------------------------------------ */
/* link update U <- exp(i eps V) U, and helpers on raw matrices          */
/* ------------------------------------------------------------------ */

void orc_link_update(const int L[4], const double *V, double eps, const double *Uin, double *Uout) {
    init_generators();
    long vol = volume(L);
    #pragma omp parallel for schedule(static)
    for (long s = 0; s < vol; s++)
        for (int mu = 0; mu < 4; mu++) {
            mat3 h = from_coef(V + 32 * s + 8 * mu);
            mat3 e = m_exp(m_scale(h, I * eps));
            m_store(Uout + 18 * (4 * s + mu), m_mul(e, m_load(Uin + 18 * (4 * s + mu))));
        }
}

/* exp(i h) for a list of Hermitian matrices given by coefficients */
void orc_exp_i(long n, const double *h, double *out) {
    init_generators();
    for (long k = 0; k < n; k++) m_store(out + 18 * k, m_exp(m_scale(from_coef(h + 8 * k), I)));
}

/* matrix product of n pairs: out_k = a_k b_k (used to build gauge transforms) */
void orc_mat_mul(long n, const double *a, const double *b, double *out) {
    for (long k = 0; k < n; k++) m_store(out + 18 * k, m_mul(m_load(a + 18 * k), m_load(b + 18 * k)));
}

/* coefficient <-> matrix conversion for n su(3) elements */
void orc_coef_to_mat(long n, const double *p, double *m) {
    init_generators();
    for (long k = 0; k < n; k++) m_store(m + 18 * k, from_coef(p + 8 * k));
}
void orc_mat_to_coef(long n, const double *m, double *p) {
    init_generators();
    for (long k = 0; k < n; k++) to_coef(m_load(m + 18 * k), p + 8 * k);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
