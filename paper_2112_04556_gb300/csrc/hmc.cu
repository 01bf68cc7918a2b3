// Sec. 3: the RMHMC trajectory.  Heatbath, Hamiltonian H = 1/2 <P, M^{-1} P> + S[U] (Eq. 5 without
// the log|M| term), the generalised (implicit) leapfrog of Girolami & Calderhead on SU(3), the float64
// link update exp(i eps V) U with reunitarisation, and the Metropolis test.
//
// One leapfrog step (F = F_G + F_K, V = M^{-1} P):
//   (1) P' = P + eps/2 F(U, P')                                      fixed point in P'
//   (2) U' = exp(i eps/2 V(U', P')) exp(i eps/2 V(U, P')) U          fixed point in U'
//   (3) P'' = P' + eps/2 F(U', P')
// Iteration rules: (1) starts from the previous step's P'' + eps/2 F (or P + eps/2 F_G(U) on the first
// step); at iterate Q_i it evaluates F_K and V at (U, Q_i) with one Krylov run and stops when
// max|Q_{i+1} - Q_i| <= fp_tol, keeping V(U, Q_i).  (2) starts from exp(i eps V) U, evaluates V and F_K
// at (W_i, P') and stops when max|W_{i+1} - W_i| <= fp_tol, keeping F_K(W_i, P') for (3).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "df.cuh"
#include "krylov.cuh"
#include "ops.cuh"
#include "philox.cuh"

namespace rm {

// ------------------------------------------------------------------------------------------------
// exp(i Q) for Hermitian traceless Q by the Cayley-Hamilton theorem: exp(iQ) = f0 + f1 Q + f2 Q^2.
// Small Q (c1 = Tr Q^2 / 2 < 1/4): the power series with Q^3 = c1 Q + c0 reducing every power.
// Otherwise: the closed form of Morningstar & Peardon, Phys. Rev. D 69 (2004) 054501.
// ------------------------------------------------------------------------------------------------
// series cut-off per real type: a term below it no longer changes the sum
template <typename T> struct ExpiCut;
template <> struct ExpiCut<double> { static constexpr double v = 1e-18; };
template <> struct ExpiCut<float> { static constexpr float v = 1e-9f; };

template <typename T>
__device__ __forceinline__ void expi_coeffs(T c0, T c1, cplx<T> f[3]) {
    if (c1 < T(0.25)) {
        // f_k = sum_n (i^n / n!) {a_n, b_n, c_n}_k with Q^n = a_n I + b_n Q + c_n Q^2.  The eigenvalues of
        // Q are below sqrt(4 c1 / 3) < 1 in modulus, so |a_n| + |b_n| + |c_n| bounds the size of Q^n and the
        // sum stops once a term falls below the cut-off; 1/n! are compile-time constants (no division)
        T fr0 = 0, fr1 = 0, fr2 = 0, fi0 = 0, fi1 = 0, fi2 = 0;
        T a = 1, b = 0, c = 0;
        T inv = 1;   // 1/n!
#pragma unroll
        for (int n = 0; n < 26; n++) {
            const T sa = inv * a, sb = inv * b, sc = inv * c;
            switch (n & 3) {   // i^n = 1, i, -1, -i
                case 0: fr0 += sa; fr1 += sb; fr2 += sc; break;
                case 1: fi0 += sa; fi1 += sb; fi2 += sc; break;
                case 2: fr0 -= sa; fr1 -= sb; fr2 -= sc; break;
                default: fi0 -= sa; fi1 -= sb; fi2 -= sc; break;
            }
            if (n >= 3 && (fabs(sa) + fabs(sb) + fabs(sc)) < ExpiCut<T>::v) break;
            const T an = c0 * c, bn = fma(c1, c, a), cn = b;
            a = an; b = bn; c = cn;
            inv *= T(1.0 / (double)(n + 1));
        }
        f[0] = cmk(fr0, fi0); f[1] = cmk(fr1, fi1); f[2] = cmk(fr2, fi2);
        return;
    }
    const bool neg = c0 < T(0);
    const T c0p = fabs(c0);
    const T c0max = T(2) * pow(c1 / T(3), T(1.5));
    const T ratio = fmin(T(1), c0p / c0max);
    const T theta = acos(ratio);
    const T u = sqrt(c1 / T(3)) * cos(theta / T(3));
    const T w = sqrt(c1) * sin(theta / T(3));
    const T u2 = u * u, w2 = w * w;
    const T xi0 = fabs(w) < T(0.05) ? T(1) - w2 / T(6) * (T(1) - w2 / T(20) * (T(1) - w2 / T(42))) : sin(w) / w;
    const T cw = cos(w);
    const cplx<T> e2iu = cmk(cos(T(2) * u), sin(T(2) * u));
    const cplx<T> emiu = cmk(cos(u), -sin(u));
    const cplx<T> h0 = cadd(cscale(e2iu, u2 - w2), cmul(emiu, cmk(T(8) * u2 * cw, T(2) * u * (T(3) * u2 + w2) * xi0)));
    const cplx<T> h1 = csub(cscale(e2iu, T(2) * u), cmul(emiu, cmk(T(2) * u * cw, -(T(3) * u2 - w2) * xi0)));
    const cplx<T> h2 = csub(e2iu, cmul(emiu, cmk(cw, T(3) * u * xi0)));
    const T den = T(1) / (T(9) * u2 - w2);
    f[0] = cscale(h0, den);
    f[1] = cscale(h1, den);
    f[2] = cscale(h2, den);
    if (neg) {   // f_j(-c0) = (-1)^j conj(f_j(c0))
        f[0] = cconj(f[0]);
        f[1] = cscale(cconj(f[1]), T(-1));
        f[2] = cconj(f[2]);
    }
}

// exp(i Q) for Q Hermitian traceless given in the compact form (3 real diagonal, 3 complex upper entries):
// Q^2 is Hermitian too, c1 = Tr Q^2 / 2 and c0 = det Q (= Tr Q^3 / 3) come from the entries directly
template <typename T>
__device__ __forceinline__ mat3<T> expi(const herm<T>& Q) {
    const T d0 = Q.d[0], d1 = Q.d[1], d2 = Q.d[2];
    const cplx<T> q01 = Q.o[0], q02 = Q.o[1], q12 = Q.o[2];
    const T n01 = q01.re * q01.re + q01.im * q01.im;
    const T n02 = q02.re * q02.re + q02.im * q02.im;
    const T n12 = q12.re * q12.re + q12.im * q12.im;
    herm<T> Q2;
    Q2.d[0] = d0 * d0 + n01 + n02;
    Q2.d[1] = d1 * d1 + n01 + n12;
    Q2.d[2] = d2 * d2 + n02 + n12;
    Q2.o[0] = cfma(q02, cconj(q12), cscale(q01, d0 + d1));   // Q01 (d0 + d1) + Q02 Q21
    Q2.o[1] = cfma(q01, q12, cscale(q02, d0 + d2));          // Q02 (d0 + d2) + Q01 Q12
    Q2.o[2] = cfma(cconj(q01), q02, cscale(q12, d1 + d2));   // Q12 (d1 + d2) + Q10 Q02
    const T c1 = T(0.5) * (Q2.d[0] + Q2.d[1] + Q2.d[2]);
    const cplx<T> t = cmul(q01, q12);                        // Q01 Q12 Q20 = t conj(Q02)
    const T c0 = d0 * d1 * d2 + T(2) * (t.re * q02.re + t.im * q02.im) - d0 * n12 - d1 * n02 - d2 * n01;
    cplx<T> f[3];
    expi_coeffs<T>(c0, c1, f);
    const mat3<T> Qf = herm_full(Q), Q2f = herm_full(Q2);
    mat3<T> E;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cplx<T> v = cadd(cmul(f[1], Qf.e[i][j]), cmul(f[2], Q2f.e[i][j]));
            if (i == j) v = cadd(v, f[0]);
            E.e[i][j] = v;
        }
    return E;
}

// Gram-Schmidt on the first two rows, third row = conj(row0 x row1)
__device__ __forceinline__ void reunitarise(mat3<double>& U) {
    double n0 = 0.0;
#pragma unroll
    for (int j = 0; j < 3; j++) n0 += U.e[0][j].re * U.e[0][j].re + U.e[0][j].im * U.e[0][j].im;
    n0 = rsqrt(n0);
#pragma unroll
    for (int j = 0; j < 3; j++) U.e[0][j] = cscale(U.e[0][j], n0);
    cplx<double> p = cmk(0.0, 0.0);   // <row0, row1>
#pragma unroll
    for (int j = 0; j < 3; j++) p = ccfma(U.e[0][j], U.e[1][j], p);
#pragma unroll
    for (int j = 0; j < 3; j++) U.e[1][j] = csub(U.e[1][j], cmul(p, U.e[0][j]));
    double n1 = 0.0;
#pragma unroll
    for (int j = 0; j < 3; j++) n1 += U.e[1][j].re * U.e[1][j].re + U.e[1][j].im * U.e[1][j].im;
    n1 = rsqrt(n1);
#pragma unroll
    for (int j = 0; j < 3; j++) U.e[1][j] = cscale(U.e[1][j], n1);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        U.e[2][j] = cconj(csub(cmul(U.e[0][j1], U.e[1][j2]), cmul(U.e[0][j2], U.e[1][j1])));
    }
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    if (!(v == v)) v = INFINITY;   // NaN counts as divergence
    atomicMax((unsigned long long*)addr, (unsigned long long)__double_as_longlong(v));
}

// Uout = exp(i eps V) Uin per link (canonical layouts).  Optionally: reunitarise, write the internal
// copies, and record max |Uout - Wold| (max over all entries) into *maxdiff.
__global__ void __launch_bounds__(kBlock) k_link_update(const double* __restrict__ Uin, const double* __restrict__ V,
                                                        double eps, int reunit, double* __restrict__ Uout,
                                                        const double* __restrict__ Wold, double* maxdiff,
                                                        double2* u64, float4* u32a, float2* u32b, int nsite) {
    // one thread per link, links of a site adjacent: a warp reads 32 consecutive 144-byte link records
    const int lk = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = lk >> 2, mu = lk & 3;
    double diff = 0.0;
    if (s < nsite) {
        const size_t l = (size_t)s * 4 + mu;
        double v[8];
        load8(V + l * 8, v);
#pragma unroll
        for (int a = 0; a < 8; a++) v[a] *= eps;
        herm<double> Q = coef_to_herm2(v);   // 2 eps V
#pragma unroll
        for (int k = 0; k < 3; k++) { Q.d[k] *= 0.5; Q.o[k] = cscale(Q.o[k], 0.5); }
        const mat3<double> E = expi<double>(Q);
        mat3<double> U;
        const double2* src = reinterpret_cast<const double2*>(Uin + l * 18);
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) { const double2 z = src[3 * i + j]; U.e[i][j] = cmk(z.x, z.y); }
        mat3<double> R = m_mul(E, U);
        if (reunit) reunitarise(R);
        double2* dst = reinterpret_cast<double2*>(Uout + l * 18);
        const double2* old = Wold ? reinterpret_cast<const double2*>(Wold + l * 18) : nullptr;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const double2 z = make_double2(R.e[i][j].re, R.e[i][j].im);
                if (old) {
                    const double2 o = old[3 * i + j];
                    diff = fmax(diff, fmax(fabs(z.x - o.x), fabs(z.y - o.y)));
                }
                dst[3 * i + j] = z;
                if (u64) u64[(size_t)(mu * 9 + 3 * i + j) * nsite + s] = z;
            }
        if (u32a) {
            u32a[(size_t)(mu * 3 + 0) * nsite + s] = make_float4(R.e[0][0].re, R.e[0][0].im, R.e[0][1].re, R.e[0][1].im);
            u32a[(size_t)(mu * 3 + 1) * nsite + s] = make_float4(R.e[0][2].re, R.e[0][2].im, R.e[1][0].re, R.e[1][0].im);
            u32a[(size_t)(mu * 3 + 2) * nsite + s] = make_float4(R.e[1][1].re, R.e[1][1].im, R.e[1][2].re, R.e[1][2].im);
#pragma unroll
            for (int j = 0; j < 3; j++) u32b[(size_t)(mu * 3 + j) * nsite + s] = make_float2(R.e[2][j].re, R.e[2][j].im);
        }
    }
    if (maxdiff) {
        __shared__ double sh[kBlock / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) diff = fmax(diff, __shfl_down_sync(0xffffffffu, diff, o));
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = diff;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int w = 0; w < kBlock / 32; w++) m = fmax(m, sh[w]);
            atomic_max_nonneg(maxdiff, m);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// The same update in float-float arithmetic (df.cuh): exp(i Q) by the Cayley-Hamilton power series (the
// branch expi takes for c1 = Tr Q^2 / 2 < 1/4, which covers every MD step), the product with U and the
// reunitarisation, all to ~2^-48 relative, at a fraction of the float64 cost.  Links with c1 >= 0.24 (a
// rotation by more than about half a radian) take the float64 path of k_link_update.
// ------------------------------------------------------------------------------------------------
// 1/n! as float pairs (hi = the nearest float, lo = the nearest float to the remainder)
#define RM_DFC(x) {(float)(x), (float)((x) - (double)(float)(x))}
__constant__ float2 kInvFactorialDF[26] = {
    RM_DFC(1.0), RM_DFC(1.0), RM_DFC(1.0 / 2), RM_DFC(1.0 / 6),
    RM_DFC(1.0 / 24), RM_DFC(1.0 / 120), RM_DFC(1.0 / 720), RM_DFC(1.0 / 5040),
    RM_DFC(1.0 / 40320), RM_DFC(1.0 / 362880), RM_DFC(1.0 / 3628800.0), RM_DFC(1.0 / 39916800.0),
    RM_DFC(1.0 / 479001600.0), RM_DFC(1.0 / 6227020800.0), RM_DFC(1.0 / 87178291200.0), RM_DFC(1.0 / 1307674368000.0),
    RM_DFC(1.0 / 20922789888000.0), RM_DFC(1.0 / 355687428096000.0), RM_DFC(1.0 / 6402373705728000.0), RM_DFC(1.0 / 121645100408832000.0),
    RM_DFC(1.0 / 2432902008176640000.0), RM_DFC(1.0 / 51090942171709440000.0), RM_DFC(1.0 / 1124000727777607680000.0), RM_DFC(1.0 / 25852016738884976640000.0),
    RM_DFC(1.0 / 620448401733239439360000.0), RM_DFC(1.0 / 15511210043330985984000000.0),
};
#undef RM_DFC

struct hermdf { dfl d[3]; cdfl o[3]; };   // d: diagonal, o: 01, 02, 12

__device__ __forceinline__ cdfl hdf_entry(const hermdf& h, int i, int j) {
    if (i == j) return cdf_make(h.d[i], df_zero());
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    const int idx = lo == 0 ? (hi == 1 ? 0 : 1) : 2;
    return i < j ? h.o[idx] : cdf_conj(h.o[idx]);
}

// R = exp(i Q) U in float-float, Q = eps V (V: 8 coefficients and U already split into float pairs), optionally
// reunitarised
__device__ __forceinline__ void link_update_df(const dfl (&v)[8], dfl eps, const cdfl (&Ud)[3][3], bool reunit,
                                               cdfl (&R)[3][3]) {
    // Q = eps sum_a v_a T^a: diagonal (v3 + v8/sqrt3, -v3 + v8/sqrt3, -2 v8/sqrt3)/2, off-diagonal (v1 - i v2)/2, ...
    constexpr double kR3 = 0.57735026918962576451;   // 1/sqrt(3), split at compile time
    const dfl r3 = df_make((float)kR3, (float)(kR3 - (double)(float)kR3));
    const dfl he = df_make(0.5f * eps.hi, 0.5f * eps.lo);
    const dfl w8 = df_mul(v[7], r3);
    hermdf Q;
    Q.d[0] = df_mul(he, df_add(v[2], w8));
    Q.d[1] = df_mul(he, df_sub(w8, v[2]));
    Q.d[2] = df_neg(df_mul(eps, w8));
    Q.o[0] = cdf_make(df_mul(he, v[0]), df_neg(df_mul(he, v[1])));
    Q.o[1] = cdf_make(df_mul(he, v[3]), df_neg(df_mul(he, v[4])));
    Q.o[2] = cdf_make(df_mul(he, v[5]), df_neg(df_mul(he, v[6])));
    // Q^2 (Hermitian), c1 = Tr Q^2 / 2, c0 = det Q
    const dfl n01 = cdf_norm(Q.o[0]), n02 = cdf_norm(Q.o[1]), n12 = cdf_norm(Q.o[2]);
    hermdf Q2;
    Q2.d[0] = df_add(df_mul(Q.d[0], Q.d[0]), df_add(n01, n02));
    Q2.d[1] = df_add(df_mul(Q.d[1], Q.d[1]), df_add(n01, n12));
    Q2.d[2] = df_add(df_mul(Q.d[2], Q.d[2]), df_add(n02, n12));
    Q2.o[0] = cdf_add(cdf_scale(Q.o[0], df_add(Q.d[0], Q.d[1])), cdf_mul(Q.o[1], cdf_conj(Q.o[2])));
    Q2.o[1] = cdf_add(cdf_scale(Q.o[1], df_add(Q.d[0], Q.d[2])), cdf_mul(Q.o[0], Q.o[2]));
    Q2.o[2] = cdf_add(cdf_scale(Q.o[2], df_add(Q.d[1], Q.d[2])), cdf_mul(cdf_conj(Q.o[0]), Q.o[1]));
    const dfl c1 = df_mulf(df_add(df_add(Q2.d[0], Q2.d[1]), Q2.d[2]), 0.5f);
    const cdfl t = cdf_mul(Q.o[0], Q.o[2]);   // Q01 Q12; Q01 Q12 Q20 = t conj(Q02)
    dfl c0 = df_mul(df_mul(Q.d[0], Q.d[1]), Q.d[2]);
    c0 = df_add(c0, df_mulf(df_add(df_mul(t.re, Q.o[1].re), df_mul(t.im, Q.o[1].im)), 2.f));
    c0 = df_sub(c0, df_add(df_add(df_mul(Q.d[0], n12), df_mul(Q.d[1], n02)), df_mul(Q.d[2], n01)));
    // f_k = sum_n (i^n / n!) {a_n, b_n, c_n}_k, Q^n = a_n + b_n Q + c_n Q^2, Q^3 = c1 Q + c0
    dfl fr[3] = {df_zero(), df_zero(), df_zero()}, fi[3] = {df_zero(), df_zero(), df_zero()};
    dfl a = df_make(1.f, 0.f), b = df_zero(), c = df_zero();
    for (int n = 0; n < 26; n++) {
        const float2 fz = kInvFactorialDF[n];
        const dfl inv = df_make(fz.x, fz.y);
        const dfl sa = df_mul(inv, a), sb = df_mul(inv, b), sc = df_mul(inv, c);
        const int ph = n & 3;   // i^n = 1, i, -1, -i
        if (ph == 0) { fr[0] = df_add(fr[0], sa); fr[1] = df_add(fr[1], sb); fr[2] = df_add(fr[2], sc); }
        else if (ph == 1) { fi[0] = df_add(fi[0], sa); fi[1] = df_add(fi[1], sb); fi[2] = df_add(fi[2], sc); }
        else if (ph == 2) { fr[0] = df_sub(fr[0], sa); fr[1] = df_sub(fr[1], sb); fr[2] = df_sub(fr[2], sc); }
        else { fi[0] = df_sub(fi[0], sa); fi[1] = df_sub(fi[1], sb); fi[2] = df_sub(fi[2], sc); }
        if (n >= 3 && fabsf(sa.hi) + fabsf(sb.hi) + fabsf(sc.hi) < 1e-18f) break;
        const dfl an = df_mul(c0, c), bn = df_add(df_mul(c1, c), a);
        c = b; a = an; b = bn;
    }
    const cdfl f0 = cdf_make(fr[0], fi[0]), f1 = cdf_make(fr[1], fi[1]), f2 = cdf_make(fr[2], fi[2]);
    // E = f0 + f1 Q + f2 Q^2, R = E U
    cdfl E[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cdfl e = cdf_add(cdf_mul(f1, hdf_entry(Q, i, j)), cdf_mul(f2, hdf_entry(Q2, i, j)));
            if (i == j) e = cdf_add(e, f0);
            E[i][j] = e;
        }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cdfl s = cdf_mul(E[i][0], Ud[0][j]);
            s = cdf_add(s, cdf_mul(E[i][1], Ud[1][j]));
            s = cdf_add(s, cdf_mul(E[i][2], Ud[2][j]));
            R[i][j] = s;
        }
    if (!reunit) return;
    // Gram-Schmidt on the first two rows, third row = conj(row0 x row1)
    dfl nn = df_add(df_add(cdf_norm(R[0][0]), cdf_norm(R[0][1])), cdf_norm(R[0][2]));
    dfl sc0 = df_rsqrt(nn);
#pragma unroll
    for (int j = 0; j < 3; j++) R[0][j] = cdf_scale(R[0][j], sc0);
    cdfl p = cdf_make(df_zero(), df_zero());   // <row0, row1>
#pragma unroll
    for (int j = 0; j < 3; j++) p = cdf_add(p, cdf_mul(cdf_conj(R[0][j]), R[1][j]));
#pragma unroll
    for (int j = 0; j < 3; j++) R[1][j] = cdf_sub(R[1][j], cdf_mul(p, R[0][j]));
    nn = df_add(df_add(cdf_norm(R[1][0]), cdf_norm(R[1][1])), cdf_norm(R[1][2]));
    sc0 = df_rsqrt(nn);
#pragma unroll
    for (int j = 0; j < 3; j++) R[1][j] = cdf_scale(R[1][j], sc0);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        R[2][j] = cdf_conj(cdf_sub(cdf_mul(R[0][j1], R[1][j2]), cdf_mul(R[0][j2], R[1][j1])));
    }
}

__global__ void __launch_bounds__(kBlock) k_link_update_ff(const double* __restrict__ Uin, const double* __restrict__ V,
                                                           double eps, int reunit, double* __restrict__ Uout,
                                                           const double* __restrict__ Wold, double* maxdiff,
                                                           double2* u64, float4* u32a, float2* u32b, int nsite) {
    const int lk = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = lk >> 2, mu = lk & 3;
    double diff = 0.0;
    float diff32 = 0.f;   // the float-float branch's max |W_new - W_old|, from the float pairs
    if (s < nsite) {
        const size_t l = (size_t)s * 4 + mu;
        double v[8];
        load8(V + l * 8, v);
        // inputs split into float pairs by integer operations: the float-float branch runs no float64
        // arithmetic except one addition per output value
        dfl vs[8];
        float vv = 0.f;
#pragma unroll
        for (int a = 0; a < 8; a++) {
            vs[a] = df_split(v[a]);
            vv = fmaf(vs[a].hi, vs[a].hi, vv);
        }
        const dfl es = df_split(eps);
        // c1 = Tr Q^2 / 2 = eps^2 |v|^2 / 4 decides the branch
        const float c1 = 0.25f * es.hi * es.hi * vv;
        const double2* src = reinterpret_cast<const double2*>(Uin + l * 18);
        double2* dst = reinterpret_cast<double2*>(Uout + l * 18);
        const double2* old = Wold ? reinterpret_cast<const double2*>(Wold + l * 18) : nullptr;
        if (c1 < 0.24f) {
            cdfl Ud[3][3], R[3][3];
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const double2 z = src[3 * i + j];
                    Ud[i][j] = cdf_make(df_split(z.x), df_split(z.y));
                }
            link_update_df(vs, es, Ud, reunit != 0, R);
            float rf[3][3][2];   // nearest float32 of each entry
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const cdfl r = R[i][j];
                    if (old) {
                        const double2 o = old[3 * i + j];
                        const dfl ore = df_split(o.x), oim = df_split(o.y);
                        const float dr = __fadd_rn(__fsub_rn(r.re.hi, ore.hi), __fsub_rn(r.re.lo, ore.lo));
                        const float di = __fadd_rn(__fsub_rn(r.im.hi, oim.hi), __fsub_rn(r.im.lo, oim.lo));
                        diff32 = fmaxf(diff32, fmaxf(fabsf(dr), fabsf(di)));
                    }
                    const double2 z = make_double2(df_join(r.re), df_join(r.im));
                    dst[3 * i + j] = z;
                    if (u64) u64[(size_t)(mu * 9 + 3 * i + j) * nsite + s] = z;
                    rf[i][j][0] = __fadd_rn(r.re.hi, r.re.lo);
                    rf[i][j][1] = __fadd_rn(r.im.hi, r.im.lo);
                }
            if (u32a) {
                u32a[(size_t)(mu * 3 + 0) * nsite + s] = make_float4(rf[0][0][0], rf[0][0][1], rf[0][1][0], rf[0][1][1]);
                u32a[(size_t)(mu * 3 + 1) * nsite + s] = make_float4(rf[0][2][0], rf[0][2][1], rf[1][0][0], rf[1][0][1]);
                u32a[(size_t)(mu * 3 + 2) * nsite + s] = make_float4(rf[1][1][0], rf[1][1][1], rf[1][2][0], rf[1][2][1]);
#pragma unroll
                for (int j = 0; j < 3; j++) u32b[(size_t)(mu * 3 + j) * nsite + s] = make_float2(rf[2][j][0], rf[2][j][1]);
            }
        } else {
            mat3<double> U;
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) { const double2 z = src[3 * i + j]; U.e[i][j] = cmk(z.x, z.y); }
            double w[8];
#pragma unroll
            for (int a = 0; a < 8; a++) w[a] = v[a] * eps;
            herm<double> Q = coef_to_herm2(w);
#pragma unroll
            for (int k = 0; k < 3; k++) { Q.d[k] *= 0.5; Q.o[k] = cscale(Q.o[k], 0.5); }
            mat3<double> Rd = m_mul(expi<double>(Q), U);
            if (reunit) reunitarise(Rd);
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const double2 z = make_double2(Rd.e[i][j].re, Rd.e[i][j].im);
                    if (old) {
                        const double2 o = old[3 * i + j];
                        diff = fmax(diff, fmax(fabs(z.x - o.x), fabs(z.y - o.y)));
                    }
                    dst[3 * i + j] = z;
                    if (u64) u64[(size_t)(mu * 9 + 3 * i + j) * nsite + s] = z;
                }
            if (u32a) {
                u32a[(size_t)(mu * 3 + 0) * nsite + s] = make_float4(Rd.e[0][0].re, Rd.e[0][0].im, Rd.e[0][1].re, Rd.e[0][1].im);
                u32a[(size_t)(mu * 3 + 1) * nsite + s] = make_float4(Rd.e[0][2].re, Rd.e[0][2].im, Rd.e[1][0].re, Rd.e[1][0].im);
                u32a[(size_t)(mu * 3 + 2) * nsite + s] = make_float4(Rd.e[1][1].re, Rd.e[1][1].im, Rd.e[1][2].re, Rd.e[1][2].im);
#pragma unroll
                for (int j = 0; j < 3; j++) u32b[(size_t)(mu * 3 + j) * nsite + s] = make_float2(Rd.e[2][j].re, Rd.e[2][j].im);
            }
        }
    }
    diff = fmax(diff, (double)diff32);
    if (maxdiff) {
        __shared__ double sh[kBlock / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) diff = fmax(diff, __shfl_down_sync(0xffffffffu, diff, o));
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = diff;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int w = 0; w < kBlock / 32; w++) m = fmax(m, sh[w]);
            atomic_max_nonneg(maxdiff, m);
        }
    }
}

// One iterate of the link fixed point of the mixed-precision MD: W = exp(i eps V) B in float32 (B and V
// float64, rounded on load).  Writes the float32 internal link copies (read by the float32 Krylov runs and
// the float32 gauge force) and the compact iterate W32 [V][4][18] in place; with have_old, records
// max |W_new - W_old| into *maxdiff.  Only the accepted iterate is recomputed in float64.
__global__ void __launch_bounds__(kBlock) k_link_iter32(const double* __restrict__ B, const double* __restrict__ V,
                                                        float eps, float* __restrict__ W32, int have_old,
                                                        double* maxdiff, float4* u32a, float2* u32b, int nsite) {
    const int lk = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = lk >> 2, mu = lk & 3;
    float diff = 0.f;
    if (s < nsite) {
        const size_t l = (size_t)s * 4 + mu;
        double vd[8];
        load8(V + l * 8, vd);
        float v[8];
#pragma unroll
        for (int a = 0; a < 8; a++) v[a] = (float)vd[a] * eps;
        herm<float> Q = coef_to_herm2(v);   // 2 eps V
#pragma unroll
        for (int k = 0; k < 3; k++) { Q.d[k] *= 0.5f; Q.o[k] = cscale(Q.o[k], 0.5f); }
        const mat3<float> E = expi<float>(Q);
        mat3<float> Bf;
        const double2* src = reinterpret_cast<const double2*>(B + l * 18);
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) { const double2 z = src[3 * i + j]; Bf.e[i][j] = cmk((float)z.x, (float)z.y); }
        const mat3<float> R = m_mul(E, Bf);
        float2* w = reinterpret_cast<float2*>(W32 + l * 18);
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                if (have_old) {
                    const float2 o = w[3 * i + j];
                    diff = fmaxf(diff, fmaxf(fabsf(R.e[i][j].re - o.x), fabsf(R.e[i][j].im - o.y)));
                }
                w[3 * i + j] = make_float2(R.e[i][j].re, R.e[i][j].im);
            }
        u32a[(size_t)(mu * 3 + 0) * nsite + s] = make_float4(R.e[0][0].re, R.e[0][0].im, R.e[0][1].re, R.e[0][1].im);
        u32a[(size_t)(mu * 3 + 1) * nsite + s] = make_float4(R.e[0][2].re, R.e[0][2].im, R.e[1][0].re, R.e[1][0].im);
        u32a[(size_t)(mu * 3 + 2) * nsite + s] = make_float4(R.e[1][1].re, R.e[1][1].im, R.e[1][2].re, R.e[1][2].im);
#pragma unroll
        for (int j = 0; j < 3; j++) u32b[(size_t)(mu * 3 + j) * nsite + s] = make_float2(R.e[2][j].re, R.e[2][j].im);
    }
    if (maxdiff) {
        __shared__ float sh[kBlock / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) diff = fmaxf(diff, __shfl_down_sync(0xffffffffu, diff, o));
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = diff;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = 0.f;
            for (int k = 0; k < kBlock / 32; k++) m = fmaxf(m, sh[k]);
            atomic_max_nonneg(maxdiff, (double)m);
        }
    }
}

// Qn = P + h (F1 + F2); maxdiff = max |Qn - Qold|; Qn may alias Qold
__global__ void k_mom_update(const double* __restrict__ P, double h, const double* __restrict__ F1,
                             const double* __restrict__ F2, const double* Qold, double* Qn, size_t n, double* maxdiff) {
    double diff = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double q = P[i] + h * (F1[i] + (F2 ? F2[i] : 0.0));
        if (Qold) diff = fmax(diff, fabs(q - Qold[i]));
        Qn[i] = q;
    }
    if (maxdiff) {
        __shared__ double sh[kBlock / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) diff = fmax(diff, __shfl_down_sync(0xffffffffu, diff, o));
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = diff;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int w = 0; w < kBlock / 32; w++) m = fmax(m, sh[w]);
            atomic_max_nonneg(maxdiff, m);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Exactly symplectic form of Sec. 3's implicit leapfrog (rmhmc_params.symplectic): the generalised leapfrog
// is symplectic Euler followed by its adjoint, and on the group each half is the discrete Legendre
// transform of the discrete Lagrangian h L(U, xi), exp(i h xi) = U_{k+1} U_k^{-1}.  The momenta then pass
// through the right-trivialised derivative of the exponential, dexp_X = sum_n ad_X^n / (n+1)!, per link, with
// ad_X Y = coefficients of i[X.T, Y.T] = -f_abc X_a Y_b e_c (f the totally antisymmetric su(3)
// structure constants).  The identity term is added in float64; the series terms are summed in TC
// (float64 on the float64 path, float32 on the mixed one, where they are a correction of relative
// size |X| to momenta whose forces are float32 already).
// ------------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void ad_su3(const T (&X)[8], const T (&Y)[8], T (&Z)[8]) {
    constexpr int tr[9][3] = {{0, 1, 2}, {0, 3, 6}, {0, 4, 5}, {1, 3, 5}, {1, 4, 6},
                              {2, 3, 4}, {2, 5, 6}, {3, 4, 7}, {5, 6, 7}};
    constexpr double fv[9] = {1.0, 0.5, -0.5, 0.5, 0.5, 0.5, -0.5, 0.86602540378443864676, 0.86602540378443864676};
#pragma unroll
    for (int c = 0; c < 8; c++) Z[c] = T(0);
#pragma unroll
    for (int t = 0; t < 9; t++) {
        const int i = tr[t][0], j = tr[t][1], k = tr[t][2];
        const T v = (T)fv[t];
        Z[k] -= v * (X[i] * Y[j] - X[j] * Y[i]);
        Z[i] -= v * (X[j] * Y[k] - X[k] * Y[j]);
        Z[j] -= v * (X[k] * Y[i] - X[i] * Y[k]);
    }
}

// S = sum_{n>=1} ad_X^n Y / (n+1)!  (dexp_X Y = Y + S); the terms fall at least as |X|^n/(n+1)!
template <typename T>
__device__ __forceinline__ void dexp_tail(const T (&X)[8], const T (&Y)[8], T (&S)[8]) {
    T t[8], u[8];
    T ymax = T(0);
#pragma unroll
    for (int a = 0; a < 8; a++) { t[a] = Y[a]; S[a] = T(0); ymax = fmax(ymax, fabs(Y[a])); }
    const T stop = ymax * (sizeof(T) == 8 ? T(1e-18) : T(1e-9));
    for (int n = 1; n <= 40; n++) {
        ad_su3(X, t, u);
        T mx = T(0);
#pragma unroll
        for (int a = 0; a < 8; a++) { t[a] = u[a] / T(n + 1); S[a] += t[a]; mx = fmax(mx, fabs(t[a])); }
        if (mx <= stop) break;
    }
}

// S = sum_{n>=1} (B_n / n!) ad_X^n Y, Bernoulli numbers B_n (z/(e^z - 1) = sum B_n z^n / n!), to n = 16:
// dexp^{-1}_X Y = Y + S up to (|ad_X|/2 pi)^18
__constant__ double kBernoulliOverFactorial[17] = {
    1.0, -0.5, 1.0 / 12.0, 0.0, -1.0 / 720.0, 0.0, 1.0 / 30240.0, 0.0, -1.0 / 1209600.0, 0.0, 1.0 / 47900160.0, 0.0,
    -691.0 / 1307674368000.0, 0.0, 1.0 / 74724249600.0, 0.0, -3617.0 / 10670622842880000.0};

template <typename T>
__device__ __forceinline__ void dexpinv_tail(const T (&X)[8], const T (&Y)[8], T (&S)[8]) {
    const double* bn = kBernoulliOverFactorial;
    T w[8], u[8];
#pragma unroll
    for (int a = 0; a < 8; a++) { w[a] = Y[a]; S[a] = T(0); }
#pragma unroll 1
    for (int n = 1; n <= 16; n++) {
        ad_su3(X, w, u);
#pragma unroll
        for (int a = 0; a < 8; a++) { w[a] = u[a]; S[a] += T(bn[n]) * w[a]; }
    }
}

// Per link (thread per link of [V][4][8] coefficient fields), X = h V:
//   inverse = 0:  out = dexp_X (Y + h (F1 + F2))
//   inverse = 1:  out = dexp^{-1}_{-X} Y + h (F1 + F2)   (Bernoulli series plus residual corrections)
// F1, F2 may be null.  With Qold, max |out - Qold| goes to *maxdiff; |X| > 4 (the step turns a link
// by more than 4 radians: the Bernoulli series needs |ad_X| < 2 pi) writes NaN and reports divergence.
template <typename TC>
__global__ void __launch_bounds__(kBlock) k_mom_dexp(int inverse, const double* __restrict__ Y, double h,
                                                     const double* __restrict__ F1, const double* __restrict__ F2,
                                                     const double* __restrict__ V, const double* Qold, double* out,
                                                     size_t nlink, double* maxdiff) {
    double diff = 0.0;
    for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < nlink; l += (size_t)gridDim.x * blockDim.x) {
        const size_t o = l * 8;
        double y[8], f[8], r[8];
        TC x[8], yc[8], s[8];
        double xx = 0.0;
#pragma unroll
        for (int a = 0; a < 8; a++) {
            const double xa = (inverse ? -h : h) * V[o + a];
            xx += xa * xa;
            x[a] = (TC)xa;
            f[a] = h * ((F1 ? F1[o + a] : 0.0) + (F2 ? F2[o + a] : 0.0));
            y[a] = inverse ? Y[o + a] : Y[o + a] + f[a];
            yc[a] = (TC)y[a];
        }
        if (!inverse) {
            dexp_tail(x, yc, s);
#pragma unroll
            for (int a = 0; a < 8; a++) r[a] = y[a] + (double)s[a];
        } else {
            // z = y + d with d = B(y) - y (B the truncated Bernoulli series), then refinements
            // d += B(y - dexp(z)), y - dexp(z) = -(d + dexp_tail(z)), each gaining (|ad_X| / 2 pi)^17
            TC d[8], z[8], t[8], rr[8], b[8];
            dexpinv_tail(x, yc, d);
            TC ymax = TC(0);
#pragma unroll
            for (int a = 0; a < 8; a++) ymax = fmax(ymax, fabs(yc[a]));
            const TC stop = ymax * (sizeof(TC) == 8 ? TC(1e-17) : TC(1e-8));
#pragma unroll 1
            for (int it = 0; it < 8; it++) {
#pragma unroll
                for (int a = 0; a < 8; a++) z[a] = yc[a] + d[a];
                dexp_tail(x, z, t);
#pragma unroll
                for (int a = 0; a < 8; a++) rr[a] = -(d[a] + t[a]);
                dexpinv_tail(x, rr, b);
                TC mx = TC(0);
#pragma unroll
                for (int a = 0; a < 8; a++) { const TC c = rr[a] + b[a]; d[a] += c; mx = fmax(mx, fabs(c)); }
                if (mx <= stop) break;
            }
#pragma unroll
            for (int a = 0; a < 8; a++) r[a] = y[a] + (double)d[a] + f[a];
        }
        const bool bad = xx > 16.0;
#pragma unroll
        for (int a = 0; a < 8; a++) {
            if (bad) r[a] = __longlong_as_double(0x7ff8000000000000LL);
            if (Qold) diff = fmax(diff, bad ? INFINITY : fabs(r[a] - Qold[o + a]));
        }
#pragma unroll
        for (int a = 0; a < 8; a++) out[o + a] = r[a];
    }
    if (maxdiff) {
        __shared__ double sh[kBlock / 32];
#pragma unroll
        for (int w = 16; w > 0; w >>= 1) diff = fmax(diff, __shfl_down_sync(0xffffffffu, diff, w));
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = diff;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int w = 0; w < kBlock / 32; w++) m = fmax(m, sh[w]);
            atomic_max_nonneg(maxdiff, m);
        }
    }
}

__global__ void k_gauss_field(double* __restrict__ out, int V, uint64_t seed, uint32_t stream, uint32_t tag) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    double* dst = out + (size_t)s * 32;
    for (int k = 0; k < 16; k++) {
        u32x4 c{{(uint32_t)k, (uint32_t)s, stream, tag}};
        const u32x4 w = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        const double u0 = u53(w.v[0], w.v[1]), u1 = u53(w.v[2], w.v[3]);
        const double r = sqrt(-2.0 * log(u0));
        double sn, cs;
        sincospi(2.0 * u1, &sn, &cs);
        dst[2 * k] = r * cs;
        dst[2 * k + 1] = r * sn;
    }
}

// ------------------------------------------------------------------------------------------------
// host driver
// ------------------------------------------------------------------------------------------------
int link_update_launch(rmhmc_ctx* ctx, const double* Uin, const double* V, double eps, bool reunit, double* Uout,
                       const double* Wold, double* dmax, bool internal, bool ff, cudaStream_t st) {
    const int grid = lane_blocks(ctx);   // 4 V threads
    if (ff && ctx->link_update_ff)
        k_link_update_ff<<<grid, kBlock, 0, st>>>(Uin, V, eps, reunit ? 1 : 0, Uout, Wold, dmax,
                                                  internal ? ctx->u64 : nullptr, internal ? ctx->u32a : nullptr,
                                                  internal ? ctx->u32b : nullptr, ctx->g.V);
    else
        k_link_update<<<grid, kBlock, 0, st>>>(Uin, V, eps, reunit ? 1 : 0, Uout, Wold, dmax, internal ? ctx->u64 : nullptr,
                                               internal ? ctx->u32a : nullptr, internal ? ctx->u32b : nullptr, ctx->g.V);
    ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    if (internal) {
        ctx->links_valid = true;
        ctx->link_gen++;
    }
    return RMHMC_OK;
}

// float32 iterates of the link fixed point need a tolerance above float32 resolution of the O(1) link
// entries (their rounding noise is ~1e-7); tighter tolerances iterate in float64
constexpr double kIter32MinTol = 1e-6;
static bool link_iterates_fp32(const rmhmc_params* p) { return p->prec != RMHMC_FP64 && p->fp_tol >= kIter32MinTol; }

static int link_iter32_launch(rmhmc_ctx* ctx, const double* B, const double* V, double eps, float* W32, bool have_old,
                              double* dmax, cudaStream_t st) {
    const int grid = lane_blocks(ctx);   // 4 V threads
    k_link_iter32<<<grid, kBlock, 0, st>>>(B, V, (float)eps, W32, have_old ? 1 : 0, dmax, ctx->u32a, ctx->u32b, ctx->g.V);
    ++ctx->launches;
    ctx->link_gen++;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}

static int mom_update(rmhmc_ctx* ctx, const double* P, double h, const double* F1, const double* F2, const double* Qold,
                      double* Qn, double* dmax, cudaStream_t st) {
    const size_t n = field_elems(ctx);
    const int grid = (int)std::min<size_t>((n + kBlock - 1) / kBlock, (size_t)ctx->num_sms * 8);
    k_mom_update<<<grid, kBlock, 0, st>>>(P, h, F1, F2, Qold, Qn, n, dmax); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}

static int mom_dexp(rmhmc_ctx* ctx, int prec, bool inverse, const double* Y, double h, const double* F1,
                    const double* F2, const double* V, const double* Qold, double* out, double* dmax, cudaStream_t st) {
    const size_t nl = (size_t)ctx->g.V * 4;
    const int grid = (int)std::min<size_t>((nl + kBlock - 1) / kBlock, (size_t)ctx->num_sms * 8);
    if (prec == RMHMC_FP64)
        k_mom_dexp<double><<<grid, kBlock, 0, st>>>(inverse ? 1 : 0, Y, h, F1, F2, V, Qold, out, nl, dmax);
    else
        k_mom_dexp<float><<<grid, kBlock, 0, st>>>(inverse ? 1 : 0, Y, h, F1, F2, V, Qold, out, nl, dmax);
    ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}

struct MDWork {
    double *FG, *FK, *V0, *Q, *B, *W, *dmax;
    double* Ph;   // the symplectic step's momenta after its first half (dexp^{-1}_{-X1} mu)
    float* W32;   // float32 iterate of the link fixed point (mixed precision)
};

static int md_work(rmhmc_ctx* ctx, MDWork& w) {
    int status = RMHMC_OK;
    const size_t fs = field_elems(ctx), ls = (size_t)ctx->g.V * 72;
    w.FG = (double*)workspace(ctx, "md_fg", sizeof(double) * fs, &status);
    w.FK = (double*)workspace(ctx, "md_fk", sizeof(double) * fs, &status);
    w.V0 = (double*)workspace(ctx, "md_v0", sizeof(double) * fs, &status);
    w.Q = (double*)workspace(ctx, "md_q", sizeof(double) * fs, &status);
    w.B = (double*)workspace(ctx, "md_b", sizeof(double) * ls, &status);
    w.W = (double*)workspace(ctx, "md_w", sizeof(double) * ls, &status);
    w.dmax = (double*)workspace(ctx, "md_dmax", 64, &status);
    w.W32 = (float*)workspace(ctx, "md_w32", sizeof(float) * (size_t)ctx->g.V * 72, &status);
    w.Ph = (double*)workspace(ctx, "md_ph", sizeof(double) * fs, &status);
    if (!w.FG || !w.FK || !w.V0 || !w.Q || !w.B || !w.W || !w.dmax || !w.W32 || !w.Ph) return status;
    return RMHMC_OK;
}

static int read_max(rmhmc_ctx* ctx, double* dmax, double* out, cudaStream_t st) {
    RM_TRY(fetch(ctx, dmax, out, 1, st));
    return RMHMC_OK;
}

static int check_params(rmhmc_ctx* ctx, const rmhmc_params* p) {
    if (!p) return set_err(ctx, RMHMC_EINVAL, "null parameters");
    if (p->nsteps < 1 || !(p->tau > 0.0)) return set_err(ctx, RMHMC_EINVAL, "need tau > 0 and nsteps >= 1");
    if (!(p->tol_md > 0.0) || !(p->tol_h > 0.0) || !(p->fp_tol > 0.0) || p->fp_maxit < 1 || p->maxiter < 1)
        return set_err(ctx, RMHMC_EINVAL, "tolerances and iteration caps must be positive");
    if (p->prec != RMHMC_FP64 && p->prec != RMHMC_MIXED) return set_err(ctx, RMHMC_EINVAL, "bad prec");
    if (p->symplectic != 0 && p->symplectic != 1) return set_err(ctx, RMHMC_EINVAL, "symplectic must be 0 or 1");
    if (p->fg_fp64 != 0 && p->fg_fp64 != 1) return set_err(ctx, RMHMC_EINVAL, "fg_fp64 must be 0 or 1");
    if (p->fp_extra < 0 || p->fp_extra >= p->fp_maxit)
        return set_err(ctx, RMHMC_EINVAL, "fp_extra must lie in [0, fp_maxit)");
    return RMHMC_OK;
}

// precision of the gauge force inside the MD (the float64 MD is float64 throughout)
static int md_gauge_prec(const rmhmc_params* p) {
    return (p->prec == RMHMC_FP64 || p->fg_fp64) ? RMHMC_FP64 : RMHMC_FP32;
}

// The log|M| term of Eq. (5) through an auxiliary field: phi (fixed in the MD) with action
// 1/2 <phi, M phi> = 1/2 |Q phi|^2, Q = 1/R as a partial fraction (inv); its force is the kinetic force of phi
// under Q and joins the gauge force as part of the U-only potential force.
struct AuxTerm {
    const double* phi = nullptr;
    MassTerm inv;
    double* FA = nullptr;   // scratch force
    double* VA = nullptr;   // scratch velocity (the captured kinetic evaluation writes one)
};

// F = F_G(U) (+ F_aux(U) with an auxiliary field) at the context's links
static int potential_force(rmhmc_ctx* ctx, const rmhmc_params* p, int gprec, const AuxTerm* lg, double* F,
                           cudaStream_t st) {
    RM_TRY(gauge_force_launch(ctx, p->beta, p->c1, gprec, F, st));
    if (!lg) return RMHMC_OK;
    int it = 0;
    RM_TRY(kinetic_from_krylov(ctx, lg->inv, lg->phi, p->tol_md, p->maxiter, p->prec, lg->FA, nullptr, nullptr, &it, st));
    return axpby64(ctx, 1.0, F, 1.0, lg->FA, F, field_elems(ctx), st);
}

// MD on (U, P) in place.  U canonical device links; the context's links follow U.
static int md_run(rmhmc_ctx* ctx, double* U, double* P, const rmhmc_params* p, const MassTerm& m, rmhmc_result* r,
                  cudaStream_t st, const AuxTerm* lg = nullptr) {
    MDWork w;
    RM_TRY(md_work(ctx, w));
    const size_t fs = field_elems(ctx), lb = sizeof(double) * (size_t)ctx->g.V * 72;
    const double eps = p->tau / p->nsteps;
    const int gprec = md_gauge_prec(p);
    const bool ff = p->prec == RMHMC_MIXED;   // float-float link updates in mixed precision only
    int fp_p = 0, fp_u = 0, solves = 0;
    long long kiters = 0;
    double worst = 0.0;
    RM_TRY(import_links(ctx, U, st));
    RM_TRY(potential_force(ctx, p, gprec, lg, w.FG, st));
    RM_TRY(mom_update(ctx, P, 0.5 * eps, w.FG, nullptr, nullptr, w.Q, nullptr, st));   // Q0 = P + eps/2 F_G
    for (int step = 0; step < p->nsteps; step++) {
        // (1) momentum fixed point at fixed U; extra: iterations still to run after convergence (-1: not
        // converged yet)
        bool conv = false;
        int extra = -1;
        for (int i = 0; i < p->fp_maxit; i++) {
            int it = 0;
            RM_TRY(kinetic_from_krylov(ctx, m, w.Q, p->tol_md, p->maxiter, p->prec, w.FK, w.V0, nullptr, &it, st));
            solves++;
            kiters += it;
            RM_CHECK(ctx, cudaMemsetAsync(w.dmax, 0, sizeof(double), st));
            if (p->symplectic) RM_TRY(mom_dexp(ctx, p->prec, false, P, 0.5 * eps, w.FG, w.FK, w.V0, w.Q, w.Q, w.dmax, st));
            else RM_TRY(mom_update(ctx, P, 0.5 * eps, w.FG, w.FK, w.Q, w.Q, w.dmax, st));
            double d = 0.0;
            RM_TRY(read_max(ctx, w.dmax, &d, st));
            fp_p++;
            if (!isfinite(d)) return set_err(ctx, RMHMC_ENAN, "NaN/Inf in the momentum fixed point");
            if (extra < 0 && d <= p->fp_tol) { extra = p->fp_extra; worst = std::max(worst, d); }
            if (extra == 0) { conv = true; break; }
            if (extra > 0) extra--;
        }
        if (!conv) return set_err(ctx, RMHMC_ENOCONV, "momentum fixed point: no convergence in %d iterations", p->fp_maxit);
        // (2) link fixed point: B = exp(i eps/2 V0) U ; W = exp(i eps V0) U ; W <- exp(i eps/2 V(W)) B.
        // float64: every iterate in float64.  Mixed (fp_tol >= 1e-6): the iterates (which only feed the
        // float32 Krylov runs and the convergence test) in float32; the accepted one,
        // exp(i eps/2 V(W_i)) B, in float64.
        const bool it32 = link_iterates_fp32(p);
        // symplectic: P_h = dexp^{-1}_{-X1} mu (X1 = eps/2 V0); the link loop then also iterates mu2 = dexp_{X2} P_h
        if (p->symplectic) RM_TRY(mom_dexp(ctx, p->prec, true, w.Q, 0.5 * eps, nullptr, nullptr, w.V0, nullptr, w.Ph, nullptr, st));
        RM_TRY(link_update_launch(ctx, U, w.V0, 0.5 * eps, false, w.B, nullptr, nullptr, false, ff, st));
        if (it32) RM_TRY(link_iter32_launch(ctx, U, w.V0, eps, w.W32, false, nullptr, st));
        else RM_TRY(link_update_launch(ctx, U, w.V0, eps, false, w.W, nullptr, nullptr, true, ff, st));
        conv = false;
        extra = -1;
        for (int i = 0; i < p->fp_maxit; i++) {
            int it = 0;
            RM_TRY(kinetic_from_krylov(ctx, m, w.Q, p->tol_md, p->maxiter, p->prec, w.FK, w.V0, nullptr, &it, st));
            solves++;
            kiters += it;
            RM_CHECK(ctx, cudaMemsetAsync(w.dmax, 0, sizeof(double), st));
            // W_{i+1} (float64: into U's buffer, U is no longer needed as B holds exp(i eps/2 V0) U)
            if (it32) RM_TRY(link_iter32_launch(ctx, w.B, w.V0, 0.5 * eps, w.W32, true, w.dmax, st));
            else RM_TRY(link_update_launch(ctx, w.B, w.V0, 0.5 * eps, false, U, w.W, w.dmax, true, ff, st));
            if (p->symplectic) RM_TRY(mom_dexp(ctx, p->prec, false, w.Ph, 0.5 * eps, nullptr, nullptr, w.V0, w.Q, w.Q, w.dmax, st));
            double d = 0.0;
            RM_TRY(read_max(ctx, w.dmax, &d, st));
            fp_u++;
            if (!isfinite(d)) return set_err(ctx, RMHMC_ENAN, "NaN/Inf in the link fixed point");
            if (!it32) RM_CHECK(ctx, cudaMemcpyAsync(w.W, U, lb, cudaMemcpyDeviceToDevice, st));
            if (extra < 0 && d <= p->fp_tol) { extra = p->fp_extra; worst = std::max(worst, d); }
            if (extra == 0) { conv = true; break; }
            if (extra > 0) extra--;
        }
        if (!conv) return set_err(ctx, RMHMC_ENOCONV, "link fixed point: no convergence in %d iterations", p->fp_maxit);
        // the accepted links, reunitarised, with fresh internal copies
        if (it32) RM_TRY(link_update_launch(ctx, w.B, w.V0, 0.5 * eps, true, U, nullptr, nullptr, true, ff, st));
        else RM_TRY(link_update_launch(ctx, w.W, w.V0, 0.0, true, U, nullptr, nullptr, true, ff, st));
        // (3) explicit half step with F_K(W_i, P') kept from the last iteration
        RM_TRY(potential_force(ctx, p, gprec, lg, w.FG, st));
        if (p->symplectic) RM_TRY(mom_dexp(ctx, p->prec, true, w.Q, 0.5 * eps, w.FG, w.FK, w.V0, nullptr, P, nullptr, st));
        else RM_TRY(mom_update(ctx, w.Q, 0.5 * eps, w.FG, w.FK, nullptr, P, nullptr, st));
        RM_TRY(mom_update(ctx, P, 0.5 * eps, w.FG, w.FK, nullptr, w.Q, nullptr, st));   // next initial guess
    }
    if (r) {
        r->md_solves = solves;
        r->md_iters = kiters;
        r->fp_iters_p = fp_p;
        r->fp_iters_u = fp_u;
        r->max_fp_change = worst;
    }
    (void)fs;
    return RMHMC_OK;
}

// ------------------------------------------------------------------------------------------------
// the molecular dynamics as one CUDA graph (mixed precision): the fixed points and the Krylov runs are
// conditional WHILE nodes whose conditions the kernels set on the device, so a whole MD trajectory is one
// graph launch with no host round trip.  Status codes written on the device: 1 Krylov cap, 2 Krylov NaN,
// 3 fixed point without convergence, 4 fixed point NaN.
// ------------------------------------------------------------------------------------------------
// iter[0]: iterations of this fixed point; iter[1]: iterations still to run after convergence (-1 before it)
__global__ void k_fp_decide(double* dmax, int* iter, int cap, double tol, int extra, cudaGraphConditionalHandle h,
                            long long* count, int* status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double d = *dmax;
    const int it = ++iter[0];
    (*count)++;
    const bool bad = !(d == d) || isinf(d);
    int rem = iter[1];
    if (rem < 0 && d <= tol) rem = extra;
    const bool done = rem == 0;
    if (rem > 0) rem--;
    iter[1] = rem;
    if (bad) atomicMax(status, 4);
    else if (!done && it >= cap) atomicMax(status, 3);
    cudaGraphSetConditional(h, (!done && !bad && it < cap) ? 1u : 0u);
    *dmax = 0.0;
}

struct MDGraphBufs {
    double *U, *P;               // the trajectory's links and momenta (context-owned copies)
    long long* stats;            // [0] Krylov iterations, [1] momentum fixed-point iterations, [2] link ones
    int* ints;                   // [0] status, [1] loop iteration counter, [2] iterations left after convergence
};

static int md_graph_bufs(rmhmc_ctx* ctx, MDGraphBufs& b) {
    int status = RMHMC_OK;
    const size_t fs = field_elems(ctx), ls = (size_t)ctx->g.V * 72;
    b.U = (double*)workspace(ctx, "mg_u", sizeof(double) * ls, &status);
    b.P = (double*)workspace(ctx, "mg_p", sizeof(double) * fs, &status);
    void* st = workspace(ctx, "mg_stats", 256, &status);
    if (!b.U || !b.P || !st) return status;
    b.stats = (long long*)st;
    b.ints = (int*)((char*)st + 128);
    return RMHMC_OK;
}

// a captured trajectory is reused while the parameters, the mass term and the pinned kernel shapes are the same
static std::string md_key(const rmhmc_ctx* ctx, const rmhmc_params* p, const MassTerm& m) {
    char buf[512];
    snprintf(buf, sizeof buf, "%d|%.17g|%.17g|%.17g|%d|%.17g|%.17g|%d|%d|%d|%d|%.17g|%d|%d", p->prec, p->beta, p->c1,
             p->tau, p->nsteps, p->tol_md, p->fp_tol, p->fp_maxit, p->fp_extra, md_gauge_prec(p), p->maxiter, m.c,
             m.npole(), ctx->shape_gen);
    std::string k(buf);
    for (int j = 0; j < m.npole(); j++) {
        snprintf(buf, sizeof buf, "|%.17g,%.17g", m.alpha[j], m.sigma[j]);
        k += buf;
    }
    return k;
}

static int md_graph_capture(rmhmc_ctx* ctx, const rmhmc_params* p, const MassTerm& m, const MDGraphBufs& gb,
                            const MDWork& w, const AuxTerm* lg, cudaGraph_t* out) {
    cudaStream_t st = ctx->cap_st[0], aux = ctx->cap_st[1], aux2 = ctx->cap_st[2];
    const double eps = p->tau / p->nsteps;
    const int gprec = md_gauge_prec(p);
    const bool ff = p->prec == RMHMC_MIXED;
    RM_CHECK(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    int s = RMHMC_OK;
    do {
        // U-only potential force: gauge force, plus the auxiliary-field force as one more captured kinetic
        // evaluation (its Krylov iterations count with the MD's)
        auto potential = [&]() -> int {
            RM_TRY(gauge_force_launch(ctx, p->beta, p->c1, gprec, w.FG, st));
            if (!lg) return RMHMC_OK;
            RM_TRY(kinetic_enqueue(ctx, lg->inv, lg->phi, p->tol_md, p->maxiter, lg->FA, lg->VA, gb.stats, gb.ints,
                                   st, aux2));
            return axpby64(ctx, 1.0, w.FG, 1.0, lg->FA, w.FG, field_elems(ctx), st);
        };
        if ((s = import_links(ctx, gb.U, st)) != RMHMC_OK) break;
        if ((s = potential()) != RMHMC_OK) break;
        if ((s = mom_update(ctx, gb.P, 0.5 * eps, w.FG, nullptr, nullptr, w.Q, nullptr, st)) != RMHMC_OK) break;
        for (int step = 0; step < p->nsteps && s == RMHMC_OK; step++) {
            // (1) momentum fixed point
            if (cudaMemsetAsync(w.dmax, 0, sizeof(double), st) != cudaSuccess ||
                cudaMemsetAsync(gb.ints + 1, 0, sizeof(int), st) != cudaSuccess ||
                cudaMemsetAsync(gb.ints + 2, 0xff, sizeof(int), st) != cudaSuccess) { s = RMHMC_ECUDA; break; }
            cudaGraphConditionalHandle h1;
            cudaGraph_t body;
            if ((s = capture_handle(ctx, st, 1u, &h1)) != RMHMC_OK) break;
            if ((s = capture_while(ctx, st, h1, &body)) != RMHMC_OK) break;
            if (cudaStreamBeginCaptureToGraph(aux, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                s = RMHMC_ECUDA;
                break;
            }
            s = kinetic_enqueue(ctx, m, w.Q, p->tol_md, p->maxiter, w.FK, w.V0, gb.stats, gb.ints, aux, aux2);
            if (s == RMHMC_OK) s = mom_update(ctx, gb.P, 0.5 * eps, w.FG, w.FK, w.Q, w.Q, w.dmax, aux);
            if (s == RMHMC_OK) {
                k_fp_decide<<<1, 32, 0, aux>>>(w.dmax, gb.ints + 1, p->fp_maxit, p->fp_tol, p->fp_extra, h1, gb.stats + 1,
                                                gb.ints);
                ++ctx->launches;
            }
            {
                cudaGraph_t tmp;
                if (cudaStreamEndCapture(aux, &tmp) != cudaSuccess && s == RMHMC_OK) s = RMHMC_ECUDA;
            }
            if (s != RMHMC_OK) break;
            // (2) link fixed point (float32 iterates and the accepted one in float64, or float64 iterates)
            const bool it32 = link_iterates_fp32(p);
            if ((s = link_update_launch(ctx, gb.U, w.V0, 0.5 * eps, false, w.B, nullptr, nullptr, false, ff, st)) != RMHMC_OK) break;
            if (it32) s = link_iter32_launch(ctx, gb.U, w.V0, eps, w.W32, false, nullptr, st);
            else s = link_update_launch(ctx, gb.U, w.V0, eps, false, w.W, nullptr, nullptr, true, ff, st);
            if (s != RMHMC_OK) break;
            if (cudaMemsetAsync(w.dmax, 0, sizeof(double), st) != cudaSuccess ||
                cudaMemsetAsync(gb.ints + 1, 0, sizeof(int), st) != cudaSuccess ||
                cudaMemsetAsync(gb.ints + 2, 0xff, sizeof(int), st) != cudaSuccess) { s = RMHMC_ECUDA; break; }
            cudaGraphConditionalHandle h2;
            if ((s = capture_handle(ctx, st, 1u, &h2)) != RMHMC_OK) break;
            if ((s = capture_while(ctx, st, h2, &body)) != RMHMC_OK) break;
            if (cudaStreamBeginCaptureToGraph(aux, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                s = RMHMC_ECUDA;
                break;
            }
            const size_t lb = sizeof(double) * (size_t)ctx->g.V * 72;
            s = kinetic_enqueue(ctx, m, w.Q, p->tol_md, p->maxiter, w.FK, w.V0, gb.stats, gb.ints, aux, aux2);
            if (s == RMHMC_OK && it32) s = link_iter32_launch(ctx, w.B, w.V0, 0.5 * eps, w.W32, true, w.dmax, aux);
            if (s == RMHMC_OK && !it32) {
                s = link_update_launch(ctx, w.B, w.V0, 0.5 * eps, false, gb.U, w.W, w.dmax, true, ff, aux);
                if (s == RMHMC_OK && cudaMemcpyAsync(w.W, gb.U, lb, cudaMemcpyDeviceToDevice, aux) != cudaSuccess)
                    s = RMHMC_ECUDA;
            }
            if (s == RMHMC_OK) {
                k_fp_decide<<<1, 32, 0, aux>>>(w.dmax, gb.ints + 1, p->fp_maxit, p->fp_tol, p->fp_extra, h2, gb.stats + 2,
                                                gb.ints);
                ++ctx->launches;
            }
            {
                cudaGraph_t tmp;
                if (cudaStreamEndCapture(aux, &tmp) != cudaSuccess && s == RMHMC_OK) s = RMHMC_ECUDA;
            }
            if (s != RMHMC_OK) break;
            // the accepted links in float64, reunitarised; (3) explicit half step, next initial guess
            if (it32) s = link_update_launch(ctx, w.B, w.V0, 0.5 * eps, true, gb.U, nullptr, nullptr, true, ff, st);
            else s = link_update_launch(ctx, w.W, w.V0, 0.0, true, gb.U, nullptr, nullptr, true, ff, st);
            if (s != RMHMC_OK) break;
            if ((s = potential()) != RMHMC_OK) break;
            if ((s = mom_update(ctx, w.Q, 0.5 * eps, w.FG, w.FK, nullptr, gb.P, nullptr, st)) != RMHMC_OK) break;
            if ((s = mom_update(ctx, gb.P, 0.5 * eps, w.FG, w.FK, nullptr, w.Q, nullptr, st)) != RMHMC_OK) break;
        }
    } while (0);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (s != RMHMC_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return s;
    }
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_check(ctx, e, "cudaStreamEndCapture");
    }
    *out = g;
    return RMHMC_OK;
}

// Runs the MD through the cached graph; returns RMHMC_OK, a status of the run, or a negative code of the
// capture (the caller then falls back to the host-driven path)
static int md_graph_run(rmhmc_ctx* ctx, double* U, double* P, const rmhmc_params* p, const MassTerm& m, rmhmc_result* r,
                        cudaStream_t stream, bool* used, const AuxTerm* lg = nullptr) {
    *used = false;
    if (!ctx->use_graphs || p->prec == RMHMC_FP64 || p->symplectic || m.npole() == 0 || 2 * m.npole() + 1 > 32)
        return RMHMC_OK;
    MDWork w;
    RM_TRY(md_work(ctx, w));
    MDGraphBufs gb;
    RM_TRY(md_graph_bufs(ctx, gb));
    RM_TRY(kinetic_graph_prepare(ctx, m, p->maxiter));
    if (lg) {
        if (lg->inv.npole() == 0 || 2 * lg->inv.npole() + 1 > 32) return RMHMC_OK;
        RM_TRY(kinetic_graph_prepare(ctx, lg->inv, p->maxiter));
    }
    for (int i = 0; i < 3; i++)
        if (!ctx->cap_st[i]) RM_CHECK(ctx, cudaStreamCreateWithFlags(&ctx->cap_st[i], cudaStreamNonBlocking));
    const std::string key = md_key(ctx, p, m) + (lg ? "|logdet" : "");
    if (!ctx->md_exec || ctx->md_key != key || ctx->md_gen != ctx->ws_gen) {
        if (ctx->md_exec) {
            cudaGraphExecDestroy(ctx->md_exec);
            ctx->md_exec = nullptr;
        }
        const long long saved = ctx->launches;
        cudaGraph_t g = nullptr;
        const int s = md_graph_capture(ctx, p, m, gb, w, lg, &g);
        ctx->launches = saved;
        if (s != RMHMC_OK) {
            ctx->graph_note = "capture failed: " + ctx->err;
            ctx->err.clear();
            ctx->use_graphs = false;
            return RMHMC_OK;
        }
        const cudaError_t e = cudaGraphInstantiate(&ctx->md_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->md_exec = nullptr;
            ctx->graph_note = std::string("instantiate failed: ") + cudaGetErrorString(e);
            ctx->use_graphs = false;
            return RMHMC_OK;
        }
        ctx->md_key = key;
        ctx->md_gen = ctx->ws_gen;
        ctx->graph_note = "md graph captured";
    }
    const size_t fs = field_elems(ctx), lb = sizeof(double) * (size_t)ctx->g.V * 72;
    RM_CHECK(ctx, cudaMemcpyAsync(gb.U, U, lb, cudaMemcpyDeviceToDevice, stream));
    RM_CHECK(ctx, cudaMemcpyAsync(gb.P, P, sizeof(double) * fs, cudaMemcpyDeviceToDevice, stream));
    RM_CHECK(ctx, cudaMemsetAsync(gb.stats, 0, 256, stream));
    RM_CHECK(ctx, cudaGraphLaunch(ctx->md_exec, stream));
    ctx->link_gen++;   // the graph's link updates changed the internal copies
    RM_CHECK(ctx, cudaMemcpyAsync(U, gb.U, lb, cudaMemcpyDeviceToDevice, stream));
    RM_CHECK(ctx, cudaMemcpyAsync(P, gb.P, sizeof(double) * fs, cudaMemcpyDeviceToDevice, stream));
    long long st[4];
    int ints[2];
    RM_CHECK(ctx, cudaMemcpyAsync(ctx->h_pinned, gb.stats, 128 + 8, cudaMemcpyDeviceToHost, stream));
    RM_CHECK(ctx, cudaStreamSynchronize(stream));
    memcpy(st, ctx->h_pinned, sizeof st);
    memcpy(ints, (char*)ctx->h_pinned + 128, sizeof ints);
    *used = true;
    // kernels the graph ran: 3 + 6 per step outside the loops, 8 per fixed-point iteration, 2 per Krylov iteration
    ctx->launches += 3 + 6LL * p->nsteps + 8 * (st[1] + st[2]) + 2 * st[0];
    ctx->krylov_iters += st[0];
    ctx->links_valid = true;
    if (r) {
        r->md_solves = (int)(st[1] + st[2]);
        r->md_iters = st[0];
        r->fp_iters_p = (int)st[1];
        r->fp_iters_u = (int)st[2];
        r->max_fp_change = 0.0;
    }
    switch (ints[0]) {
        case 0: return RMHMC_OK;
        case 1: return set_err(ctx, RMHMC_ENOCONV, "MD graph: a Krylov run hit its iteration cap");
        case 3: return set_err(ctx, RMHMC_ENOCONV, "MD graph: a fixed point did not converge in %d iterations", p->fp_maxit);
        default: return set_err(ctx, RMHMC_ENAN, "MD graph: NaN/Inf");
    }
}

// T = 1/2 |R(A) P|^2 with every shift at relative residual tol_h (float64 check), S, plaquette
static int hamiltonian_run(rmhmc_ctx* ctx, const double* U, const double* P, const rmhmc_params* p, const MassTerm& m,
                           double* H, double* T, double* S, double* plaq, cudaStream_t st) {
    int status = RMHMC_OK;
    const size_t fs = field_elems(ctx);
    RM_TRY(import_links(ctx, U, st));
    double* Y = (double*)workspace(ctx, "hm_y", sizeof(double) * fs, &status);
    if (!Y) return status;
    RM_TRY(rational_apply(ctx, m, P, p->tol_h, p->maxiter, p->prec, Y, nullptr, st));
    double y2 = 0.0, s = 0.0, pl = 0.0;
    RM_TRY(norm2_64(ctx, Y, fs, &y2, st));
    RM_TRY(action_launch(ctx, p->beta, p->c1, &s, &pl, st));
    const double t = 0.5 * y2;
    if (!isfinite(t) || !isfinite(s)) return set_err(ctx, RMHMC_ENAN, "NaN/Inf in the Hamiltonian");
    if (T) *T = t;
    if (S) *S = s;
    if (H) *H = t + s;
    if (plaq) *plaq = pl;
    return RMHMC_OK;
}

}  // namespace rm

using namespace rm;

extern "C" int rmhmc_gauss_field(rmhmc_ctx* ctx, double* out, uint64_t seed, uint32_t stream_id, uint32_t tag,
                                 cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (!out) return set_err(ctx, RMHMC_EINVAL, "rmhmc_gauss_field: null output");
    k_gauss_field<<<site_blocks(ctx), kBlock, 0, stream>>>(out, ctx->g.V, seed, stream_id, tag); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}

extern "C" int rmhmc_link_update(rmhmc_ctx* ctx, const double* U, const double* V, double eps, int reunit, double* Uout,
                                 cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (!U || !V || !Uout) return set_err(ctx, RMHMC_EINVAL, "rmhmc_link_update: null argument");
    return link_update_launch(ctx, U, V, eps, reunit != 0, Uout, nullptr, nullptr, false, true, stream);
}

extern "C" int rmhmc_hamiltonian(rmhmc_ctx* ctx, const double* U, const double* P, const rmhmc_params* p, double* H,
                                 double* T, double* S, cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (!U || !P) return set_err(ctx, RMHMC_EINVAL, "rmhmc_hamiltonian: null argument");
    RM_TRY(check_params(ctx, p));
    MassTerm m;
    RM_TRY(parse_mass(ctx, &p->mass, m));
    return hamiltonian_run(ctx, U, P, p, m, H, T, S, nullptr, stream);
}

extern "C" int rmhmc_md(rmhmc_ctx* ctx, double* U, double* P, const rmhmc_params* p, rmhmc_result* r,
                        cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (!U || !P) return set_err(ctx, RMHMC_EINVAL, "rmhmc_md: null argument");
    RM_TRY(check_params(ctx, p));
    MassTerm m;
    RM_TRY(parse_mass(ctx, &p->mass, m));
    if (r) memset(r, 0, sizeof *r);
    bool used = false;
    RM_TRY(md_graph_run(ctx, U, P, p, m, r, stream, &used));
    if (used) return RMHMC_OK;
    return md_run(ctx, U, P, p, m, r, stream);
}

extern "C" int rmhmc_trajectory(rmhmc_ctx* ctx, double* U, const double* xi, const rmhmc_params* p, rmhmc_result* r,
                                double* P_out, cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (!U) return set_err(ctx, RMHMC_EINVAL, "rmhmc_trajectory: null links");
    RM_TRY(check_params(ctx, p));
    MassTerm m;
    RM_TRY(parse_mass(ctx, &p->mass, m));
    rmhmc_result res;
    memset(&res, 0, sizeof res);
    int status = RMHMC_OK;
    const size_t fs = field_elems(ctx), lb = sizeof(double) * (size_t)ctx->g.V * 72;
    double* U0 = (double*)workspace(ctx, "tr_u0", lb, &status);
    double* P = (double*)workspace(ctx, "tr_p", sizeof(double) * fs, &status);
    double* X = (double*)workspace(ctx, "tr_xi", sizeof(double) * fs, &status);
    if (!U0 || !P || !X) return status;
    RM_CHECK(ctx, cudaMemcpyAsync(U0, U, lb, cudaMemcpyDeviceToDevice, stream));
    if (xi) {
        RM_CHECK(ctx, cudaMemcpyAsync(X, xi, sizeof(double) * fs, cudaMemcpyDeviceToDevice, stream));
    } else {
        k_gauss_field<<<site_blocks(ctx), kBlock, 0, stream>>>(X, ctx->g.V, p->seed, p->traj_index, 0u); ++ctx->launches;
        RM_LAUNCH_CHECK(ctx);
    }
    auto restore = [&](int code) {
        cudaMemcpyAsync(U, U0, lb, cudaMemcpyDeviceToDevice, stream);
        cudaStreamSynchronize(stream);
        ctx->links_valid = false;
        return code;
    };
    RM_TRY(import_links(ctx, U, stream));
    // the log|M| term: phi = R(A) eta with eta from Philox (tag 3), Q = 1/R as a partial fraction
    AuxTerm lgt;
    const AuxTerm* lg = nullptr;
    double* Yaux = nullptr;
    if (p->logdet) {
        if (m.npole() == 0) return set_err(ctx, RMHMC_EINVAL, "logdet needs a mass term with poles");
        double p1 = 0.0;
        RM_TRY(inverse_rational(ctx, m, lgt.inv, p1));
        if (p1 != 0.0) return set_err(ctx, RMHMC_EINVAL, "logdet needs c > 0 (1/R without a linear term)");
        double* phi = (double*)workspace(ctx, "lg_phi", sizeof(double) * fs, &status);
        double* eta = (double*)workspace(ctx, "lg_eta", sizeof(double) * fs, &status);
        lgt.FA = (double*)workspace(ctx, "lg_fa", sizeof(double) * fs, &status);
        lgt.VA = (double*)workspace(ctx, "lg_va", sizeof(double) * fs, &status);
        Yaux = (double*)workspace(ctx, "lg_y", sizeof(double) * fs, &status);
        if (!phi || !eta || !lgt.FA || !lgt.VA || !Yaux) return status;
        k_gauss_field<<<site_blocks(ctx), kBlock, 0, stream>>>(eta, ctx->g.V, p->seed, p->traj_index, 3u); ++ctx->launches;
        RM_LAUNCH_CHECK(ctx);
        int s0 = rational_apply(ctx, m, eta, p->tol_h, p->maxiter, p->prec, phi, nullptr, stream);
        if (s0 != RMHMC_OK) return restore(s0);
        lgt.phi = phi;
        lg = &lgt;
    }
    // auxiliary action 1/2 |Q phi|^2 at the context's links
    auto aux_action = [&](double* A) -> int {
        *A = 0.0;
        if (!lg) return RMHMC_OK;
        RM_TRY(rational_apply(ctx, lg->inv, lg->phi, p->tol_h, p->maxiter, p->prec, Yaux, nullptr, stream));
        double y2 = 0.0;
        RM_TRY(norm2_64(ctx, Yaux, fs, &y2, stream));
        *A = 0.5 * y2;
        return isfinite(*A) ? RMHMC_OK : set_err(ctx, RMHMC_ENAN, "NaN/Inf in the auxiliary action");
    };
    // the heatbath at the Hamiltonian's tolerance: mixed and float64 trajectories from the same noise then
    // start from the same momenta
    int s = heatbath_apply(ctx, m, X, p->tol_h, p->maxiter, p->prec, P, stream);
    if (s != RMHMC_OK) return restore(s);
    s = hamiltonian_run(ctx, U, P, p, m, &res.H0, &res.T0, &res.S0, nullptr, stream);
    if (s == RMHMC_OK) s = aux_action(&res.A0);
    if (s != RMHMC_OK) return restore(s);
    bool used = false;
    s = md_graph_run(ctx, U, P, p, m, &res, stream, &used, lg);
    if (s == RMHMC_OK && !used) s = md_run(ctx, U, P, p, m, &res, stream, lg);
    if (s != RMHMC_OK) return restore(s);
    s = hamiltonian_run(ctx, U, P, p, m, &res.H1, &res.T1, &res.S1, &res.plaq, stream);
    if (s == RMHMC_OK) s = aux_action(&res.A1);
    if (s != RMHMC_OK) return restore(s);
    res.H0 += res.A0;
    res.H1 += res.A1;
    res.dH = res.H1 - res.H0;
    res.u = philox_uniform(p->seed, p->traj_index, 1u);
    res.accepted = (!p->metropolis || res.dH <= 0.0 || res.u <= exp(-res.dH)) ? 1 : 0;
    if (P_out) RM_CHECK(ctx, cudaMemcpyAsync(P_out, P, sizeof(double) * fs, cudaMemcpyDeviceToDevice, stream));
    if (!res.accepted) {
        RM_CHECK(ctx, cudaMemcpyAsync(U, U0, lb, cudaMemcpyDeviceToDevice, stream));
        RM_TRY(import_links(ctx, U, stream));
        RM_TRY(action_launch(ctx, p->beta, p->c1, nullptr, &res.plaq, stream));
    }
    RM_CHECK(ctx, cudaStreamSynchronize(stream));
    if (r) *r = res;
    return RMHMC_OK;
}
