// Device SU(3) / su(3) algebra for the hot path (the links and su(3)-valued fields of Sec. 2),
// templated on the real type (float or double).
//
// su(3) elements travel as 8 coefficients p^a of P = sum_a p^a T^a, T^a = lambda^a / 2.  Inside the
// stencil they are expanded to a "doubled" Hermitian matrix 2P (3 real diagonal entries and the
// three complex entries above the diagonal); the factor 2 is folded back when projecting.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace rm {

template <typename T> struct cplx { T re, im; };
template <typename T> struct mat3 { cplx<T> e[3][3]; };
// Hermitian 3x3: d[k] = H_kk (real), o[0] = H_01, o[1] = H_02, o[2] = H_12
template <typename T> struct herm { T d[3]; cplx<T> o[3]; };

#define RM_HD __host__ __device__ __forceinline__

template <typename T> RM_HD cplx<T> cmk(T re, T im) { cplx<T> c; c.re = re; c.im = im; return c; }
template <typename T> RM_HD cplx<T> cconj(cplx<T> a) { return cmk(a.re, -a.im); }
template <typename T> RM_HD cplx<T> cadd(cplx<T> a, cplx<T> b) { return cmk(a.re + b.re, a.im + b.im); }
template <typename T> RM_HD cplx<T> csub(cplx<T> a, cplx<T> b) { return cmk(a.re - b.re, a.im - b.im); }
template <typename T> RM_HD cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return cmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// c + a*b
template <typename T> RM_HD cplx<T> cfma(cplx<T> a, cplx<T> b, cplx<T> c) {
    c.re = fma(a.re, b.re, c.re); c.re = fma(-a.im, b.im, c.re);
    c.im = fma(a.re, b.im, c.im); c.im = fma(a.im, b.re, c.im);
    return c;
}
// c + a*conj(b)
template <typename T> RM_HD cplx<T> cfmac(cplx<T> a, cplx<T> b, cplx<T> c) {
    c.re = fma(a.re, b.re, c.re); c.re = fma(a.im, b.im, c.re);
    c.im = fma(a.im, b.re, c.im); c.im = fma(-a.re, b.im, c.im);
    return c;
}
// c + conj(a)*b
template <typename T> RM_HD cplx<T> ccfma(cplx<T> a, cplx<T> b, cplx<T> c) {
    c.re = fma(a.re, b.re, c.re); c.re = fma(a.im, b.im, c.re);
    c.im = fma(a.re, b.im, c.im); c.im = fma(-a.im, b.re, c.im);
    return c;
}
template <typename T> RM_HD cplx<T> cscale(cplx<T> a, T s) { return cmk(a.re * s, a.im * s); }

template <typename T> RM_HD mat3<T> m_zero() {
    mat3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.e[i][j] = cmk<T>(0, 0);
    return r;
}
template <typename T> RM_HD mat3<T> m_unit() {
    mat3<T> r = m_zero<T>();
    r.e[0][0].re = r.e[1][1].re = r.e[2][2].re = T(1);
    return r;
}
template <typename T> RM_HD mat3<T> m_mul(const mat3<T>& a, const mat3<T>& b) {
    mat3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cplx<T> s = cmul(a.e[i][0], b.e[0][j]);
            s = cfma(a.e[i][1], b.e[1][j], s);
            s = cfma(a.e[i][2], b.e[2][j], s);
            r.e[i][j] = s;
        }
    return r;
}
// a * b^dag
template <typename T> RM_HD mat3<T> m_mul_nd(const mat3<T>& a, const mat3<T>& b) {
    mat3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cplx<T> s = cmk<T>(0, 0);
#pragma unroll
            for (int k = 0; k < 3; k++) s = cfmac(a.e[i][k], b.e[j][k], s);
            r.e[i][j] = s;
        }
    return r;
}
// a^dag * b
template <typename T> RM_HD mat3<T> m_mul_dn(const mat3<T>& a, const mat3<T>& b) {
    mat3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cplx<T> s = cmk<T>(0, 0);
#pragma unroll
            for (int k = 0; k < 3; k++) s = ccfma(a.e[k][i], b.e[k][j], s);
            r.e[i][j] = s;
        }
    return r;
}
template <typename T> RM_HD mat3<T> m_dag(const mat3<T>& a) {
    mat3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.e[i][j] = cconj(a.e[j][i]);
    return r;
}
template <typename T> RM_HD void m_acc(mat3<T>& a, const mat3<T>& b) {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) a.e[i][j] = cadd(a.e[i][j], b.e[i][j]);
}
template <typename T> RM_HD mat3<T> m_scale(const mat3<T>& a, T s) {
    mat3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.e[i][j] = cscale(a.e[i][j], s);
    return r;
}
template <typename T> RM_HD T re_trace(const mat3<T>& a) { return a.e[0][0].re + a.e[1][1].re + a.e[2][2].re; }

template <typename T> RM_HD herm<T> h_zero() {
    herm<T> h;
#pragma unroll
    for (int k = 0; k < 3; k++) { h.d[k] = T(0); h.o[k] = cmk<T>(0, 0); }
    return h;
}

// entry (l,k) of a Hermitian matrix stored as herm (l != k)
template <typename T> RM_HD cplx<T> h_off(const herm<T>& X, int l, int k) {
    // upper index: (0,1)->0, (0,2)->1, (1,2)->2
    const int lo = l < k ? l : k, hi = l < k ? k : l;
    const int idx = lo == 0 ? (hi == 1 ? 0 : 1) : 2;
    return l < k ? X.o[idx] : cconj(X.o[idx]);
}

// 2 X for X = sum_a x^a T^a
template <typename T> RM_HD herm<T> coef_to_herm2(const T* x) {
    const T r3 = T(0.57735026918962576451);   // 1/sqrt(3)
    herm<T> h;
    h.d[0] = x[2] + x[7] * r3;
    h.d[1] = -x[2] + x[7] * r3;
    h.d[2] = T(-2) * x[7] * r3;
    h.o[0] = cmk(x[0], -x[1]);
    h.o[1] = cmk(x[3], -x[4]);
    h.o[2] = cmk(x[5], -x[6]);
    return h;
}

// coefficients y^a = Tr(lambda^a Y) of Y given H = 2 Y (traceless part)
template <typename T> RM_HD void herm2_to_coef(const herm<T>& H, T* y) {
    const T r3h = T(0.28867513459481288225);  // 1/(2 sqrt 3)
    y[0] = H.o[0].re;
    y[1] = -H.o[0].im;
    y[2] = T(0.5) * (H.d[0] - H.d[1]);
    y[3] = H.o[1].re;
    y[4] = -H.o[1].im;
    y[5] = H.o[2].re;
    y[6] = -H.o[2].im;
    y[7] = (H.d[0] + H.d[1] - T(2) * H.d[2]) * r3h;
}

// acc += U X U^dag  (X Hermitian; only the Hermitian result's independent entries are formed)
template <typename T> __device__ __forceinline__ void acc_uxud(herm<T>& acc, const mat3<T>& U, const herm<T>& X) {
    cplx<T> W[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            cplx<T> w = cmk(U.e[i][k].re * X.d[k], U.e[i][k].im * X.d[k]);
#pragma unroll
            for (int l = 0; l < 3; l++)
                if (l != k) w = cfma(U.e[i][l], h_off(X, l, k), w);
            W[i][k] = w;
        }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        T d = acc.d[i];
#pragma unroll
        for (int k = 0; k < 3; k++) { d = fma(W[i][k].re, U.e[i][k].re, d); d = fma(W[i][k].im, U.e[i][k].im, d); }
        acc.d[i] = d;
    }
#pragma unroll
    for (int p = 0; p < 3; p++) {
        const int i = p == 2 ? 1 : 0, j = p == 0 ? 1 : 2;
        cplx<T> s = acc.o[p];
#pragma unroll
        for (int k = 0; k < 3; k++) s = cfmac(W[i][k], U.e[j][k], s);
        acc.o[p] = s;
    }
}

// acc += U^dag X U
template <typename T> __device__ __forceinline__ void acc_udxu(herm<T>& acc, const mat3<T>& U, const herm<T>& X) {
    // W = X U ; H = U^dag W, H_ij = sum_l conj(U_li) W_lj
    cplx<T> W[3][3];
#pragma unroll
    for (int l = 0; l < 3; l++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cplx<T> w = cmk(U.e[l][j].re * X.d[l], U.e[l][j].im * X.d[l]);
#pragma unroll
            for (int k = 0; k < 3; k++)
                if (k != l) w = cfma(h_off(X, l, k), U.e[k][j], w);
            W[l][j] = w;
        }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        T d = acc.d[i];
#pragma unroll
        for (int l = 0; l < 3; l++) { d = fma(U.e[l][i].re, W[l][i].re, d); d = fma(U.e[l][i].im, W[l][i].im, d); }
        acc.d[i] = d;
    }
#pragma unroll
    for (int p = 0; p < 3; p++) {
        const int i = p == 2 ? 1 : 0, j = p == 0 ? 1 : 2;
        cplx<T> s = acc.o[p];
#pragma unroll
        for (int l = 0; l < 3; l++) s = ccfma(U.e[l][i], W[l][j], s);
        acc.o[p] = s;
    }
}

// The same two conjugations with the result's third diagonal entry left out.  For a unitary V and a traceless
// Hermitian X, V X V^dag is traceless, so its entry (2,2) is -(H00 + H11) and the coefficients of the
// traceless part need only H00, H11 and the three upper entries (herm2_to_coef_tl).  Leaving out H22 drops
// row 2 of W = V X too: 108 instead of 144 FMA per conjugation.  U^dag X U is the same form with V = U^dag.
// acc.d[2] is not touched; read the sum with herm2_to_coef_tl.
template <typename T, bool DAG>
__device__ __forceinline__ void acc_conj_tl(herm<T>& acc, const mat3<T>& U, const herm<T>& X) {
    // V_ik = U_ik, or conj(U_ki) for DAG
    auto V = [&](int i, int k) { return DAG ? cconj(U.e[k][i]) : U.e[i][k]; };
    cplx<T> W[2][3];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const cplx<T> vik = V(i, k);
            cplx<T> w = cmk(vik.re * X.d[k], vik.im * X.d[k]);
#pragma unroll
            for (int l = 0; l < 3; l++)
                if (l != k) w = cfma(V(i, l), h_off(X, l, k), w);
            W[i][k] = w;
        }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        T d = acc.d[i];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const cplx<T> vik = V(i, k);
            d = fma(W[i][k].re, vik.re, d);
            d = fma(W[i][k].im, vik.im, d);
        }
        acc.d[i] = d;
    }
#pragma unroll
    for (int p = 0; p < 3; p++) {
        const int i = p == 2 ? 1 : 0, j = p == 0 ? 1 : 2;
        cplx<T> s = acc.o[p];
#pragma unroll
        for (int k = 0; k < 3; k++) s = cfmac(W[i][k], V(j, k), s);
        acc.o[p] = s;
    }
}
template <typename T> __device__ __forceinline__ void acc_uxud_tl(herm<T>& acc, const mat3<T>& U, const herm<T>& X) {
    acc_conj_tl<T, false>(acc, U, X);
}
template <typename T> __device__ __forceinline__ void acc_udxu_tl(herm<T>& acc, const mat3<T>& U, const herm<T>& X) {
    acc_conj_tl<T, true>(acc, U, X);
}
// herm2_to_coef of a traceless H from H00, H11 and the upper entries (H22 = -(H00 + H11))
template <typename T> RM_HD void herm2_to_coef_tl(const herm<T>& H, T* y) {
    const T r3t = T(0.86602540378443864676);  // 3 / (2 sqrt 3) = sqrt(3) / 2
    y[0] = H.o[0].re;
    y[1] = -H.o[0].im;
    y[2] = T(0.5) * (H.d[0] - H.d[1]);
    y[3] = H.o[1].re;
    y[4] = -H.o[1].im;
    y[5] = H.o[2].re;
    y[6] = -H.o[2].im;
    y[7] = (H.d[0] + H.d[1]) * r3t;
}

// full matrix of a Hermitian
template <typename T> RM_HD mat3<T> herm_full(const herm<T>& h) {
    mat3<T> m;
#pragma unroll
    for (int k = 0; k < 3; k++) m.e[k][k] = cmk(h.d[k], T(0));
    m.e[0][1] = h.o[0]; m.e[1][0] = cconj(h.o[0]);
    m.e[0][2] = h.o[1]; m.e[2][0] = cconj(h.o[1]);
    m.e[1][2] = h.o[2]; m.e[2][1] = cconj(h.o[2]);
    return m;
}

// coefficients k^a = Tr(lambda^a K) of the Hermitian K = -i M for an anti-Hermitian M
// (only the anti-Hermitian part of M is read:  K = -i (M - M^dag)/2)
template <typename T> RM_HD void antiherm_coef(const mat3<T>& M, T* k) {
    // K_ij = -i (M_ij - conj(M_ji)) / 2
    const T r3 = T(0.57735026918962576451);
    // diagonal: K_ii = Im M_ii
    T k0 = M.e[0][0].im, k1 = M.e[1][1].im, k2 = M.e[2][2].im;
    // K_01 = -i (M01 - conj M10)/2 ; (-i) z = (z.im, -z.re)
    cplx<T> a = cscale(csub(M.e[0][1], cconj(M.e[1][0])), T(0.5));
    cplx<T> b = cscale(csub(M.e[0][2], cconj(M.e[2][0])), T(0.5));
    cplx<T> c = cscale(csub(M.e[1][2], cconj(M.e[2][1])), T(0.5));
    cplx<T> K01 = cmk(a.im, -a.re), K02 = cmk(b.im, -b.re), K12 = cmk(c.im, -c.re);
    // Tr(lambda^a K): l1: 2Re K01, l2: -2 Im K01, l3: K00-K11, l4: 2Re K02, l5: -2Im K02,
    // l6: 2 Re K12, l7: -2 Im K12, l8: (K00+K11-2K22)/sqrt3
    k[0] = T(2) * K01.re; k[1] = T(-2) * K01.im; k[2] = k0 - k1;
    k[3] = T(2) * K02.re; k[4] = T(-2) * K02.im;
    k[5] = T(2) * K12.re; k[6] = T(-2) * K12.im;
    k[7] = (k0 + k1 - T(2) * k2) * r3;
}

}  // namespace rm

namespace rm {

// Adjoint matrix of a link: Ad[a][b] = 2 Tr(T^a U T^b U^dag), the real 8x8 orthogonal matrix with
// (U X U^dag)^a = sum_b Ad[a][b] x^b for X = sum_b x^b T^b (and (U^dag X U)^a = sum_b Ad[b][a] x^b).
// Built from the columns u_k of U: U lambda^b U^dag is a combination of the outer products
// p_kl = u_k u_l^dag (lambda^{1,2}: k,l = 0,1; lambda^{4,5}: 0,2; lambda^{6,7}: 1,2; lambda^{3,8}: p_kk),
// and Ad[a][b] = Tr(lambda^a U lambda^b U^dag) / 2 reads the Hermitian entries of that combination.
// The columns are handed to sink(b, col) one at a time (col[a] = Ad[a][b]), in the order 0, 1, 3, 4, 5, 6, 2, 7.
template <typename T, class Sink>
__device__ __forceinline__ void adjoint_columns(const mat3<T>& U, Sink&& sink) {
    const T r3 = T(0.57735026918962576451);   // 1/sqrt(3)
    // column b from the entries 00, 11, 22 (real) and 01, 02, 12 of the Hermitian M = U lambda^b U^dag
    auto put = [&](int b, T m00, T m11, T m22, cplx<T> m01, cplx<T> m02, cplx<T> m12) {
        const T col[8] = {m01.re, -m01.im, T(0.5) * (m00 - m11), m02.re, -m02.im, m12.re, -m12.im,
                          T(0.5) * r3 * (m00 + m11 - T(2) * m22)};
        sink(b, col);
    };
    // (k, l) pairs: S = p + p^dag (lambda^{1,4,6}), D = -i (p - p^dag) (lambda^{2,5,7})
    constexpr int pk[3] = {0, 0, 1}, pl[3] = {1, 2, 2}, pb[3] = {0, 3, 5};
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const int k = pk[q], l = pl[q];
        cplx<T> p[3][3];   // p[i][j] = U_ik conj(U_jl)
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) p[i][j] = cmul(U.e[i][k], cconj(U.e[j][l]));
        // S_ii = 2 Re p_ii, S_ij = p_ij + conj(p_ji); D_ii = 2 Im p_ii, D_ij = -i (p_ij - conj(p_ji))
        auto s_off = [&](int i, int j) { return cadd(p[i][j], cconj(p[j][i])); };
        auto d_off = [&](int i, int j) {
            const cplx<T> e = csub(p[i][j], cconj(p[j][i]));
            return cmk(e.im, -e.re);
        };
        put(pb[q], T(2) * p[0][0].re, T(2) * p[1][1].re, T(2) * p[2][2].re, s_off(0, 1), s_off(0, 2), s_off(1, 2));
        put(pb[q] + 1, T(2) * p[0][0].im, T(2) * p[1][1].im, T(2) * p[2][2].im, d_off(0, 1), d_off(0, 2), d_off(1, 2));
    }
    // g_k = u_k u_k^dag: lambda^3 -> g_0 - g_1, lambda^8 -> (g_0 + g_1 - 2 g_2)/sqrt(3)
    T gd[3][3];
    cplx<T> go[3][3];   // [k][01, 02, 12]
#pragma unroll
    for (int k = 0; k < 3; k++) {
#pragma unroll
        for (int i = 0; i < 3; i++) gd[k][i] = U.e[i][k].re * U.e[i][k].re + U.e[i][k].im * U.e[i][k].im;
        go[k][0] = cmul(U.e[0][k], cconj(U.e[1][k]));
        go[k][1] = cmul(U.e[0][k], cconj(U.e[2][k]));
        go[k][2] = cmul(U.e[1][k], cconj(U.e[2][k]));
    }
    put(2, gd[0][0] - gd[1][0], gd[0][1] - gd[1][1], gd[0][2] - gd[1][2], csub(go[0][0], go[1][0]),
        csub(go[0][1], go[1][1]), csub(go[0][2], go[1][2]));
    T d8[3];
    cplx<T> o8[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        d8[i] = r3 * (gd[0][i] + gd[1][i] - T(2) * gd[2][i]);
        o8[i] = cscale(csub(cadd(go[0][i], go[1][i]), cscale(go[2][i], T(2))), r3);
    }
    put(7, d8[0], d8[1], d8[2], o8[0], o8[1], o8[2]);
}

}  // namespace rm
