// The adjoint covariant hop sum of Sec. 2, Eq. (3) for one site and one field component mu:
//   acc = 2 * sum_nu [ U_nu(x) X_mu(x+nu) U_nu(x)^dag + U_nu(x-nu)^dag X_mu(x-nu) U_nu(x-nu) ]
// (the factor 2 comes from the doubled Hermitian expansion of the coefficients).
//
// Thread layout of every stencil kernel: four consecutive lanes own one site, lane & 3 = mu.  A warp
// therefore covers 8 consecutive sites; its loads of the 8 colour coefficients of X_mu at a neighbour
// are one contiguous 1 KB segment of the [V][4][8] field, and its link loads hit 8 consecutive entries
// of the structure-of-arrays link copy (the four lanes of a site read the same address).
#pragma once
#include "common.cuh"

namespace rm {

template <typename T> struct LinksOf;
template <> struct LinksOf<double> { using type = Links64; };
template <> struct LinksOf<float> { using type = Links32; };

template <typename T, int LF, class Src>
__device__ __forceinline__ void hop_sum1(const Geom& g, const typename LinksOf<T>::type& U, int s, int mu,
                                         const Src& src, herm<T>& acc) {
    int fwd[4], bwd[4];
    neighbours(g, s, fwd, bwd);
    acc = h_zero<T>();
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        T xf[8], xb[8];
        src(fwd[nu], mu, xf);
        src(bwd[nu], mu, xb);
        const mat3<T> uf = LinkLoad<T, LF>::load(U, s, nu);
        const mat3<T> ub = LinkLoad<T, LF>::load(U, bwd[nu], nu);
        acc_uxud(acc, uf, coef_to_herm2(xf));
        acc_udxu(acc, ub, coef_to_herm2(xb));
    }
}

// plain field source: X[s][mu][8]
template <typename T> struct SrcField {
    const T* X;
    __device__ __forceinline__ void operator()(int s, int mu, T* x) const { load8(X + (size_t)s * 32 + mu * 8, x); }
};

// fused source r + beta * p (conjugate-gradient search direction)
template <typename T> struct SrcAxpy {
    const T* r;
    const T* p;
    T beta;
    __device__ __forceinline__ void operator()(int s, int mu, T* x) const {
        load8(r + (size_t)s * 32 + mu * 8, x);
        if (p) {
            T y[8];
            load8(p + (size_t)s * 32 + mu * 8, y);
#pragma unroll
            for (int a = 0; a < 8; a++) x[a] = fma(beta, y[a], x[a]);
        }
    }
};

}  // namespace rm
