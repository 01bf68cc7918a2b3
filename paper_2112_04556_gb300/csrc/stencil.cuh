// The adjoint covariant hop sum of Sec. 2, Eq. (3) for one site and all four field components:
//   acc_mu = 2 * sum_nu [ U_nu(x) X_mu(x+nu) U_nu(x)^dag + U_nu(x-nu)^dag X_mu(x-nu) U_nu(x-nu) ]
// (the factor 2 comes from the doubled Hermitian expansion of the coefficients).  Every link of the
// site is loaded once and applied to the four components; a field value is produced by the source
// functor `src(site, mu, x[8])`, which lets callers fuse an axpy into the stencil's loads.
#pragma once
#include "common.cuh"

namespace rm {

template <typename T> struct LinksOf;
template <> struct LinksOf<double> { using type = Links64; };
template <> struct LinksOf<float> { using type = Links32; };

template <typename T, int LF, class Src>
__device__ __forceinline__ void hop_sum4(const Geom& g, const typename LinksOf<T>::type& U, int s,
                                         const Src& src, herm<T> (&acc)[4]) {
    int fwd[4], bwd[4];
    neighbours(g, s, fwd, bwd);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) acc[mu] = h_zero<T>();
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        {
            const mat3<T> u = LinkLoad<T, LF>::load(U, s, nu);
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                T x[8];
                src(fwd[nu], mu, x);
                acc_uxud(acc[mu], u, coef_to_herm2(x));
            }
        }
        {
            const mat3<T> u = LinkLoad<T, LF>::load(U, bwd[nu], nu);
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                T x[8];
                src(bwd[nu], mu, x);
                acc_udxu(acc[mu], u, coef_to_herm2(x));
            }
        }
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
