// The adjoint covariant hop sum of Sec. 2, Eq. (3) for one site and one field component mu:
//   acc = 2 * sum_nu [ U_nu(x) X_mu(x+nu) U_nu(x)^dag + U_nu(x-nu)^dag X_mu(x-nu) U_nu(x-nu) ]
// (the factor 2 comes from the doubled Hermitian expansion of the coefficients).  Every term is traceless, so
// the sum is accumulated without its (2,2) entry (acc_*_tl) and read with herm2_to_coef_tl.
//
// Thread layout of the stencil kernels: 4 / NMU consecutive lanes own one site, each lane NMU of its four
// field components (NMU = 1: a warp covers 8 consecutive sites, its loads of X_mu at a neighbour are one
// contiguous 1 KB segment of the [V][4][8] field and its link loads hit 8 consecutive entries of the
// structure-of-arrays link copy).  NMU and the block size are chosen per context by the autotuner
// (tune.cuh): fewer lanes per site load each link fewer times but hold more registers.
#pragma once
#include "common.cuh"

namespace rm {

template <typename T> struct LinksOf;
template <> struct LinksOf<double> { using type = Links64; };
template <> struct LinksOf<float> { using type = Links32; };

// NMU consecutive field components mu0 .. mu0+NMU-1 of one site per lane (NMU = 1, 2 or 4: four, two or one
// lane(s) per site); every link is loaded once per lane and applied to the lane's components
template <typename T, int LF, int NMU, class Src>
__device__ __forceinline__ void hop_sum(const Geom& g, const typename LinksOf<T>::type& U, int s, int mu0,
                                        const Src& src, herm<T> (&acc)[NMU]) {
    int fwd[4], bwd[4];
    neighbours(g, s, fwd, bwd);
#pragma unroll
    for (int m = 0; m < NMU; m++) acc[m] = h_zero<T>();
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        {
            const mat3<T> uf = LinkLoad<T, LF>::load(U, s, nu);
#pragma unroll
            for (int m = 0; m < NMU; m++) {
                T x[8];
                src(fwd[nu], mu0 + m, x);
                acc_uxud_tl(acc[m], uf, coef_to_herm2(x));
            }
        }
        {
            const mat3<T> ub = LinkLoad<T, LF>::load(U, bwd[nu], nu);
#pragma unroll
            for (int m = 0; m < NMU; m++) {
                T x[8];
                src(bwd[nu], mu0 + m, x);
                acc_udxu_tl(acc[m], ub, coef_to_herm2(x));
            }
        }
    }
}

// NMU = 1 with the eight neighbour values of the lane's component loaded before any arithmetic (more
// loads in flight per lane, more registers); the links follow hop by hop
template <typename T, int LF, class Src>
__device__ __forceinline__ void hop_sum_prefetch(const Geom& g, const typename LinksOf<T>::type& U, int s, int mu,
                                                 const Src& src, herm<T>& acc) {
    int fwd[4], bwd[4];
    neighbours(g, s, fwd, bwd);
    T xf[4][8], xb[4][8];
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        src(fwd[nu], mu, xf[nu]);
        src(bwd[nu], mu, xb[nu]);
    }
    acc = h_zero<T>();
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        const mat3<T> uf = LinkLoad<T, LF>::load(U, s, nu);
        const mat3<T> ub = LinkLoad<T, LF>::load(U, bwd[nu], nu);
        acc_uxud_tl(acc, uf, coef_to_herm2(xf[nu]));
        acc_udxu_tl(acc, ub, coef_to_herm2(xb[nu]));
    }
}

// dispatch on the lane shape: NMU in {1, 2, 4}; NMU = 0 means NMU = 1 with the prefetching variant
template <typename T, int LF, int NMU, class Src>
__device__ __forceinline__ void hop_sum_shape(const Geom& g, const typename LinksOf<T>::type& U, int s, int mu0,
                                              const Src& src, herm<T> (&acc)[NMU == 0 ? 1 : NMU]) {
    if constexpr (NMU == 0) hop_sum_prefetch<T, LF>(g, U, s, mu0, src, acc[0]);
    else hop_sum<T, LF, NMU>(g, U, s, mu0, src, acc);
}

template <typename T, int LF, class Src>
__device__ __forceinline__ void hop_sum1(const Geom& g, const typename LinksOf<T>::type& U, int s, int mu,
                                         const Src& src, herm<T>& acc) {
    herm<T> a[1];
    hop_sum<T, LF, 1>(g, U, s, mu, src, a);
    acc = a[0];
}

// plain field source: X[s][mu][8]
template <typename T> struct SrcField {
    const T* X;
    __device__ __forceinline__ void operator()(int s, int mu, T* x) const { load8(X + (size_t)s * 32 + mu * 8, x); }
};

// plain float32 field of the context's own (32-byte aligned, read-only during the kernel) buffers, read with
// 256-bit loads
struct SrcFieldV8 {
    const float* X;
    __device__ __forceinline__ void operator()(int s, int mu, float* x) const { load8_v8(X + (size_t)s * 32 + mu * 8, x); }
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
