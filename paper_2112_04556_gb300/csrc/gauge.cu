// Gauge action and force (Sec. 2: F_G = -dS/dU with the left-multiplication derivative), for the
// Wilson plaquette action plus 1x2 rectangles (c1 = 0: Wilson; c1 = -0.331: Iwasaki; c0 = 1 - 8 c1).
//
// For the link U = U_mu(x) the loops through it are written as Re Tr(U Sigma) with the staple sum
// Sigma = c0 Sigma_plaq + c1 Sigma_rect (6 plaquette and 18 rectangle staples, each a product of the
// other links starting at x+mu and returning to x).  With U -> exp(i w^a T^a) U,
//   F^a = (beta/3) Re Tr(i T^a U Sigma) = -(beta/6) Tr(lambda^a K),  K = -i (M - M^dag)/2,  M = U Sigma.
#include "common.cuh"
#include "ops.cuh"

namespace rm {

constexpr int kSlotAction = 40;

// index of the site c + n1 e_d1 + n2 e_d2 (|n1|, |n2| <= 2, d1 != d2 or n2 = 0), periodic, without division
__device__ __forceinline__ int site_at(const Geom& g, const int c[4], int d1, int n1, int d2, int n2) {
    int s = 0;
#pragma unroll
    for (int e = 3; e >= 0; e--) {
        int v = c[e] + (e == d1 ? n1 : 0) + (e == d2 ? n2 : 0);
        if (v >= g.L[e]) v -= g.L[e];
        if (v >= g.L[e]) v -= g.L[e];
        if (v < 0) v += g.L[e];
        if (v < 0) v += g.L[e];
        s = s * g.L[e] + v;
    }
    return s;
}

template <typename T> RM_HD void m_acc_w(mat3<T>& a, const mat3<T>& b, T w) {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            a.e[i][j].re = fma(w, b.e[i][j].re, a.e[i][j].re);
            a.e[i][j].im = fma(w, b.e[i][j].im, a.e[i][j].im);
        }
}

template <typename T> struct GLinks;
template <> struct GLinks<double> {
    Links64 U;
    __device__ __forceinline__ mat3<double> operator()(int s, int mu) const { return LinkLoad<double, 18>::load(U, s, mu); }
};
template <> struct GLinks<float> {
    Links32 U;
    __device__ __forceinline__ mat3<float> operator()(int s, int mu) const { return LinkLoad<float, 18>::load(U, s, mu); }
};

// weighted staple sum S = c0 Sigma_plaq + c1 Sigma_rect of link (x, mu)
template <typename T>
__device__ __forceinline__ mat3<T> staple_sum(const Geom& g, const GLinks<T>& U, const int c[4], int x, int mu, T c0,
                                              T c1) {
    mat3<T> S = m_zero<T>();
    const bool rect = c1 != T(0);
#pragma unroll 1
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        const int xpm = site_at(g, c, mu, 1, nu, 0);
        const int xpn = site_at(g, c, nu, 1, mu, 0);
        const int xmn = site_at(g, c, nu, -1, mu, 0);
        const int xpmmn = site_at(g, c, mu, 1, nu, -1);
        // plaquettes: up U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag ; down U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
        m_acc_w(S, m_mul_nd(m_mul_nd(U(xpm, nu), U(xpn, mu)), U(x, nu)), c0);
        m_acc_w(S, m_mul(m_mul_dn(U(xpmmn, nu), m_dag(U(xmn, mu))), U(xmn, nu)), c0);
        if (!rect) continue;
        const int x2m = site_at(g, c, mu, 2, nu, 0);
        const int xpmpn = site_at(g, c, mu, 1, nu, 1);
        const int xmm = site_at(g, c, mu, -1, nu, 0);
        const int xmmpn = site_at(g, c, mu, -1, nu, 1);
        const int x2mmn = site_at(g, c, mu, 2, nu, -1);
        const int xmmmn = site_at(g, c, mu, -1, nu, -1);
        const int xp2n = site_at(g, c, nu, 2, mu, 0);
        const int xpmm2n = site_at(g, c, mu, 1, nu, -2);
        const int xm2n = site_at(g, c, nu, -2, mu, 0);
        // (a) U_mu(x+mu) U_nu(x+2mu) U_mu(x+mu+nu)^dag U_mu(x+nu)^dag U_nu(x)^dag
        {
            mat3<T> a = m_mul(U(xpm, mu), U(x2m, nu));
            a = m_mul_nd(a, U(xpmpn, mu));
            a = m_mul_nd(a, U(xpn, mu));
            m_acc_w(S, m_mul_nd(a, U(x, nu)), c1);
        }
        // (b) U_nu(x+mu) U_mu(x+nu)^dag U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
        {
            mat3<T> a = m_mul_nd(U(xpm, nu), U(xpn, mu));
            a = m_mul_nd(a, U(xmmpn, mu));
            a = m_mul_nd(a, U(xmm, nu));
            m_acc_w(S, m_mul(a, U(xmm, mu)), c1);
        }
        // (c) U_mu(x+mu) U_nu(x+2mu-nu)^dag U_mu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
        {
            mat3<T> a = m_mul_nd(U(xpm, mu), U(x2mmn, nu));
            a = m_mul_nd(a, U(xpmmn, mu));
            a = m_mul_nd(a, U(xmn, mu));
            m_acc_w(S, m_mul(a, U(xmn, nu)), c1);
        }
        // (d) U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_mu(x-mu-nu)^dag U_nu(x-mu-nu) U_mu(x-mu)
        {
            mat3<T> a = m_mul_dn(U(xpmmn, nu), m_dag(U(xmn, mu)));
            a = m_mul_nd(a, U(xmmmn, mu));
            a = m_mul(a, U(xmmmn, nu));
            m_acc_w(S, m_mul(a, U(xmm, mu)), c1);
        }
        // (e) U_nu(x+mu) U_nu(x+mu+nu) U_mu(x+2nu)^dag U_nu(x+nu)^dag U_nu(x)^dag
        {
            mat3<T> a = m_mul(U(xpm, nu), U(xpmpn, nu));
            a = m_mul_nd(a, U(xp2n, mu));
            a = m_mul_nd(a, U(xpn, nu));
            m_acc_w(S, m_mul_nd(a, U(x, nu)), c1);
        }
        // (f) U_nu(x+mu-nu)^dag U_nu(x+mu-2nu)^dag U_mu(x-2nu)^dag U_nu(x-2nu) U_nu(x-nu)
        {
            mat3<T> a = m_mul_dn(U(xpmmn, nu), m_dag(U(xpmm2n, nu)));
            a = m_mul_nd(a, U(xm2n, mu));
            a = m_mul(a, U(xm2n, nu));
            m_acc_w(S, m_mul(a, U(xmn, nu)), c1);
        }
    }
    return S;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_gauge_force(Geom g, GLinks<T> U, T beta, T c0, T c1, double* __restrict__ F) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (x >= g.V) return;
    int c[4];
    site_coords(g, x, c);
    const mat3<T> S = staple_sum<T>(g, U, c, x, mu, c0, c1);
    const mat3<T> M = m_mul(U(x, mu), S);
    T k[8];
    antiherm_coef(M, k);
    double* out = F + (size_t)x * 32 + mu * 8;
#pragma unroll
    for (int a = 0; a < 8; a++) out[a] = -(double)(beta / T(6)) * (double)k[a];
}

// action density beta [c0 sum_{mu<nu}(1 - ReTr P/3) + c1 sum_{mu!=nu}(1 - ReTr R/3)] and the plaquette sum
__global__ void __launch_bounds__(kBlock) k_action(Geom g, Links64 U64, double beta, double c0, double c1,
                                                   double* partials, unsigned* counter, double* out) {
    __shared__ double sh[2 * (kBlock / 32)];
    const GLinks<double> U{U64};
    double act = 0.0, plaq = 0.0;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.V; x += gridDim.x * blockDim.x) {
        double ax = 0.0;
        int c[4];
        site_coords(g, x, c);
        for (int mu = 0; mu < 4; mu++)
            for (int nu = 0; nu < 4; nu++) {
                if (mu == nu) continue;
                const int xpm = site_at(g, c, mu, 1, nu, 0);
                const int xpn = site_at(g, c, nu, 1, mu, 0);
                if (mu < nu) {
                    mat3<double> p = m_mul(U(x, mu), U(xpm, nu));
                    p = m_mul_nd(p, U(xpn, mu));
                    const double rt = re_trace(m_mul_nd(p, U(x, nu))) / 3.0;
                    plaq += rt;
                    ax += c0 * (1.0 - rt);
                }
                if (c1 != 0.0) {
                    const int x2m = site_at(g, c, mu, 2, nu, 0);
                    const int xpmpn = site_at(g, c, mu, 1, nu, 1);
                    mat3<double> r = m_mul(U(x, mu), U(xpm, mu));
                    r = m_mul(r, U(x2m, nu));
                    r = m_mul_nd(r, U(xpmpn, mu));
                    r = m_mul_nd(r, U(xpn, mu));
                    const double rt = re_trace(m_mul_nd(r, U(x, nu))) / 3.0;
                    ax += c1 * (1.0 - rt);
                }
            }
        act += beta * ax;
    }
    double v[2] = {act, plaq};
    block_sum<2>(v, sh);
    grid_sum_finish<2>(v, partials, counter, out, gridDim.x, blockIdx.x, sh);
}

int gauge_force_launch(rmhmc_ctx* ctx, double beta, double c1, int prec, double* F, cudaStream_t st) {
    const dim3 grid(site_blocks(ctx), 4);
    const double c0 = 1.0 - 8.0 * c1;
    if (prec == RMHMC_FP64)
        k_gauge_force<double><<<grid, kBlock, 0, st>>>(ctx->g, GLinks<double>{links64(ctx)}, beta, c0, c1, F);
    else
        k_gauge_force<float><<<grid, kBlock, 0, st>>>(ctx->g, GLinks<float>{links32(ctx)}, (float)beta, (float)c0, (float)c1, F);
    ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}

int action_launch(rmhmc_ctx* ctx, double beta, double c1, double* S, double* plaq, cudaStream_t st) {
    k_action<<<capped_grid(ctx, ctx->g.V, kBlock), kBlock, 0, st>>>(ctx->g, links64(ctx), beta, 1.0 - 8.0 * c1, c1,
                                                  red_slot_partials(ctx, kSlotAction), red_slot_counter(ctx, kSlotAction),
                                                  red_slot_out(ctx, kSlotAction)); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    double out[2];
    RM_TRY(fetch(ctx, red_slot_out(ctx, kSlotAction), out, 2, st));
    if (S) *S = out[0];
    if (plaq) *plaq = out[1] / (6.0 * ctx->g.V);
    return RMHMC_OK;
}

}  // namespace rm

using namespace rm;

extern "C" int gauge_force(rmhmc_ctx* ctx, const double* U, double beta, double c1, int prec, double* F, double* action,
                           double* plaq, cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (prec != RMHMC_FP64 && prec != RMHMC_FP32) return set_err(ctx, RMHMC_EINVAL, "gauge_force: bad prec");
    if (!F && !action && !plaq) return set_err(ctx, RMHMC_EINVAL, "gauge_force: nothing to compute");
    RM_TRY(ensure_links(ctx, U, stream));
    if (F) RM_TRY(gauge_force_launch(ctx, beta, c1, prec, F, stream));
    if (action || plaq) RM_TRY(action_launch(ctx, beta, c1, action, plaq, stream));
    return RMHMC_OK;
}
