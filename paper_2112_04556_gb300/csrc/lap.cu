// Sec. 2, Eq. (3): the normalised adjoint covariant Laplacian A = -Delta_G/16 as a fused stencil
//   Y = a X + b * H(X) + c W,   H(X)_mu(x) = sum_nu [U X(x+nu) U^dag + U^dag X(x-nu) U]
// with optional per-field float64 sums <Y,Y> and <Y,X> (the Chebyshev moments).  Four lanes per site,
// one per field component (see stencil.cuh).
#include "common.cuh"
#include "ops.cuh"
#include "stencil.cuh"

namespace rm {

template <typename T, int LF, bool HAS_W, bool DOTS>
__global__ void __launch_bounds__(kBlock) k_lap(Geom g, typename LinksOf<T>::type U, const T* __restrict__ X,
                                                 T* __restrict__ Y, const T* __restrict__ W, T a, T b, T c,
                                                 size_t fstride, double* partials, unsigned* counters, double* out,
                                                 size_t slot_stride) {
    __shared__ double sh[2 * (kBlock / 32)];
    const int f = blockIdx.y;
    const T* Xf = X + f * fstride;
    T* Yf = Y + f * fstride;
    const int lane = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = lane >> 2, mu = lane & 3;
    T dyy = T(0), dyx = T(0);
    if (s < g.V) {
        herm<T> acc;
        hop_sum1<T, LF>(g, U, s, mu, SrcField<T>{Xf}, acc);
        T h[8], x[8], y[8];
        herm2_to_coef(acc, h);
        load8(Xf + (size_t)s * 32 + mu * 8, x);
#pragma unroll
        for (int k = 0; k < 8; k++) y[k] = fma(b, h[k], a * x[k]);
        if (HAS_W) {
            T w[8];
            load8(W + f * fstride + (size_t)s * 32 + mu * 8, w);
#pragma unroll
            for (int k = 0; k < 8; k++) y[k] = fma(c, w[k], y[k]);
        }
        store8(Yf + (size_t)s * 32 + mu * 8, y);
        if (DOTS) {
#pragma unroll
            for (int k = 0; k < 8; k++) { dyy = fma(y[k], y[k], dyy); dyx = fma(y[k], x[k], dyx); }
        }
    }
    if (DOTS) {
        double v[2];
        if (sizeof(T) == 4) {
            float fv[2] = {(float)dyy, (float)dyx};
            block_sum_f<2>(fv, sh);
            if (threadIdx.x == 0) {
                for (int n = 0; n < 2; n++) {
                    double t = 0.0;
                    for (int w = 0; w < kBlock / 32; w++) t += sh[n * (kBlock / 32) + w];
                    v[n] = t;
                }
            }
        } else {
            v[0] = (double)dyy;
            v[1] = (double)dyx;
            block_sum<2>(v, sh);
        }
        if (threadIdx.x == 0)
            grid_sum_finish<2>(v, partials + f * slot_stride, counters + f, out + (size_t)f * 8, gridDim.x, blockIdx.x);
    }
}

template <typename T, int LF>
static int launch_lap_t(rmhmc_ctx* ctx, const T* X, T* Y, int nfield, double a, double b, const T* W, double c,
                        int slot, cudaStream_t st) {
    const dim3 grid(lane_blocks(ctx), nfield);
    const size_t fs = field_elems(ctx);
    const size_t ss = (size_t)ctx->max_blocks * 8;
    double* part = slot >= 0 ? red_slot_partials(ctx, slot) : nullptr;
    unsigned* cnt = slot >= 0 ? red_slot_counter(ctx, slot) : nullptr;
    double* out = slot >= 0 ? red_slot_out(ctx, slot) : nullptr;
    typename LinksOf<T>::type U;
    if constexpr (sizeof(T) == 8) U = links64(ctx); else U = links32(ctx);
    if (W) {
        if (slot >= 0) k_lap<T, LF, true, true><<<grid, kBlock, 0, st>>>(ctx->g, U, X, Y, W, (T)a, (T)b, (T)c, fs, part, cnt, out, ss);
        else k_lap<T, LF, true, false><<<grid, kBlock, 0, st>>>(ctx->g, U, X, Y, W, (T)a, (T)b, (T)c, fs, part, cnt, out, ss);
    } else {
        if (slot >= 0) k_lap<T, LF, false, true><<<grid, kBlock, 0, st>>>(ctx->g, U, X, Y, W, (T)a, (T)b, (T)c, fs, part, cnt, out, ss);
        else k_lap<T, LF, false, false><<<grid, kBlock, 0, st>>>(ctx->g, U, X, Y, W, (T)a, (T)b, (T)c, fs, part, cnt, out, ss);
    }
    ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}

int launch_lap(rmhmc_ctx* ctx, int prec, int linkfmt, const void* X, void* Y, int nfield, double a, double b,
               const void* W, double c, int slot, cudaStream_t st) {
    if (slot >= 0 && slot + nfield > kRedSlots) return set_err(ctx, RMHMC_EINVAL, "too many reduced fields");
    if (prec == RMHMC_FP64) {
        if (linkfmt == 12)
            return launch_lap_t<double, 12>(ctx, (const double*)X, (double*)Y, nfield, a, b, (const double*)W, c, slot, st);
        return launch_lap_t<double, 18>(ctx, (const double*)X, (double*)Y, nfield, a, b, (const double*)W, c, slot, st);
    }
    if (linkfmt == 12)
        return launch_lap_t<float, 12>(ctx, (const float*)X, (float*)Y, nfield, a, b, (const float*)W, c, slot, st);
    return launch_lap_t<float, 18>(ctx, (const float*)X, (float*)Y, nfield, a, b, (const float*)W, c, slot, st);
}

}  // namespace rm

using namespace rm;

extern "C" int lap_apply(rmhmc_ctx* ctx, const double* U, const void* X, void* Y, int nfield, int prec,
                         int linkfmt, int op, cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (!X || !Y || nfield < 0 || nfield > 65535) return set_err(ctx, RMHMC_EINVAL, "lap_apply: bad field arguments");
    if (prec != RMHMC_FP64 && prec != RMHMC_FP32) return set_err(ctx, RMHMC_EINVAL, "lap_apply: bad prec");
    if (linkfmt != 18 && linkfmt != 12) return set_err(ctx, RMHMC_EINVAL, "lap_apply: linkfmt must be 18 or 12");
    if (op != RMHMC_OP_A && op != RMHMC_OP_DELTA) return set_err(ctx, RMHMC_EINVAL, "lap_apply: bad op");
    if ((uintptr_t)X % 16 || (uintptr_t)Y % 16) return set_err(ctx, RMHMC_EINVAL, "lap_apply: fields must be 16-byte aligned");
    const size_t bytes = field_elems(ctx) * (prec == RMHMC_FP64 ? 8 : 4) * (size_t)nfield;
    const char *xb = (const char*)X, *yb = (const char*)Y;
    if (xb < yb + bytes && yb < xb + bytes) return set_err(ctx, RMHMC_EINVAL, "lap_apply: X and Y overlap");
    RM_TRY(ensure_links(ctx, U, stream));
    if (nfield == 0) return RMHMC_OK;
    const double a = op == RMHMC_OP_A ? 0.5 : -8.0;
    const double b = op == RMHMC_OP_A ? -1.0 / 16.0 : 1.0;
    return launch_lap(ctx, prec, linkfmt, X, Y, nfield, a, b, nullptr, 0.0, -1, stream);
}
