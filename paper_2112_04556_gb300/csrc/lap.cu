// Sec. 2, Eq. (3): the normalised adjoint covariant Laplacian A = -Delta_G/16 as a fused stencil
//   Y = a X + b * H(X) + c W,   H(X)_mu(x) = sum_nu [U X(x+nu) U^dag + U^dag X(x-nu) U]
// with optional per-field float64 sums <Y,Y> and <Y,X> (the Chebyshev moments).  Four lanes per site,
// one per field component (see stencil.cuh).
#include "common.cuh"
#include "ops.cuh"
#include "stencil.cuh"
#include "tune.cuh"

namespace rm {

template <typename T, int LF, int NMU, bool HAS_W, bool DOTS>
__global__ void __launch_bounds__(kBlockMax, (stencil_min_blocks<T, NMU>())) k_lap(Geom g, typename LinksOf<T>::type U, const T* __restrict__ X,
                                                    T* __restrict__ Y, const T* __restrict__ W, T a, T b, T c,
                                                    size_t fstride, double* partials, unsigned* counters, double* out,
                                                    size_t slot_stride) {
    constexpr int NC = NMU == 0 ? 1 : NMU;   // components per lane
    constexpr int LPS = 4 / NC;
    __shared__ double sh[2 * (kBlockMax / 32)];
    const int f = blockIdx.y;
    const T* Xf = X + f * fstride;
    T* Yf = Y + f * fstride;
    T dyy = T(0), dyx = T(0);
    const int nlane = g.V * LPS;
    for (int lane = blockIdx.x * blockDim.x + threadIdx.x; lane < nlane; lane += gridDim.x * blockDim.x) {
        const int s = lane / LPS, mu0 = (lane % LPS) * NC;
        herm<T> acc[NC];
        hop_sum_shape<T, LF, NMU>(g, U, s, mu0, SrcField<T>{Xf}, acc);
#pragma unroll
        for (int m = 0; m < NC; m++) {
            const int mu = mu0 + m;
            T h[8], x[8], y[8];
            herm2_to_coef_tl(acc[m], h);
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
    }
    if (DOTS) {
        double v[2] = {0.0, 0.0};
        if (sizeof(T) == 4) {
            float fv[2] = {(float)dyy, (float)dyx};
            block_sum_f<2>(fv, sh);
            if (threadIdx.x == 0) {
                const int nw = blockDim.x >> 5;
                for (int n = 0; n < 2; n++) {
                    double t = 0.0;
                    for (int w = 0; w < nw; w++) t += sh[n * nw + w];
                    v[n] = t;
                }
            }
        } else {
            v[0] = (double)dyy;
            v[1] = (double)dyx;
            block_sum<2>(v, sh);
        }
        grid_sum_finish<2>(v, partials + f * slot_stride, counters + f, out + (size_t)f * 8, gridDim.x, blockIdx.x, sh);
    }
}

template <typename T, int LF, int NMU>
static void launch_lap_shape(rmhmc_ctx* ctx, const StencilShape& shp, const T* X, T* Y, int nfield, double a, double b,
                             const T* W, double c, int slot, cudaStream_t st) {
    const dim3 grid(stencil_blocks(ctx, shp), nfield);
    const size_t fs = field_elems(ctx);
    const size_t ss = (size_t)ctx->max_blocks * 2;
    double* part = slot >= 0 ? red_slot_partials(ctx, slot) : nullptr;
    unsigned* cnt = slot >= 0 ? red_slot_counter(ctx, slot) : nullptr;
    double* out = slot >= 0 ? red_slot_out(ctx, slot) : nullptr;
    typename LinksOf<T>::type U;
    if constexpr (sizeof(T) == 8) U = links64(ctx); else U = links32(ctx);
    if (W) {
        if (slot >= 0) k_lap<T, LF, NMU, true, true><<<grid, shp.block, 0, st>>>(ctx->g, U, X, Y, W, (T)a, (T)b, (T)c, fs, part, cnt, out, ss);
        else k_lap<T, LF, NMU, true, false><<<grid, shp.block, 0, st>>>(ctx->g, U, X, Y, W, (T)a, (T)b, (T)c, fs, part, cnt, out, ss);
    } else {
        if (slot >= 0) k_lap<T, LF, NMU, false, true><<<grid, shp.block, 0, st>>>(ctx->g, U, X, Y, W, (T)a, (T)b, (T)c, fs, part, cnt, out, ss);
        else k_lap<T, LF, NMU, false, false><<<grid, shp.block, 0, st>>>(ctx->g, U, X, Y, W, (T)a, (T)b, (T)c, fs, part, cnt, out, ss);
    }
    ++ctx->launches;
}

template <typename T, int LF>
static int launch_lap_t(rmhmc_ctx* ctx, const T* X, T* Y, int nfield, double a, double b, const T* W, double c,
                        int slot, cudaStream_t st) {
    StencilShape shp;
    RM_TRY((stencil_shape<T, LF>(ctx, st, shp)));
    if (shp.nmu == 8) {
        // the link-centric kernel serves one plain field; with a third term or dots the gather kernel runs
        if (sizeof(T) == 4 && nfield == 1 && !W && slot < 0)
            return launch_lap_lc(ctx, LF, (const float*)X, (float*)Y, a, b, st);
        shp = StencilShape{2, 256};
    }
    if (shp.nmu == 4) launch_lap_shape<T, LF, 4>(ctx, shp, X, Y, nfield, a, b, W, c, slot, st);
    else if (shp.nmu == 2) launch_lap_shape<T, LF, 2>(ctx, shp, X, Y, nfield, a, b, W, c, slot, st);
    else if (shp.nmu == 0) launch_lap_shape<T, LF, 0>(ctx, shp, X, Y, nfield, a, b, W, c, slot, st);
    else launch_lap_shape<T, LF, 1>(ctx, shp, X, Y, nfield, a, b, W, c, slot, st);
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}

// ------------------------------------------------------------------------------------------------
// the autotuner (declared in tune.cuh)
// ------------------------------------------------------------------------------------------------
template <typename T, int LF>
int stencil_shape(rmhmc_ctx* ctx, cudaStream_t st, StencilShape& out) {
    const int key = (int)sizeof(T) * 100 + LF;
    auto it = ctx->tune.find(key);
    if (it != ctx->tune.end()) {
        out.nmu = it->second.first;
        out.block = it->second.second;
        return RMHMC_OK;
    }
    int status = RMHMC_OK;
    const size_t fs = field_elems(ctx);
    T* X = (T*)workspace(ctx, "tune_x", sizeof(double) * fs, &status);
    T* Y = (T*)workspace(ctx, "tune_y", sizeof(double) * fs, &status);
    if (!X || !Y) return status;
    RM_CHECK(ctx, cudaMemsetAsync(X, 0, sizeof(T) * fs, st));
    cudaEvent_t e0, e1;
    RM_CHECK(ctx, cudaEventCreate(&e0));
    RM_CHECK(ctx, cudaEventCreate(&e1));
    float best = 1e30f;
    StencilShape bs;
    char line[128];
    std::string rep;
    for (int nmu : {1, 2, 4, 0, 8})
        for (int block : {64, 128, 256}) {
            if (nmu == 8 && (sizeof(T) == 8 || block != 256)) continue;   // the link-centric kernel: float32, 256
            const StencilShape shp{nmu, block};
            auto run = [&]() {
                if (nmu == 8) launch_lap_lc(ctx, LF, (const float*)X, (float*)Y, 0.5, -0.0625, st);
                else if (nmu == 4) launch_lap_shape<T, LF, 4>(ctx, shp, X, Y, 1, 0.5, -0.0625, nullptr, 0.0, -1, st);
                else if (nmu == 2) launch_lap_shape<T, LF, 2>(ctx, shp, X, Y, 1, 0.5, -0.0625, nullptr, 0.0, -1, st);
                else if (nmu == 0) launch_lap_shape<T, LF, 0>(ctx, shp, X, Y, 1, 0.5, -0.0625, nullptr, 0.0, -1, st);
                else launch_lap_shape<T, LF, 1>(ctx, shp, X, Y, 1, 0.5, -0.0625, nullptr, 0.0, -1, st);
            };
            run();
            RM_CHECK(ctx, cudaEventRecord(e0, st));
            for (int r = 0; r < 3; r++) run();
            RM_CHECK(ctx, cudaEventRecord(e1, st));
            RM_CHECK(ctx, cudaEventSynchronize(e1));
            RM_LAUNCH_CHECK(ctx);
            float ms = 0.f;
            RM_CHECK(ctx, cudaEventElapsedTime(&ms, e0, e1));
            ms /= 3.f;
            snprintf(line, sizeof line, "%s%d/%d:%.4f", rep.empty() ? "" : " ", nmu, block, ms);
            rep += line;
            if (ms < best) { best = ms; bs = shp; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tune[key] = {bs.nmu, bs.block};
    snprintf(line, sizeof line, "%s%s LF%d -> nmu %d block %d [", ctx->tune_report.empty() ? "" : "; ",
             sizeof(T) == 8 ? "fp64" : "fp32", LF, bs.nmu, bs.block);
    ctx->tune_report += line + rep + "]";
    out = bs;
    return RMHMC_OK;
}

template int stencil_shape<float, 18>(rmhmc_ctx*, cudaStream_t, StencilShape&);
template int stencil_shape<float, 12>(rmhmc_ctx*, cudaStream_t, StencilShape&);
template int stencil_shape<double, 18>(rmhmc_ctx*, cudaStream_t, StencilShape&);
template int stencil_shape<double, 12>(rmhmc_ctx*, cudaStream_t, StencilShape&);

int launch_lap(rmhmc_ctx* ctx, int prec, int linkfmt, const void* X, void* Y, int nfield, double a, double b,
               const void* W, double c, int slot, cudaStream_t st) {
    if (slot >= 0 && slot + nfield > kRedSlots) return set_err(ctx, RMHMC_EINVAL, "too many reduced fields");
    if (prec == RMHMC_FP64) {
        if (linkfmt == 12)
            return launch_lap_t<double, 12>(ctx, (const double*)X, (double*)Y, nfield, a, b, (const double*)W, c, slot, st);
        return launch_lap_t<double, 18>(ctx, (const double*)X, (double*)Y, nfield, a, b, (const double*)W, c, slot, st);
    }
    if (nfield >= kAdMinFields)
        return launch_lap_ad(ctx, linkfmt, (const float*)X, (float*)Y, nfield, a, b, (const float*)W, c, slot, st);
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
