// Sec. 2, Eq. (4): Chebyshev band-pass filters B_w = sum_k C[w][k] T_k(2A - 1) and the per-mode
// power spectrum <F|B_w|F> / Tr B_w.
//
// Every field (forces and noise vectors) runs the three-term recurrence
//   v_0 = G, v_1 = (2A-1) v_0 = -H(v_0)/8, v_{k+1} = 2(2A-1) v_k - v_{k-1} = -H(v_k)/4 - v_{k-1}
// in one batched launch per step (all fields share the links).  The moments mu_k = <G, T_k G> come from
// the products T_k T_l = (T_{k+l} + T_{|k-l|})/2:
//   mu_{2k} = 2 <v_k, v_k> - mu_0,  mu_{2k-1} = 2 <v_k, v_{k-1}> - mu_1,
// so K = ceil(N/2) stencil applications give mu_0 .. mu_N.  All windows share the moments.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "krylov.cuh"
#include "ops.cuh"
#include "philox.cuh"

namespace rm {

constexpr int kSlotCheb = 128;   // first reduction slot of the batched moments (kRedSlots - 128 fields)

template <typename T>
__global__ void k_copy_norms(const double* __restrict__ in, T* __restrict__ out, size_t fs, int V, double* partials,
                             unsigned* counters, double* red_out, size_t slot_stride) {
    __shared__ double sh[kBlock / 32];
    const int f = blockIdx.y;
    double acc = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += gridDim.x * blockDim.x) {
        const double* src = in + f * fs + (size_t)s * 32;
        T* dst = out + f * fs + (size_t)s * 32;
#pragma unroll 4
        for (int k = 0; k < 32; k++) {
            const T x = (T)src[k];
            dst[k] = x;
            acc += (double)x * (double)x;
        }
    }
    double v[1] = {acc};
    block_sum<1>(v, sh);
    grid_sum_finish<1>(v, partials + f * slot_stride, counters + f, red_out + (size_t)f * 8, gridDim.x, blockIdx.x, sh);
}

__global__ void k_gauss_fields(double* __restrict__ out, size_t fs, int V, uint64_t seed, uint32_t tag) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int f = blockIdx.y;
    if (s >= V) return;
    double* dst = out + f * fs + (size_t)s * 32;
    for (int k = 0; k < 16; k++) {
        u32x4 c{{(uint32_t)k, (uint32_t)s, (uint32_t)f, tag}};
        const u32x4 w = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        const double u0 = u53(w.v[0], w.v[1]), u1 = u53(w.v[2], w.v[3]);
        const double r = sqrt(-2.0 * log(u0));
        double sn, cs;
        sincospi(2.0 * u1, &sn, &cs);
        dst[2 * k] = r * cs;
        dst[2 * k + 1] = r * sn;
    }
}

// window coefficients: Chebyshev expansion (in x = 2 lam - 1) of the indicator of [a, b] with
// theta = arccos x:  c_0 = (th_a - th_b)/pi, c_k = 2 (sin k th_a - sin k th_b)/(k pi), times the Jackson
// damping g_k = [(N-k+1) cos(pi k/(N+1)) + sin(pi k/(N+1)) cot(pi/(N+1))]/(N+1) if requested
static void window_coefficients(const double* edges, int nwin, int N, bool jackson, std::vector<double>& C) {
    C.assign((size_t)nwin * (N + 1), 0.0);
    const double q = M_PI / (N + 1);
    for (int w = 0; w < nwin; w++) {
        const double ta = acos(std::max(-1.0, std::min(1.0, 2.0 * edges[w] - 1.0)));
        const double tb = acos(std::max(-1.0, std::min(1.0, 2.0 * edges[w + 1] - 1.0)));
        for (int k = 0; k <= N; k++) {
            double c = k == 0 ? (ta - tb) / M_PI : 2.0 * (sin(k * ta) - sin(k * tb)) / (k * M_PI);
            if (jackson) c *= ((N - k + 1) * cos(q * k) + sin(q * k) / tan(q)) / (N + 1);
            C[(size_t)w * (N + 1) + k] = c;
        }
    }
}

template <typename T>
static int cheb_run(rmhmc_ctx* ctx, const double* fields64, int nr, int N, int prec, std::vector<double>& mu,
                    cudaStream_t st) {
    int status = RMHMC_OK;
    const size_t fs = field_elems(ctx);
    const bool f32 = sizeof(T) == 4;
    T* buf = (T*)workspace(ctx, f32 ? "cb_v32" : "cb_v64", sizeof(T) * fs * nr * 3, &status);
    double* dmom = (double*)workspace(ctx, "cb_mom", sizeof(double) * 8 * nr * (N / 2 + 2), &status);
    if (!buf || !dmom) return status;
    T* v[3] = {buf, buf + fs * nr, buf + 2 * fs * nr};
    const size_t ss = (size_t)ctx->max_blocks * 2;
    // v0 and mu_0
    k_copy_norms<T><<<dim3(capped_grid(ctx, ctx->g.V, kBlock), nr), kBlock, 0, st>>>(fields64, v[0], fs, ctx->g.V,
                                                                   red_slot_partials(ctx, kSlotCheb), red_slot_counter(ctx, kSlotCheb),
                                                                   red_slot_out(ctx, kSlotCheb), ss); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    RM_CHECK(ctx, cudaMemcpyAsync(dmom, red_slot_out(ctx, kSlotCheb), sizeof(double) * 8 * nr, cudaMemcpyDeviceToDevice, st));
    const int K = (N + 1) / 2;
    for (int k = 1; k <= K; k++) {
        // v_k from v_{k-1} (and v_{k-2}); dots <v_k, v_k>, <v_k, v_{k-1}>
        T* out = v[k % 3];
        const T* in = v[(k - 1) % 3];
        const T* w = k >= 2 ? v[(k - 2) % 3] : nullptr;
        RM_TRY(launch_lap(ctx, prec, 18, in, out, nr, 0.0, k == 1 ? -0.125 : -0.25, w, -1.0, kSlotCheb, st));
        RM_CHECK(ctx, cudaMemcpyAsync(dmom + (size_t)8 * nr * k, red_slot_out(ctx, kSlotCheb), sizeof(double) * 8 * nr,
                                      cudaMemcpyDeviceToDevice, st));
    }
    std::vector<double> h((size_t)8 * nr * (K + 1));
    for (size_t off = 0; off < h.size(); off += kPinned) {
        const int cnt = (int)std::min<size_t>(kPinned, h.size() - off);
        RM_TRY(fetch(ctx, dmom + off, h.data() + off, cnt, st));
    }
    mu.assign((size_t)nr * (N + 1), 0.0);
    for (int f = 0; f < nr; f++) {
        double* m = mu.data() + (size_t)f * (N + 1);
        m[0] = h[(size_t)8 * f];
        for (int k = 1; k <= K; k++) {
            const double vv = h[(size_t)8 * nr * k + 8 * f], vw = h[(size_t)8 * nr * k + 8 * f + 1];
            if (k == 1) {
                if (N >= 1) m[1] = vw;
                if (N >= 2) m[2] = 2.0 * vv - m[0];
            } else {
                if (2 * k - 1 <= N) m[2 * k - 1] = 2.0 * vw - m[1];
                if (2 * k <= N) m[2 * k] = 2.0 * vv - m[0];
            }
        }
    }
    return RMHMC_OK;
}

// y (float64) += c x (x in the recurrence precision), grid-stride
template <typename T>
__global__ void k_accum64(const T* __restrict__ x, double c, double* __restrict__ y, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = fma(c, (double)x[i], y[i]);
}

// Y = sum_k coef[k] T_k(2A - 1) F by the forward recurrence, accumulating every term in float64
template <typename T>
static int filter_run(rmhmc_ctx* ctx, const double* F, int nf, int N, const double* coef, int prec, double* Y,
                      cudaStream_t st) {
    int status = RMHMC_OK;
    const size_t fs = field_elems(ctx), n = fs * nf;
    const bool f32 = sizeof(T) == 4;
    T* buf = (T*)workspace(ctx, f32 ? "cf_v32" : "cf_v64", sizeof(T) * n * 3, &status);
    if (!buf) return status;
    T* v[3] = {buf, buf + n, buf + 2 * n};
    if (f32) RM_TRY(to_float(ctx, F, (float*)v[0], n, st));
    else RM_CHECK(ctx, cudaMemcpyAsync(v[0], F, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    const int grid = capped_grid(ctx, n, kBlock);
    RM_CHECK(ctx, cudaMemsetAsync(Y, 0, sizeof(double) * n, st));
    k_accum64<T><<<grid, kBlock, 0, st>>>(v[0], coef[0], Y, n); ++ctx->launches;
    for (int k = 1; k <= N; k++) {
        T* out = v[k % 3];
        const T* in = v[(k - 1) % 3];
        const T* w = k >= 2 ? v[(k - 2) % 3] : nullptr;
        RM_TRY(launch_lap(ctx, prec, 18, in, out, nf, 0.0, k == 1 ? -0.125 : -0.25, w, -1.0, -1, st));
        k_accum64<T><<<grid, kBlock, 0, st>>>(out, coef[k], Y, n); ++ctx->launches;
    }
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}

}  // namespace rm

using namespace rm;

extern "C" int cheb_window_coeffs(int nwin, const double* edges, int degree, int kernel, double* C) {
    if (nwin < 1 || !edges || !C || degree < 0 || degree > 20000) return RMHMC_EINVAL;
    if (kernel != RMHMC_KERNEL_NONE && kernel != RMHMC_KERNEL_JACKSON) return RMHMC_EINVAL;
    for (int w = 0; w < nwin; w++)
        if (!(edges[w] < edges[w + 1]) || edges[w] < 0.0 || edges[w + 1] > 1.0) return RMHMC_EINVAL;
    std::vector<double> c;
    window_coefficients(edges, nwin, degree, kernel == RMHMC_KERNEL_JACKSON, c);
    memcpy(C, c.data(), sizeof(double) * c.size());
    return RMHMC_OK;
}

extern "C" int cheb_filter_apply(rmhmc_ctx* ctx, const double* U, const double* F, int nfield, int degree,
                                 const double* coef, int prec, double* Y, cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (!F || !Y || !coef || nfield < 1) return set_err(ctx, RMHMC_EINVAL, "cheb_filter_apply: bad fields");
    if (degree < 0 || degree > 20000) return set_err(ctx, RMHMC_EINVAL, "cheb_filter_apply: degree in [0, 20000]");
    if (prec != RMHMC_FP64 && prec != RMHMC_MIXED) return set_err(ctx, RMHMC_EINVAL, "cheb_filter_apply: bad prec");
    if ((uintptr_t)F % 16 || (uintptr_t)Y % 16) return set_err(ctx, RMHMC_EINVAL, "cheb_filter_apply: misaligned field");
    RM_TRY(ensure_links(ctx, U, stream));
    if (prec == RMHMC_FP64) return filter_run<double>(ctx, F, nfield, degree, coef, prec, Y, stream);
    return filter_run<float>(ctx, F, nfield, degree, coef, prec, Y, stream);
}

extern "C" int cheb_filter_spectrum(rmhmc_ctx* ctx, const double* U, const double* F, int nF, const double* noise,
                                    int nnoise, uint64_t seed, int degree, int nwin, const double* edges, int kernel,
                                    int prec, double* spec, double* num, double* tr, double* moments, cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if ((nF > 0 && !F) || nF < 0 || nnoise < 0) return set_err(ctx, RMHMC_EINVAL, "cheb_filter_spectrum: bad fields");
    if (nF + nnoise < 1 || nF + nnoise > kRedSlots - kSlotCheb)
        return set_err(ctx, RMHMC_EINVAL, "cheb_filter_spectrum: 1..%d fields per call", kRedSlots - kSlotCheb);
    if (degree < 0 || degree > 20000) return set_err(ctx, RMHMC_EINVAL, "cheb_filter_spectrum: degree in [0, 20000]");
    if (nwin < 0 || (nwin > 0 && !edges)) return set_err(ctx, RMHMC_EINVAL, "cheb_filter_spectrum: bad windows");
    if (nwin > 0 && nnoise == 0) return set_err(ctx, RMHMC_EINVAL, "cheb_filter_spectrum: the trace needs noise fields");
    for (int w = 0; w < nwin; w++)
        if (!(edges[w] < edges[w + 1]) || edges[w] < 0.0 || edges[w + 1] > 1.0)
            return set_err(ctx, RMHMC_EINVAL, "cheb_filter_spectrum: edges must increase within [0,1]");
    if (kernel != RMHMC_KERNEL_NONE && kernel != RMHMC_KERNEL_JACKSON) return set_err(ctx, RMHMC_EINVAL, "bad kernel");
    if (prec != RMHMC_FP64 && prec != RMHMC_MIXED) return set_err(ctx, RMHMC_EINVAL, "cheb_filter_spectrum: bad prec");
    RM_TRY(ensure_links(ctx, U, stream));
    const int nr = nF + nnoise;
    const size_t fs = field_elems(ctx);
    int status = RMHMC_OK;
    // gather the fields (forces first, then noise) into one float64 array
    double* all = (double*)workspace(ctx, "cb_in", sizeof(double) * fs * nr, &status);
    if (!all) return status;
    if (nF > 0) RM_CHECK(ctx, cudaMemcpyAsync(all, F, sizeof(double) * fs * nF, cudaMemcpyDeviceToDevice, stream));
    if (nnoise > 0) {
        if (noise) {
            RM_CHECK(ctx, cudaMemcpyAsync(all + fs * nF, noise, sizeof(double) * fs * nnoise, cudaMemcpyDeviceToDevice, stream));
        } else {
            k_gauss_fields<<<dim3(site_blocks(ctx), nnoise), kBlock, 0, stream>>>(all + fs * nF, fs, ctx->g.V, seed, 2u); ++ctx->launches;
            RM_LAUNCH_CHECK(ctx);
        }
    }
    std::vector<double> mu;
    if (prec == RMHMC_FP64) RM_TRY(cheb_run<double>(ctx, all, nr, degree, prec, mu, stream));
    else RM_TRY(cheb_run<float>(ctx, all, nr, degree, prec, mu, stream));
    if (moments) memcpy(moments, mu.data(), sizeof(double) * mu.size());
    if (nwin == 0) return RMHMC_OK;
    std::vector<double> C;
    window_coefficients(edges, nwin, degree, kernel == RMHMC_KERNEL_JACKSON, C);
    std::vector<double> trw(nwin, 0.0);
    for (int w = 0; w < nwin; w++) {
        for (int e = 0; e < nnoise; e++) {
            double s = 0.0;
            for (int k = 0; k <= degree; k++) s += C[(size_t)w * (degree + 1) + k] * mu[(size_t)(nF + e) * (degree + 1) + k];
            trw[w] += s;
        }
        trw[w] /= nnoise;
        if (tr) tr[w] = trw[w];
    }
    for (int f = 0; f < nF; f++)
        for (int w = 0; w < nwin; w++) {
            double s = 0.0;
            for (int k = 0; k <= degree; k++) s += C[(size_t)w * (degree + 1) + k] * mu[(size_t)f * (degree + 1) + k];
            if (num) num[(size_t)f * nwin + w] = s;
            if (spec) spec[(size_t)f * nwin + w] = s / trw[w];
        }
    return RMHMC_OK;
}
