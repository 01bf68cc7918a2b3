// Krylov engine (see krylov.cuh) for the rational mass term of Sec. 3, Eq. (6): the shifted solves
// (A + sigma_j)^{-1} b of R(A) = c + sum_j alpha_j / (A + sigma_j) by CG on the smallest shift keeping
// the residual basis in HBM, Lanczos post-processing on the host, basis combinations, float64 reliable
// updates.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "krylov.cuh"
#include "ops.cuh"
#include "stencil.cuh"
#include "tune.cuh"

namespace rm {

constexpr int kCheckChunk = 8;                                                 // iterations per flag check
constexpr int kMaxCombine = 32;                                                // outputs per combine launch

// ------------------------------------------------------------------------------------------------
// elementwise field kernels (one thread per site, 32 reals)
// ------------------------------------------------------------------------------------------------
// flat vector access: element i of a field as the i-th float4 (float) or double2 (double)
template <typename T> struct Vec;
template <> struct Vec<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ __forceinline__ static void get(const type& v, float* x) { x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w; }
    __device__ __forceinline__ static type make(const float* x) { return make_float4(x[0], x[1], x[2], x[3]); }
};
template <> struct Vec<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ __forceinline__ static void get(const type& v, double* x) { x[0] = v.x; x[1] = v.y; }
    __device__ __forceinline__ static type make(const double* x) { return make_double2(x[0], x[1]); }
};

// r_0 = b, rho_0 = |b|^2 (one vector element per thread, coalesced)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_start(const T* __restrict__ b, T* __restrict__ r0, size_t nvec, int* flags,
                                                     double* rho, double* partials, unsigned* counter) {
    __shared__ double sh[kBlock / 32];
    using VT = Vec<T>;
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += (size_t)gridDim.x * blockDim.x) {
        const typename VT::type v = reinterpret_cast<const typename VT::type*>(b)[i];
        reinterpret_cast<typename VT::type*>(r0)[i] = v;
        T x[VT::n];
        VT::get(v, x);
#pragma unroll
        for (int k = 0; k < VT::n; k++) acc += (double)x[k] * (double)x[k];
    }
    double v[1] = {acc};
    block_sum<1>(v, sh);
    {
        double out[1];
        if (grid_sum_finish<1>(v, partials, counter, out, gridDim.x, blockIdx.x, sh)) {
            rho[0] = out[0];
            flags[1] = 0;
            flags[0] = isfinite(out[0]) ? (out[0] == 0.0 ? 1 : 0) : 3;
        }
    }
}

// CG without the search direction: q_k = (A + sigma0) p_k is carried as q_k = (A + sigma0) r_k + beta_{k-1} q_{k-1}
// (p_k = r_k + beta_{k-1} p_{k-1}), so the stencil reads only r_k; gamma_k = <p_k, A p_k> = <r_k, q_k> by
// A-conjugacy of the directions, alpha_k = rho_k / gamma_k.  q is updated in place at the lane's own site.
template <typename T, int LF, int NMU>
__global__ void __launch_bounds__(kBlockMax, (stencil_min_blocks<T, NMU>())) k_cg_A(Geom g, typename LinksOf<T>::type U, const T* __restrict__ R, size_t fs,
                                                     T* __restrict__ q, T diag, const int* __restrict__ flags,
                                                     double* vals, int maxit, double* partials, unsigned* counter) {
    constexpr int NC = NMU == 0 ? 1 : NMU;   // components per lane
    constexpr int LPS = 4 / NC;
    __shared__ double sh[kBlockMax / 32];
    if (flags[0]) return;
    const int k = flags[1];
    const T* r = R + (size_t)k * fs;
    const double* rho = vals;
    double* gamma = vals + (maxit + 1);
    double* alpha = gamma + maxit;
    const double* beta = alpha + maxit;
    const T b = k > 0 ? (T)beta[k - 1] : T(0);
    T dot = T(0);
    const int nlane = g.V * LPS;
    for (int lane = blockIdx.x * blockDim.x + threadIdx.x; lane < nlane; lane += gridDim.x * blockDim.x) {
        const int s = lane / LPS, mu0 = (lane % LPS) * NC;
        herm<T> acc[NC];
        if constexpr (sizeof(T) == 4 && NMU == 1) hop_sum_shape<T, LF, NMU>(g, U, s, mu0, SrcFieldV8{r}, acc);
        else hop_sum_shape<T, LF, NMU>(g, U, s, mu0, SrcField<T>{r}, acc);
#pragma unroll
        for (int m = 0; m < NC; m++) {
            const int mu = mu0 + m;
            T h[8], x[8], y[8];
            herm2_to_coef_tl(acc[m], h);
            if constexpr (sizeof(T) == 4 && NMU == 1) load8_v8(r + (size_t)s * 32 + mu * 8, x);
            else load8(r + (size_t)s * 32 + mu * 8, x);
            T* qs = q + (size_t)s * 32 + mu * 8;
            if (k > 0) {
                load8(qs, y);
#pragma unroll
                for (int a = 0; a < 8; a++) y[a] = fma(b, y[a], fma(T(-0.0625), h[a], diag * x[a]));
            } else {
#pragma unroll
                for (int a = 0; a < 8; a++) y[a] = fma(T(-0.0625), h[a], diag * x[a]);
            }
#pragma unroll
            for (int a = 0; a < 8; a++) dot = fma(x[a], y[a], dot);
            store8(qs, y);
        }
    }
    double v[1] = {0.0};
    if (sizeof(T) == 4) {
        float fv[1] = {(float)dot};
        block_sum_f<1>(fv, sh);
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
            v[0] = t;
        }
    } else {
        v[0] = (double)dot;
        block_sum<1>(v, sh);
    }
    {
        double out[1];
        if (grid_sum_finish<1>(v, partials, counter, out, gridDim.x, blockIdx.x, sh)) {
            gamma[k] = out[0];
            alpha[k] = rho[k] / out[0];
        }
    }
}

template <typename T, int NMU>
static void launch_cg_A(rmhmc_ctx* ctx, const StencilShape& shp, typename LinksOf<T>::type U, T* R, size_t fs, T* q,
                        T diag, int* flags, double* vals, int maxit, cudaStream_t st) {
    k_cg_A<T, 18, NMU><<<stencil_blocks(ctx, shp), shp.block, 0, st>>>(ctx->g, U, R, fs, q, diag, flags, vals, maxit,
                                                                      red_slot_partials(ctx, 0), red_slot_counter(ctx, 0));
    ++ctx->launches;
}

// the CG stencil in a tuned shape: 3x3 gather kernels (nmu 1, 2, 4, 0) or, in float32, the link-centric
// adjoint kernel (nmu 8, lap_lc.cu)
template <typename T>
static int cg_stencil(rmhmc_ctx* ctx, const StencilShape& shp, typename LinksOf<T>::type U, T* R, size_t fs, T* q, T diag,
                      int* flags, double* vals, int maxit, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (shp.nmu == 8)
            return launch_cg_lc(ctx, R, q, diag, flags, vals, maxit, red_slot_partials(ctx, 0), red_slot_counter(ctx, 0), st);
    }
    if (shp.nmu == 4) launch_cg_A<T, 4>(ctx, shp, U, R, fs, q, diag, flags, vals, maxit, st);
    else if (shp.nmu == 2) launch_cg_A<T, 2>(ctx, shp, U, R, fs, q, diag, flags, vals, maxit, st);
    else if (shp.nmu == 0) launch_cg_A<T, 0>(ctx, shp, U, R, fs, q, diag, flags, vals, maxit, st);
    else launch_cg_A<T, 1>(ctx, shp, U, R, fs, q, diag, flags, vals, maxit, st);
    return RMHMC_OK;
}

// Launch shape of the CG stencil, tuned on its own (its loads differ from the plain stencil's: it also reads
// and writes q, and the one-component shape reads the basis with 256-bit loads): every shape is timed on the
// context's lattice (k = 0 on zeroed scratch, three repetitions after a warm-up) at first use.
template <typename T>
static int cg_shape(rmhmc_ctx* ctx, cudaStream_t st, StencilShape& out) {
    const int key = 10000 + (int)sizeof(T) * 100 + 18;
    auto it = ctx->tune.find(key);
    if (it != ctx->tune.end()) {
        out.nmu = it->second.first;
        out.block = it->second.second;
        return RMHMC_OK;
    }
    StencilShape base;
    RM_TRY((stencil_shape<T, 18>(ctx, st, base)));
    int status = RMHMC_OK;
    const size_t fs = field_elems(ctx);
    T* X = (T*)workspace(ctx, "tune_x", sizeof(double) * fs, &status);
    T* Y = (T*)workspace(ctx, "tune_y", sizeof(double) * fs, &status);
    int* flags = (int*)workspace(ctx, "tune_cgflags", 64, &status);
    double* vals = (double*)workspace(ctx, "tune_cgvals", 64, &status);
    if (!X || !Y || !flags || !vals) return status;
    RM_CHECK(ctx, cudaMemsetAsync(X, 0, sizeof(T) * fs, st));
    RM_CHECK(ctx, cudaMemsetAsync(flags, 0, 64, st));
    RM_CHECK(ctx, cudaMemsetAsync(vals, 0, 64, st));
    typename LinksOf<T>::type U;
    if constexpr (sizeof(T) == 8) U = links64(ctx); else U = links32(ctx);
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
            auto run = [&]() { return cg_stencil<T>(ctx, shp, U, X, fs, Y, T(1), flags, vals, 1, st); };
            RM_TRY(run());
            RM_CHECK(ctx, cudaEventRecord(e0, st));
            for (int r = 0; r < 3; r++) RM_TRY(run());
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
    snprintf(line, sizeof line, "; cg %s -> nmu %d block %d [", sizeof(T) == 8 ? "fp64" : "fp32", bs.nmu, bs.block);
    ctx->tune_report += line + rep + "]";
    out = bs;
    return RMHMC_OK;
}

// r_{k+1} = r_k - alpha_k q_k ; rho_{k+1} = |r_{k+1}|^2 ; beta_k ; convergence flags; k advances
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_B(T* __restrict__ R, size_t fs, const T* __restrict__ q, size_t nvec,
                                                  int* flags, double* vals, int maxit, double tol2, double* partials,
                                                  unsigned* counter) {
    __shared__ double sh[kBlock / 32];
    if (flags[0]) return;
    const int k = flags[1];
    double* rho = vals;
    const double* gamma = vals + (maxit + 1);
    const double* alpha = gamma + maxit;
    double* beta = (double*)(alpha + maxit);
    using VT = Vec<T>;
    const T a = (T)alpha[k];
    T dot = T(0);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += (size_t)gridDim.x * blockDim.x) {
        T x[VT::n], y[VT::n];
        VT::get(reinterpret_cast<const typename VT::type*>(R + (size_t)k * fs)[i], x);
        VT::get(reinterpret_cast<const typename VT::type*>(q)[i], y);
#pragma unroll
        for (int c = 0; c < VT::n; c++) {
            x[c] = fma(-a, y[c], x[c]);
            dot = fma(x[c], x[c], dot);
        }
        reinterpret_cast<typename VT::type*>(R + (size_t)(k + 1) * fs)[i] = VT::make(x);
    }
    double v[1] = {0.0};
    if (sizeof(T) == 4) {
        float fv[1] = {(float)dot};
        block_sum_f<1>(fv, sh);
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kBlock / 32; w++) t += sh[w];
            v[0] = t;
        }
    } else {
        v[0] = (double)dot;
        block_sum<1>(v, sh);
    }
    {
        double out[1];
        if (grid_sum_finish<1>(v, partials, counter, out, gridDim.x, blockIdx.x, sh)) {
            const double rr = out[0];
            rho[k + 1] = rr;
            beta[k] = rr / rho[k];
            flags[1] = k + 1;
            if (!isfinite(rr) || !isfinite(alpha[k]))
                flags[0] = 3;
            else if (rr <= tol2 * rho[0])
                flags[0] = 1;
            else if (k + 1 >= maxit)
                flags[0] = 2;
        }
    }
}

// out[m] = sum_{k < n} coef[m][k] basis_k for m < M <= MB.  Every coefficient is staged in shared memory
// once per block; the grid strides over vectors of 16 bytes (float4 / double2) so every basis vector is
// read with 128-bit loads, four vectors in flight per step.  n is read from flags[1] when flags is given
// (device-decided Krylov length); coefficient row stride ldc.
template <typename T, typename TO>
struct OutPtrs { TO* p[kMaxCombine]; };

template <typename T> __device__ __forceinline__ void store_vec(T* p, const T* x);
template <> __device__ __forceinline__ void store_vec<float>(float* p, const float* x) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
template <> __device__ __forceinline__ void store_vec<double>(double* p, const double* x) {
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
}

template <typename T, typename TO, int MB>
__global__ void __launch_bounds__(kBlock) k_combine(const T* __restrict__ R, size_t fs, const int* __restrict__ flags, int n,
                                                     const double* __restrict__ coef, int ldc, int M, OutPtrs<T, TO> outs) {
    using VT = Vec<T>;
    constexpr int VN = VT::n, UN = 4;
    __shared__ T cs[MB * kBasisCap];
    if (flags) n = flags[1];
    for (int t = threadIdx.x; t < M * n; t += blockDim.x) {
        const int m = t / n, k = t - m * n;
        cs[m * kBasisCap + k] = (T)coef[(size_t)m * ldc + k];
    }
    __syncthreads();
    const size_t nvec = fs / VN;
    const typename VT::type* Rv = reinterpret_cast<const typename VT::type*>(R);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += (size_t)gridDim.x * blockDim.x) {
        T acc[MB][VN];
#pragma unroll
        for (int m = 0; m < MB; m++)
#pragma unroll
            for (int v = 0; v < VN; v++) acc[m][v] = T(0);
        int k = 0;
        for (; k + UN <= n; k += UN) {
            T x[UN][VN];
#pragma unroll
            for (int u = 0; u < UN; u++) VT::get(__ldg(Rv + (size_t)(k + u) * nvec + i), x[u]);
#pragma unroll
            for (int u = 0; u < UN; u++)
#pragma unroll
                for (int m = 0; m < MB; m++)
                    if (m < M) {
                        const T c = cs[m * kBasisCap + k + u];
#pragma unroll
                        for (int v = 0; v < VN; v++) acc[m][v] = fma(c, x[u][v], acc[m][v]);
                    }
        }
        for (; k < n; k++) {
            T x[VN];
            VT::get(__ldg(Rv + (size_t)k * nvec + i), x);
#pragma unroll
            for (int m = 0; m < MB; m++)
                if (m < M) {
                    const T c = cs[m * kBasisCap + k];
#pragma unroll
                    for (int v = 0; v < VN; v++) acc[m][v] = fma(c, x[v], acc[m][v]);
                }
        }
#pragma unroll
        for (int m = 0; m < MB; m++)
            if (m < M) {
                TO o[VN];
#pragma unroll
                for (int v = 0; v < VN; v++) o[v] = (TO)acc[m][v];
                TO* dst = outs.p[m] + i * VN;
                if (sizeof(TO) == sizeof(T)) store_vec<TO>(dst, o);
                else {
#pragma unroll
                    for (int v = 0; v < VN; v += 16 / (int)sizeof(TO)) store_vec<TO>(dst + v, o + v);
                }
            }
    }
}

// r_f = b - (A + sigma_f) x_f, float64, with per-field squared norms
template <int LF>
__global__ void __launch_bounds__(kBlock) k_resid64(Geom g, Links64 U, const double* __restrict__ b, const double* __restrict__ x,
                                                     const double* __restrict__ sig, double* __restrict__ r, size_t fs,
                                                     double* partials, unsigned* counters, double* out, size_t slot_stride) {
    __shared__ double sh[kBlock / 32];
    const int f = blockIdx.y;
    const double* xf = x + f * fs;
    const double diag = 0.5 + sig[f];
    double nrm = 0.0;
    for (int lane = blockIdx.x * blockDim.x + threadIdx.x; lane < g.V * 4; lane += gridDim.x * blockDim.x) {
        const int s = lane >> 2, mu = lane & 3;
        herm<double> acc;
        hop_sum1<double, LF>(g, U, s, mu, SrcField<double>{xf}, acc);
        double h[8], xx[8], bb[8], y[8];
        herm2_to_coef_tl(acc, h);
        load8(xf + (size_t)s * 32 + mu * 8, xx);
        load8(b + (size_t)s * 32 + mu * 8, bb);
#pragma unroll
        for (int a = 0; a < 8; a++) {
            y[a] = bb[a] - (diag * xx[a] - 0.0625 * h[a]);
            nrm = fma(y[a], y[a], nrm);
        }
        if (r) store8(r + f * fs + (size_t)s * 32 + mu * 8, y);
    }
    double v[1] = {nrm};
    block_sum<1>(v, sh);
    grid_sum_finish<1>(v, partials + f * slot_stride, counters + f, out + (size_t)f * 8, gridDim.x, blockIdx.x, sh);
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}
__global__ void k_add_f2d(const float* __restrict__ in, double* __restrict__ out, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] += (double)in[i];
}
__global__ void k_axpby64(double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                          double* __restrict__ out, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}
__global__ void k_norm2_64(const double* __restrict__ x, size_t n, double* partials, unsigned* counter, double* out) {
    __shared__ double sh[kBlock / 32];
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc = fma(x[i], x[i], acc);
    double v[1] = {acc};
    block_sum<1>(v, sh);
    grid_sum_finish<1>(v, partials, counter, out, gridDim.x, blockIdx.x, sh);
}

static int elem_grid(const rmhmc_ctx* ctx, size_t n) {
    size_t b = (n + kBlock - 1) / kBlock;
    const size_t cap = (size_t)ctx->num_sms * 16;
    return (int)std::max<size_t>(1, std::min(b, cap));
}

int to_float(rmhmc_ctx* ctx, const double* in, float* out, size_t n, cudaStream_t st) {
    k_to_float<<<elem_grid(ctx, n), kBlock, 0, st>>>(in, out, n); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}
int add_float_to_double(rmhmc_ctx* ctx, const float* in, double* out, size_t n, cudaStream_t st) {
    k_add_f2d<<<elem_grid(ctx, n), kBlock, 0, st>>>(in, out, n); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}
int axpby64(rmhmc_ctx* ctx, double a, const double* x, double b, const double* y, double* out, size_t n, cudaStream_t st) {
    k_axpby64<<<elem_grid(ctx, n), kBlock, 0, st>>>(a, x, b, y, out, n); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}
int norm2_64(rmhmc_ctx* ctx, const double* x, size_t n, double* out, cudaStream_t st) {
    const int grid = std::min(elem_grid(ctx, n), ctx->max_blocks);
    k_norm2_64<<<grid, kBlock, 0, st>>>(x, n, red_slot_partials(ctx, kSlotNorm), red_slot_counter(ctx, kSlotNorm),
                                        red_slot_out(ctx, kSlotNorm)); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return fetch(ctx, red_slot_out(ctx, kSlotNorm), out, 1, st);
}

// ------------------------------------------------------------------------------------------------
// Lanczos tridiagonal matrix from the CG coefficients
//   A0 v_k = -(sqrt(beta_{k-1})/alpha_{k-1}) v_{k-1} + (1/alpha_k + beta_{k-1}/alpha_{k-1}) v_k
//            - (sqrt(beta_k)/alpha_k) v_{k+1},   v_k = r_k / |r_k|
// ------------------------------------------------------------------------------------------------
void Tridiag::build(const KrylovResult& kr) {
    n = kr.n;
    d.assign(n, 0.0);
    e.assign(n > 0 ? n - 1 : 0, 0.0);
    inv_norm.assign(n, 0.0);
    bnorm = sqrt(kr.rho[0]);
    for (int k = 0; k < n; k++) {
        d[k] = 1.0 / kr.alpha[k] + (k > 0 ? kr.beta[k - 1] / kr.alpha[k - 1] : 0.0);
        if (k < n - 1) e[k] = -sqrt(kr.beta[k]) / kr.alpha[k];
        inv_norm[k] = 1.0 / sqrt(kr.rho[k]);
    }
}

void Tridiag::solve(double shift, const std::vector<double>& rhs, std::vector<double>& y) const {
    // Thomas algorithm (T + shift is symmetric positive definite)
    std::vector<double> c(n), dd(n);
    y.assign(n, 0.0);
    if (n == 0) return;
    double den = d[0] + shift;
    c[0] = n > 1 ? e[0] / den : 0.0;
    dd[0] = rhs[0] / den;
    for (int k = 1; k < n; k++) {
        den = d[k] + shift - e[k - 1] * c[k - 1];
        c[k] = k < n - 1 ? e[k] / den : 0.0;
        dd[k] = (rhs[k] - e[k - 1] * dd[k - 1]) / den;
    }
    y[n - 1] = dd[n - 1];
    for (int k = n - 2; k >= 0; k--) y[k] = dd[k] - c[k] * y[k + 1];
}

void Tridiag::to_basis(const std::vector<double>& y, double* row) const {
    for (int k = 0; k < n; k++) row[k] = y[k] * inv_norm[k];
}

// ------------------------------------------------------------------------------------------------
// the CG run
// ------------------------------------------------------------------------------------------------
struct KWork {
    void* basis = nullptr;
    void* q = nullptr;
    int* flags = nullptr;
    double* vals = nullptr;
    double* coef = nullptr;
    int maxit = 0;
};
// the stored basis holds at most kBasisCap residuals: longer runs stop there and the caller's
// reliable-update loop continues from the true residual (a restart)

template <typename T>
static int krylov_workspace(rmhmc_ctx* ctx, int maxit, KWork& w) {
    int status = RMHMC_OK;
    const size_t fb = field_elems(ctx) * sizeof(T);
    const bool f32 = sizeof(T) == 4;
    // always the full capacity, so that the basis never moves under a captured graph
    w.basis = workspace(ctx, f32 ? "kr_basis32" : "kr_basis64", fb * (size_t)(kBasisCap + 1), &status);
    if (!w.basis) return status;
    w.q = workspace(ctx, f32 ? "kr_q32" : "kr_q64", fb, &status);
    void* sc = workspace(ctx, "kr_scal", 64 + sizeof(double) * 4 * (size_t)(kBasisCap + 2), &status);
    if (!w.q || !sc) return status;
    w.flags = (int*)sc;
    w.vals = (double*)((char*)sc + 64);
    w.maxit = maxit;
    return RMHMC_OK;
}

template <typename T>
T* krylov_basis(rmhmc_ctx* ctx) {
    auto it = ctx->bufs.find(sizeof(T) == 4 ? "kr_basis32" : "kr_basis64");
    return it == ctx->bufs.end() ? nullptr : (T*)it->second.p;
}

template <typename T>
int krylov_run(rmhmc_ctx* ctx, const T* b, double sigma0, double tol, int maxit, KrylovResult& out, cudaStream_t st) {
    if (maxit < 1) return set_err(ctx, RMHMC_EINVAL, "maxiter must be >= 1");
    if (!(sigma0 > 0.0)) return set_err(ctx, RMHMC_EINVAL, "shifts must be > 0");
    maxit = std::min(maxit, kBasisCap);
    KWork w;
    RM_TRY(krylov_workspace<T>(ctx, maxit, w));
    const size_t fs = field_elems(ctx);
    const size_t nvec = fs / Vec<T>::n;
    T* R = (T*)w.basis;
    const int nb = capped_grid(ctx, nvec, kBlock);
    StencilShape shp;
    RM_TRY(cg_shape<T>(ctx, st, shp));
    k_cg_start<T><<<nb, kBlock, 0, st>>>(b, R, nvec, w.flags, w.vals, red_slot_partials(ctx, kSlotRho),
                                         red_slot_counter(ctx, kSlotRho)); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    typename LinksOf<T>::type U;
    if constexpr (sizeof(T) == 8) U = links64(ctx); else U = links32(ctx);
    const T diag = (T)(0.5 + sigma0);
    const double tol2 = tol * tol;
    // iteration count of the previous run of the same operator and tolerance: the first chunk of launches
    // covers it, so a converged run usually stops after one host check
    char key[96];
    snprintf(key, sizeof key, "%d:%.17g:%.17g:%d", (int)sizeof(T), sigma0, tol, maxit);
    int& pred = ctx->kr_pred[key];
    int* hflags = (int*)(ctx->h_pinned + kPinned - 16);
    cudaEvent_t* ev = ctx->kr_ev;
    int launched = 0, chunk = 0;
    bool stop = false;
    while (launched < maxit && !stop) {
        const int len = chunk == 0 ? (pred > 0 ? pred : kCheckChunk) : kCheckChunk / 2;
        const int k1 = std::min(maxit, launched + len);
        for (int k = launched; k < k1; k++) {
            const bool timed = ctx->prof && k < kProfEvents;
            if (timed) RM_CHECK(ctx, cudaEventRecord(ctx->prof_ev[2 * k], st));
            // the solver streams 18-real links, in the tuned launch shape
            RM_TRY(cg_stencil<T>(ctx, shp, U, R, fs, (T*)w.q, diag, w.flags, w.vals, maxit, st));
            if (timed) RM_CHECK(ctx, cudaEventRecord(ctx->prof_ev[2 * k + 1], st));
            k_cg_B<T><<<nb, kBlock, 0, st>>>(R, fs, (const T*)w.q, nvec, w.flags, w.vals, maxit, tol2,
                                             red_slot_partials(ctx, kSlotRho), red_slot_counter(ctx, kSlotRho)); ++ctx->launches;
        }
        launched = k1;
        RM_LAUNCH_CHECK(ctx);
        const int slot = chunk & 1;
        RM_CHECK(ctx, cudaMemcpyAsync(hflags + 2 * slot, w.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        RM_CHECK(ctx, cudaEventRecord(ev[slot], st));
        if (chunk == 0) {
            // the predicted length: check at once
            RM_CHECK(ctx, cudaEventSynchronize(ev[slot]));
            if (hflags[2 * slot] != 0) stop = true;
        } else if (chunk > 1) {
            // inspect the previous chunk's flags while this chunk runs
            RM_CHECK(ctx, cudaEventSynchronize(ev[slot ^ 1]));
            if (hflags[2 * (slot ^ 1)] != 0) stop = true;
        }
        chunk++;
    }
    RM_CHECK(ctx, cudaMemcpyAsync(hflags, w.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    RM_CHECK(ctx, cudaStreamSynchronize(st));
    out.status = hflags[0];
    out.n = hflags[1];
    pred = out.n;
    ctx->krylov_iters += out.n;
    if (ctx->prof) {
        // durations of the stencil launches that did work (iterations 0 .. n-1)
        for (int k = 0; k < std::min(out.n, kProfEvents); k++) {
            float ms = 0.f;
            RM_CHECK(ctx, cudaEventElapsedTime(&ms, ctx->prof_ev[2 * k], ctx->prof_ev[2 * k + 1]));
            ctx->prof_ms += ms;
            ctx->prof_count++;
        }
    }
    if (out.status == 0) out.status = 2;   // ran out of iterations without a flag (maxit reached)
    const int n = out.n;
    // rho[0..n], alpha[0..n-1], beta[0..n-1] in one transfer of the scalar block
    const int nvals = (maxit + 1) + 3 * maxit;
    if (nvals > kPinned - 64) return set_err(ctx, RMHMC_EINVAL, "Krylov run too long for the staging area");
    std::vector<double> buf(nvals);
    RM_TRY(fetch(ctx, w.vals, buf.data(), nvals, st));
    out.rho.assign(buf.begin(), buf.begin() + n + 1);
    out.alpha.assign(buf.begin() + (maxit + 1) + maxit, buf.begin() + (maxit + 1) + maxit + n);
    out.beta.assign(buf.begin() + (maxit + 1) + 2 * maxit, buf.begin() + (maxit + 1) + 2 * maxit + n);
    if (out.status == 3) return set_err(ctx, RMHMC_ENAN, "NaN/Inf in the Krylov recurrence");
    return RMHMC_OK;
}

template <typename T, typename TO>
int krylov_combine(rmhmc_ctx* ctx, const CombineSpec& spec, TO* const* outs, cudaStream_t st) {
    if (spec.n == 0) {
        for (int m = 0; m < spec.M; m++) RM_CHECK(ctx, cudaMemsetAsync(outs[m], 0, field_elems(ctx) * sizeof(TO), st));
        return RMHMC_OK;
    }
    int status = RMHMC_OK;
    const T* R = krylov_basis<T>(ctx);
    const size_t fs = field_elems(ctx);
    constexpr int kChunk = 12;   // outputs per launch (accumulators per thread: 12 x one 16-byte vector)
    const size_t ncoef = std::max((size_t)kMaxCombine * kBasisCap, (size_t)spec.M * spec.n);
    double* dcoef = (double*)workspace(ctx, "kr_coef", sizeof(double) * ncoef, &status);
    if (!dcoef) return status;
    RM_TRY(upload(ctx, dcoef, spec.coef.data(), sizeof(double) * (size_t)spec.M * spec.n, st));
    const int grid = capped_grid(ctx, fs / Vec<T>::n, kBlock);
    for (int m0 = 0; m0 < spec.M; m0 += kChunk) {
        const int mc = std::min(kChunk, spec.M - m0);
        OutPtrs<T, TO> op{};
        for (int m = 0; m < mc; m++) op.p[m] = outs[m0 + m];
        const double* c = dcoef + (size_t)m0 * spec.n;
        if (mc == 1) k_combine<T, TO, 1><<<grid, kBlock, 0, st>>>(R, fs, nullptr, spec.n, c, spec.n, 1, op);
        else k_combine<T, TO, kChunk><<<grid, kBlock, 0, st>>>(R, fs, nullptr, spec.n, c, spec.n, mc, op);
        ++ctx->launches;
        RM_LAUNCH_CHECK(ctx);
    }
    return RMHMC_OK;
}

int resid64(rmhmc_ctx* ctx, const double* b, const double* x, int nf, const double* sigma, double* r, double* norm2,
            cudaStream_t st) {
    if (nf > kRedSlots - kSlotResid) return set_err(ctx, RMHMC_EINVAL, "too many shifts for one residual launch");
    int status = RMHMC_OK;
    double* dsig = (double*)workspace(ctx, "kr_sig", sizeof(double) * 64, &status);
    if (!dsig) return status;
    RM_TRY(upload(ctx, dsig, sigma, sizeof(double) * nf, st));
    const dim3 grid(capped_grid(ctx, (size_t)ctx->g.V * 4, kBlock), nf);
    k_resid64<18><<<grid, kBlock, 0, st>>>(ctx->g, links64(ctx), b, x, dsig, r, field_elems(ctx),
                                           red_slot_partials(ctx, kSlotResid), red_slot_counter(ctx, kSlotResid),
                                           red_slot_out(ctx, kSlotResid), (size_t)ctx->max_blocks * 2); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    std::vector<double> tmp((size_t)nf * 8);
    RM_TRY(fetch(ctx, red_slot_out(ctx, kSlotResid), tmp.data(), nf * 8, st));
    for (int f = 0; f < nf; f++) norm2[f] = tmp[(size_t)f * 8];
    return RMHMC_OK;
}

template int krylov_run<float>(rmhmc_ctx*, const float*, double, double, int, KrylovResult&, cudaStream_t);
template int krylov_run<double>(rmhmc_ctx*, const double*, double, double, int, KrylovResult&, cudaStream_t);
template float* krylov_basis<float>(rmhmc_ctx*);
template double* krylov_basis<double>(rmhmc_ctx*);
template int krylov_combine<float, float>(rmhmc_ctx*, const CombineSpec&, float* const*, cudaStream_t);
template int krylov_combine<float, double>(rmhmc_ctx*, const CombineSpec&, double* const*, cudaStream_t);
template int krylov_combine<double, double>(rmhmc_ctx*, const CombineSpec&, double* const*, cudaStream_t);

// ------------------------------------------------------------------------------------------------
// mass term parsing and the per-shift solve with float64 reliable updates
// ------------------------------------------------------------------------------------------------
int parse_mass(rmhmc_ctx* ctx, const rmhmc_mass* m, MassTerm& out) {
    if (!m) return set_err(ctx, RMHMC_EINVAL, "null mass term");
    if (m->npole < 0 || m->npole > 24) return set_err(ctx, RMHMC_EINVAL, "npole must be in [0, 24]");
    if (m->npole > 0 && (!m->alpha || !m->sigma)) return set_err(ctx, RMHMC_EINVAL, "null pole arrays");
    out.c = m->c;
    out.kappa = m->kappa;
    out.alpha.assign(m->alpha, m->alpha + m->npole);
    out.sigma.assign(m->sigma, m->sigma + m->npole);
    for (double s : out.sigma)
        if (!(s > 0.0)) return set_err(ctx, RMHMC_EINVAL, "every shift must be > 0");
    return RMHMC_OK;
}

static double min_shift(const std::vector<double>& s) { return *std::min_element(s.begin(), s.end()); }

// combination rows of the shifted solutions (T + Delta_j)^{-1} e1 |b|
static void shifted_rows(const Tridiag& tri, const std::vector<double>& sigma, double sigma0, CombineSpec& spec,
                         std::vector<std::vector<double>>* ys = nullptr) {
    const int n = tri.n, ns = (int)sigma.size();
    spec.n = n;
    spec.M = ns;
    spec.coef.assign((size_t)ns * n, 0.0);
    std::vector<double> e1(n, 0.0), y;
    if (n > 0) e1[0] = tri.bnorm;
    if (ys) ys->assign(ns, {});
    for (int j = 0; j < ns; j++) {
        tri.solve(sigma[j] - sigma0, e1, y);
        tri.to_basis(y, spec.coef.data() + (size_t)j * n);
        if (ys) (*ys)[j] = y;
    }
}

int solve_shifts(rmhmc_ctx* ctx, const MassTerm& m, const double* b, double tol, int maxiter, int prec, double* xs,
                 int* iters, double* resid, cudaStream_t st) {
    const int ns = m.npole();
    int total = 0;
    if (ns == 0) {
        if (iters) *iters = 0;
        return RMHMC_OK;
    }
    const size_t fs = field_elems(ctx);
    int status = RMHMC_OK;
    double b2 = 0.0;
    RM_TRY(norm2_64(ctx, b, fs, &b2, st));
    if (b2 == 0.0) {
        RM_CHECK(ctx, cudaMemsetAsync(xs, 0, sizeof(double) * fs * ns, st));
        if (resid) for (int j = 0; j < ns; j++) resid[j] = 0.0;
        if (iters) *iters = 0;
        return RMHMC_OK;
    }
    if (!isfinite(b2)) return set_err(ctx, RMHMC_ENAN, "NaN/Inf in the right-hand side");
    const double s0 = min_shift(m.sigma);
    const bool mixed = prec != RMHMC_FP64;
    const double floor32 = 1e-6;
    std::vector<double*> outs(ns);
    for (int j = 0; j < ns; j++) outs[j] = xs + (size_t)j * fs;
    // first pass: one Krylov space for every shift
    {
        KrylovResult kr;
        if (mixed) {
            float* b32 = (float*)workspace(ctx, "ss_b32", fs * sizeof(float), &status);
            if (!b32) return status;
            RM_TRY(to_float(ctx, b, b32, fs, st));
            RM_TRY(krylov_run<float>(ctx, b32, s0, std::max(0.5 * tol, floor32), maxiter, kr, st));
        } else {
            RM_TRY(krylov_run<double>(ctx, b, s0, 0.5 * tol, maxiter, kr, st));
        }
        total += kr.n;
        Tridiag tri;
        tri.build(kr);
        CombineSpec spec;
        shifted_rows(tri, m.sigma, s0, spec);
        if (mixed) RM_TRY((krylov_combine<float, double>(ctx, spec, outs.data(), st)));
        else RM_TRY((krylov_combine<double, double>(ctx, spec, outs.data(), st)));
        if (kr.status == 2 && !mixed) {
            // fall through to the refinement check, which reports ENOCONV if needed
        }
    }
    // reliable updates: true residuals to float64 accuracy, corrections per shift.  Mixed precision
    // forms them from float32 arithmetic with compensated sums (resid_df.cu) on the adjoint table of
    // the links, which stay fixed for the whole solve.
    double* r = !mixed ? (double*)workspace(ctx, "ss_r", sizeof(double) * fs * ns, &status) : nullptr;
    float* r32 = mixed ? (float*)workspace(ctx, "ss_r32", sizeof(float) * fs * ns, &status) : nullptr;
    float* e32 = mixed ? (float*)workspace(ctx, "ss_e32", sizeof(float) * fs, &status) : nullptr;
    double* e64 = !mixed ? (double*)workspace(ctx, "ss_e64", sizeof(double) * fs, &status) : nullptr;
    if ((mixed && (!r32 || !e32)) || (!mixed && (!r || !e64))) return status;
    float* adj = nullptr;
    if (mixed) RM_TRY(adjoint_table(ctx, &adj, st));
    std::vector<double> n2(ns);
    for (int cycle = 0;; cycle++) {
        if (mixed) RM_TRY(resid_df(ctx, adj, b, xs, ns, m.sigma.data(), r32, n2.data(), st));
        else RM_TRY(resid64(ctx, b, xs, ns, m.sigma.data(), r, n2.data(), st));
        bool all = true;
        for (int j = 0; j < ns; j++) {
            const double rel = sqrt(n2[j] / b2);
            if (resid) resid[j] = rel;
            if (!isfinite(rel)) return set_err(ctx, RMHMC_ENAN, "NaN/Inf in a true residual");
            if (rel > tol) all = false;
        }
        if (all) break;
        if (cycle >= 8 || total >= maxiter)
            return set_err(ctx, RMHMC_ENOCONV, "shifted solve did not reach %g after %d iterations", tol, total);
        for (int j = 0; j < ns; j++) {
            const double rel = sqrt(n2[j] / b2);
            if (rel <= tol) continue;
            const double want = std::max(0.5 * tol / rel, 1e-15);
            KrylovResult kr;
            if (mixed) {
                RM_TRY(krylov_run<float>(ctx, r32 + (size_t)j * fs, m.sigma[j], std::max(want, floor32), maxiter, kr,
                                         st));
            } else {
                RM_TRY(krylov_run<double>(ctx, r + (size_t)j * fs, m.sigma[j], want, maxiter, kr, st));
            }
            total += kr.n;
            Tridiag tri;
            tri.build(kr);
            CombineSpec spec;
            shifted_rows(tri, std::vector<double>{m.sigma[j]}, m.sigma[j], spec);
            if (mixed) {
                float* o[1] = {e32};
                RM_TRY((krylov_combine<float, float>(ctx, spec, o, st)));
                RM_TRY(add_float_to_double(ctx, e32, outs[j], fs, st));
            } else {
                double* o[1] = {e64};
                RM_TRY((krylov_combine<double, double>(ctx, spec, o, st)));
                RM_TRY(axpby64(ctx, 1.0, outs[j], 1.0, e64, outs[j], fs, st));
            }
        }
    }
    if (iters) *iters = total;
    return RMHMC_OK;
}

int rational_apply(rmhmc_ctx* ctx, const MassTerm& m, const double* b, double tol, int maxiter, int prec, double* Y,
                   int* iters, cudaStream_t st) {
    const size_t fs = field_elems(ctx);
    const int ns = m.npole();
    int status = RMHMC_OK;
    int it = 0;
    double* xs = nullptr;
    if (ns > 0) {
        xs = (double*)workspace(ctx, "ra_xs", sizeof(double) * fs * ns, &status);
        if (!xs) return status;
        RM_TRY(solve_shifts(ctx, m, b, tol, maxiter, prec, xs, &it, nullptr, st));
    }
    RM_TRY(axpby64(ctx, m.c, b, 0.0, nullptr, Y, fs, st));
    for (int j = 0; j < ns; j++) RM_TRY(axpby64(ctx, 1.0, Y, m.alpha[j], xs + (size_t)j * fs, Y, fs, st));
    if (iters) *iters = it;
    return RMHMC_OK;
}

// 1/R(lam) = p0 + p1 lam + sum_j beta_j / (lam + zeta_j) for R = c + sum_j alpha_j / (lam + sigma_j) with c >= 0,
// alpha_j >= 0 (terms with alpha_j = 0 dropped).  R has one zero between consecutive poles and, when c > 0, one
// below the smallest -sigma; each is bracketed and bisected in long double; beta_j = 1 / R'(-zeta_j).  At
// infinity 1/R -> 1/c (c > 0), else lam / sum(alpha) + sum(alpha sigma) / sum(alpha)^2.
int inverse_rational(rmhmc_ctx* ctx, const MassTerm& m, MassTerm& inv, double& p1) {
    typedef long double ld;
    std::vector<std::pair<double, double>> t;   // (sigma, alpha)
    for (int j = 0; j < m.npole(); j++) {
        if (m.alpha[j] < 0.0) return set_err(ctx, RMHMC_EINVAL, "general rational mass: alpha_j must be >= 0");
        if (m.alpha[j] > 0.0) t.push_back({m.sigma[j], m.alpha[j]});
    }
    if (m.c < 0.0 || (m.c == 0.0 && t.empty())) return set_err(ctx, RMHMC_EINVAL, "general rational mass: R is not positive");
    std::sort(t.begin(), t.end());
    const int n = (int)t.size();
    auto R = [&](ld x) {
        ld r = (ld)m.c;
        for (const auto& q : t) r += (ld)q.second / (x + (ld)q.first);
        return r;
    };
    auto bisect = [&](ld lo, ld hi) {   // R(lo) > 0 > R(hi)
        for (int i = 0; i < 300 && hi - lo > 0; i++) {
            const ld mid = 0.5L * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (R(mid) > 0) lo = mid; else hi = mid;
        }
        return 0.5L * (lo + hi);
    };
    std::vector<ld> zeros;
    for (int j = 0; j + 1 < n; j++) zeros.push_back(bisect(-(ld)t[j + 1].first, -(ld)t[j].first));
    if (m.c > 0.0 && n > 0) {
        const ld hi = -(ld)t[n - 1].first;
        ld d = 1.0L;
        int guard = 0;
        while (R(hi - d) <= 0 && guard++ < 400) d *= 2.0L;
        zeros.push_back(bisect(hi - d, hi));
    }
    inv.kappa = 0.0;
    inv.alpha.clear();
    inv.sigma.clear();
    for (ld z : zeros) {
        ld dr = 0.0L;
        for (const auto& q : t) dr -= (ld)q.second / ((z + (ld)q.first) * (z + (ld)q.first));
        inv.alpha.push_back((double)(1.0L / dr));
        inv.sigma.push_back((double)(-z));
    }
    if (m.c > 0.0) {
        inv.c = 1.0 / m.c;
        p1 = 0.0;
    } else {
        ld sa = 0.0L, sas = 0.0L;
        for (const auto& q : t) { sa += (ld)q.second; sas += (ld)q.second * (ld)q.first; }
        inv.c = (double)(sas / (sa * sa));
        p1 = (double)(1.0L / sa);
    }
    return RMHMC_OK;
}

int heatbath_apply(rmhmc_ctx* ctx, const MassTerm& m, const double* xi, double tol, int maxiter, int prec, double* P,
                   cudaStream_t st) {
    int status = RMHMC_OK;
    const size_t fs = field_elems(ctx);
    double* y = (double*)workspace(ctx, "hb_y", sizeof(double) * fs, &status);
    if (!y) return status;
    if (m.kappa == 0.0 && m.npole() > 0) {
        // general rational mass M = R^{-2}: P = R(A)^{-1} xi exactly, from the partial fraction of 1/R
        MassTerm inv;
        double p1 = 0.0;
        RM_TRY(inverse_rational(ctx, m, inv, p1));
        RM_TRY(rational_apply(ctx, inv, xi, tol, maxiter, prec, y, nullptr, st));
        if (p1 == 0.0) {
            RM_CHECK(ctx, cudaMemcpyAsync(P, y, sizeof(double) * fs, cudaMemcpyDeviceToDevice, st));
            return RMHMC_OK;
        }
        // P = y + p1 A xi = y + p1 (xi / 2 - H(xi) / 16) (through scratch when P is xi itself)
        double* out = P;
        if (P == xi) {
            out = (double*)workspace(ctx, "hb_t", sizeof(double) * fs, &status);
            if (!out) return status;
        }
        RM_TRY(launch_lap(ctx, RMHMC_FP64, 18, xi, out, 1, 0.5 * p1, -p1 / 16.0, y, 1.0, -1, st));
        if (out != P) RM_CHECK(ctx, cudaMemcpyAsync(P, out, sizeof(double) * fs, cudaMemcpyDeviceToDevice, st));
        return RMHMC_OK;
    }
    RM_TRY(rational_apply(ctx, m, xi, tol, maxiter, prec, y, nullptr, st));
    // P = (1-kappa) y + kappa A y = ((1-kappa) + kappa/2) y - (kappa/16) H(y)
    const double k = m.kappa;
    return launch_lap(ctx, RMHMC_FP64, 18, y, P, 1, (1.0 - k) + 0.5 * k, -k / 16.0, nullptr, 0.0, -1, st);
}

// ------------------------------------------------------------------------------------------------
// graph-capturable kinetic evaluation: every decision on the device
// ------------------------------------------------------------------------------------------------
// r_0 = b, rho_0; arms the conditional of the CG loop (1 unless b = 0)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cgg_start(const T* __restrict__ b, T* __restrict__ r0, size_t nvec,
                                                      int* flags, double* rho, double* partials, unsigned* counter,
                                                      cudaGraphConditionalHandle h) {
    __shared__ double sh[kBlock / 32];
    using VT = Vec<T>;
    if (blockIdx.x == 0 && threadIdx.x == 0) flags[2] = 0;   // pass counter of the guard in k_cgg_B
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += (size_t)gridDim.x * blockDim.x) {
        const typename VT::type v = reinterpret_cast<const typename VT::type*>(b)[i];
        reinterpret_cast<typename VT::type*>(r0)[i] = v;
        T x[VT::n];
        VT::get(v, x);
#pragma unroll
        for (int k = 0; k < VT::n; k++) acc += (double)x[k] * (double)x[k];
    }
    double v[1] = {acc};
    block_sum<1>(v, sh);
    double out[1];
    if (grid_sum_finish<1>(v, partials, counter, out, gridDim.x, blockIdx.x, sh)) {
        rho[0] = out[0];
        flags[1] = 0;
        flags[0] = isfinite(out[0]) ? (out[0] == 0.0 ? 1 : 0) : 3;
        cudaGraphSetConditional(h, flags[0] == 0 ? 1u : 0u);
    }
}

// second half of a CG iteration (as k_cg_B) that ends the graph's loop when the run stops; counts iterations
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cgg_B(T* __restrict__ R, size_t fs, const T* __restrict__ q, size_t nvec,
                                                  int* flags, double* vals, int maxit, double tol2, double* partials,
                                                  unsigned* counter, cudaGraphConditionalHandle h, long long* iters) {
    __shared__ double sh[kBlock / 32];
    // guard independent of the reduction: whatever happens to the tickets, the loop ends after maxit + 4
    // passes (the cap is recorded as a failed run)
    if (blockIdx.x == 0 && threadIdx.x == 0 && atomicAdd(&flags[2], 1) > maxit + 4) {
        flags[0] = 2;
        cudaGraphSetConditional(h, 0u);
    }
    if (flags[0]) {
        if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
        return;
    }
    const int k = flags[1];
    double* rho = vals;
    const double* gamma = vals + (maxit + 1);
    const double* alpha = gamma + maxit;
    double* beta = (double*)(alpha + maxit);
    using VT = Vec<T>;
    const T a = (T)alpha[k];
    T dot = T(0);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += (size_t)gridDim.x * blockDim.x) {
        T x[VT::n], y[VT::n];
        VT::get(reinterpret_cast<const typename VT::type*>(R + (size_t)k * fs)[i], x);
        VT::get(reinterpret_cast<const typename VT::type*>(q)[i], y);
#pragma unroll
        for (int c = 0; c < VT::n; c++) {
            x[c] = fma(-a, y[c], x[c]);
            dot = fma(x[c], x[c], dot);
        }
        reinterpret_cast<typename VT::type*>(R + (size_t)(k + 1) * fs)[i] = VT::make(x);
    }
    double v[1] = {0.0};
    if (sizeof(T) == 4) {
        float fv[1] = {(float)dot};
        block_sum_f<1>(fv, sh);
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
            v[0] = t;
        }
    } else {
        v[0] = (double)dot;
        block_sum<1>(v, sh);
    }
    double out[1];
    if (grid_sum_finish<1>(v, partials, counter, out, gridDim.x, blockIdx.x, sh)) {
        const double rr = out[0];
        rho[k + 1] = rr;
        beta[k] = rr / rho[k];
        flags[1] = k + 1;
        (*iters)++;
        if (!isfinite(rr) || !isfinite(alpha[k])) flags[0] = 3;
        else if (rr <= tol2 * rho[0]) flags[0] = 1;
        else if (k + 1 >= maxit) flags[0] = 2;
        if (flags[0] != 0) cudaGraphSetConditional(h, 0u);
    }
}

// Lanczos post-processing on the device (one block): from alpha, beta, rho of the run, the Galerkin coefficient
// vectors y_j = (T + D_j)^{-1} e1 |b|, g = R(T) e1 |b|, z_j = (T + D_j)^{-1} g, v = R(T) g, written as rows on the
// stored residuals: rows j < ns: X_j, rows ns + j: Z_j, row 2 ns: V.  Row stride: kBasisCap.  A run that did not
// converge (cap or NaN) is recorded in *status.
struct DevMass {
    int ns;
    double c;
    double alpha[24];
    double delta[24];
};

__global__ void __launch_bounds__(128) k_lanczos_rows(const int* __restrict__ flags, const double* __restrict__ vals, int maxit,
                                                      DevMass m, double* __restrict__ rows, double* __restrict__ work,
                                                      int* status) {
    constexpr int N = 160;   // kBasisCap
    __shared__ double d[N], e[N], inv[N], g[N], v[N];
    const int n = flags[1];
    const double* rho = vals;
    const double* alpha = vals + (maxit + 1) + maxit;
    const double* beta = alpha + maxit;
    if (threadIdx.x == 0 && flags[0] >= 2) atomicMax(status, flags[0] == 2 ? 1 : 2);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        d[k] = 1.0 / alpha[k] + (k > 0 ? beta[k - 1] / alpha[k - 1] : 0.0);
        e[k] = k < n - 1 ? -sqrt(beta[k]) / alpha[k] : 0.0;
        inv[k] = 1.0 / sqrt(rho[k]);
    }
    __syncthreads();
    const double bn = n > 0 ? sqrt(rho[0]) : 0.0;
    // work: [ns][N] y_j, then [ns][N] z_j, then [ns][N] Thomas scratch
    double* Y = work;
    double* Z = work + (size_t)m.ns * N;
    double* C = work + (size_t)2 * m.ns * N;
    auto thomas = [&](double shift, const double* rhs, double* y, double* c) {
        if (n == 0) return;
        double den = d[0] + shift;
        c[0] = n > 1 ? e[0] / den : 0.0;
        y[0] = rhs[0] / den;
        for (int k = 1; k < n; k++) {
            den = d[k] + shift - e[k - 1] * c[k - 1];
            c[k] = k < n - 1 ? e[k] / den : 0.0;
            y[k] = (rhs[k] - e[k - 1] * y[k - 1]) / den;
        }
        for (int k = n - 2; k >= 0; k--) y[k] -= c[k] * y[k + 1];
    };
    for (int k = threadIdx.x; k < n; k += blockDim.x) v[k] = k == 0 ? bn : 0.0;   // e1 |b| (scratch)
    __syncthreads();
    if (threadIdx.x < m.ns) thomas(m.delta[threadIdx.x], v, Y + (size_t)threadIdx.x * N, C + (size_t)threadIdx.x * N);
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double t = m.c * (k == 0 ? bn : 0.0);
        for (int j = 0; j < m.ns; j++) t += m.alpha[j] * Y[(size_t)j * N + k];
        g[k] = t;
    }
    __syncthreads();
    if (threadIdx.x < m.ns) thomas(m.delta[threadIdx.x], g, Z + (size_t)threadIdx.x * N, C + (size_t)threadIdx.x * N);
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double t = m.c * g[k];
        for (int j = 0; j < m.ns; j++) t += m.alpha[j] * Z[(size_t)j * N + k];
        rows[(size_t)(2 * m.ns) * N + k] = t * inv[k];
        for (int j = 0; j < m.ns; j++) {
            rows[(size_t)j * N + k] = Y[(size_t)j * N + k] * inv[k];
            rows[(size_t)(m.ns + j) * N + k] = Z[(size_t)j * N + k] * inv[k];
        }
    }
}

// handle of a conditional node in the graph that stream st is capturing into
int capture_handle(rmhmc_ctx* ctx, cudaStream_t st, unsigned init, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    RM_CHECK(ctx, cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) return set_err(ctx, RMHMC_ECUDA, "conditional handle outside a capture");
    RM_CHECK(ctx, cudaGraphConditionalHandleCreate(h, g, init, cudaGraphCondAssignDefault));
    return RMHMC_OK;
}

// WHILE node with handle h at the current capture point of st; *body receives its (empty) body graph and
// the capture continues after the node
int capture_while(rmhmc_ctx* ctx, cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    RM_CHECK(ctx, cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd));
    if (cs != cudaStreamCaptureStatusActive) return set_err(ctx, RMHMC_ECUDA, "WHILE node outside a capture");
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    RM_CHECK(ctx, cudaGraphAddNode(&node, g, deps, ed, nd, &p));
    *body = p.conditional.phGraph_out[0];
    RM_CHECK(ctx, cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return RMHMC_OK;
}

// buffers of the captured kinetic evaluation (allocated before any capture)
struct KinGraphBufs {
    float* P32 = nullptr;
    float* R = nullptr;
    float* q = nullptr;
    int* flags = nullptr;
    double* vals = nullptr;
    double* rows = nullptr;
    double* work = nullptr;
    double* pairs = nullptr;
    int maxit = 0;
};

static int kin_graph_bufs(rmhmc_ctx* ctx, int ns, int maxit, KinGraphBufs& b) {
    int status = RMHMC_OK;
    const size_t fs = field_elems(ctx);
    b.maxit = std::min(maxit, kBasisCap);
    b.P32 = (float*)workspace(ctx, "kg_p32", sizeof(float) * fs, &status);
    b.R = (float*)workspace(ctx, "kr_basis32", sizeof(float) * fs * (size_t)(kBasisCap + 1), &status);
    b.q = (float*)workspace(ctx, "kg_q32", sizeof(float) * fs, &status);
    void* sc = workspace(ctx, "kg_scal", 64 + sizeof(double) * 4 * (size_t)(kBasisCap + 2), &status);
    b.rows = (double*)workspace(ctx, "kg_rows", sizeof(double) * kBasisCap * (size_t)(2 * ns + 1), &status);
    b.work = (double*)workspace(ctx, "kg_work", sizeof(double) * kBasisCap * (size_t)(3 * ns + 1), &status);
    b.pairs = (double*)workspace(ctx, "kf_pairs", sizeof(double) * kBasisCap * kBasisCap, &status);
    if (!b.P32 || !b.R || !b.q || !sc || !b.rows || !b.work || !b.pairs) return status;
    b.flags = (int*)sc;
    b.vals = (double*)((char*)sc + 64);
    return RMHMC_OK;
}

int kinetic_graph_prepare(rmhmc_ctx* ctx, const MassTerm& m, int maxiter) {
    KinGraphBufs b;
    RM_TRY(kin_graph_bufs(ctx, m.npole(), maxiter, b));
    StencilShape shp;
    return cg_shape<float>(ctx, 0, shp);
}

// Enqueue (on a capturing stream) one mixed-precision kinetic evaluation at the context's links:
// F_K (float64) and the velocity M^{-1} P (float64), every decision taken on the device.  stats[0] counts
// Krylov iterations; *status records a Krylov run that hit its cap (1) or produced NaN (2).  aux is a second
// stream used to capture the body of the CG loop.
int kinetic_enqueue(rmhmc_ctx* ctx, const MassTerm& m, const double* P, double tol, int maxiter, double* F, double* Vel,
                    long long* stats, int* status, cudaStream_t st, cudaStream_t aux) {
    const int ns = m.npole();
    if (ns == 0 || 2 * ns + 1 > kMaxCombine) return set_err(ctx, RMHMC_EINVAL, "captured kinetic force needs 1..15 poles");
    KinGraphBufs b;
    RM_TRY(kin_graph_bufs(ctx, ns, maxiter, b));
    const size_t fs = field_elems(ctx);
    const size_t nvec = fs / 4;
    const int nb = capped_grid(ctx, nvec, kBlock);
    StencilShape shp;
    RM_TRY(cg_shape<float>(ctx, st, shp));
    const double s0 = *std::min_element(m.sigma.begin(), m.sigma.end());
    DevMass dm{};
    dm.ns = ns;
    dm.c = m.c;
    for (int j = 0; j < ns; j++) {
        dm.alpha[j] = m.alpha[j];
        dm.delta[j] = m.sigma[j] - s0;
    }
    RM_TRY(to_float(ctx, P, b.P32, fs, st));
    cudaGraphConditionalHandle h;
    RM_TRY(capture_handle(ctx, st, 0u, &h));
    k_cgg_start<float><<<nb, kBlock, 0, st>>>(b.P32, b.R, nvec, b.flags, b.vals, red_slot_partials(ctx, kSlotRho),
                                              red_slot_counter(ctx, kSlotRho), h); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    cudaGraph_t body;
    RM_TRY(capture_while(ctx, st, h, &body));
    {
        RM_CHECK(ctx, cudaStreamBeginCaptureToGraph(aux, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        const Links32 U = links32(ctx);
        const float diag = (float)(0.5 + s0);
        const int cs = cg_stencil<float>(ctx, shp, U, b.R, fs, b.q, diag, b.flags, b.vals, b.maxit, aux);
        if (cs != RMHMC_OK) {
            cudaGraph_t tmp;
            cudaStreamEndCapture(aux, &tmp);
            return cs;
        }
        k_cgg_B<float><<<nb, kBlock, 0, aux>>>(b.R, fs, b.q, nvec, b.flags, b.vals, b.maxit, tol * tol,
                                               red_slot_partials(ctx, kSlotRho), red_slot_counter(ctx, kSlotRho), h,
                                               stats); ++ctx->launches;
        RM_LAUNCH_CHECK(ctx);
        cudaGraph_t tmp;
        RM_CHECK(ctx, cudaStreamEndCapture(aux, &tmp));
    }
    k_lanczos_rows<<<1, 128, 0, st>>>(b.flags, b.vals, b.maxit, dm, b.rows, b.work, status); ++ctx->launches;
    const int grid = capped_grid(ctx, fs / 4, kBlock);
    OutPtrs<float, double> ov{};
    ov.p[0] = Vel;
    k_combine<float, double, 1><<<grid, kBlock, 0, st>>>(b.R, fs, b.flags, 0, b.rows + (size_t)2 * ns * kBasisCap,
                                                         kBasisCap, 1, ov);
    ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return link_grad_krylov_launch(ctx, b.R, b.rows, kBasisCap, ns, m.alpha.data(), b.flags, 0, F, st);
}

}  // namespace rm

using namespace rm;

extern "C" int rat_mass_solve(rmhmc_ctx* ctx, const double* U, const double* b, int nfield, int nshift,
                              const double* sigma, const double* alpha, double c, double tol, int maxiter, int prec,
                              double* y, double* xs, int* iters, double* resid, cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (nfield < 0 || nfield > 65535) return set_err(ctx, RMHMC_EINVAL, "rat_mass_solve: nfield in [0, 65535]");
    if (nfield > 0 && (!b || !y)) return set_err(ctx, RMHMC_EINVAL, "rat_mass_solve: null field");
    if (nshift < 0 || nshift > 24 || (nshift > 0 && (!sigma || !alpha)))
        return set_err(ctx, RMHMC_EINVAL, "rat_mass_solve: bad shifts");
    if (!(tol > 0.0) || maxiter < 1) return set_err(ctx, RMHMC_EINVAL, "rat_mass_solve: bad tolerance or maxiter");
    if (prec != RMHMC_FP64 && prec != RMHMC_MIXED) return set_err(ctx, RMHMC_EINVAL, "rat_mass_solve: bad prec");
    if ((uintptr_t)b % 16 || (uintptr_t)y % 16 || (uintptr_t)xs % 16)
        return set_err(ctx, RMHMC_EINVAL, "rat_mass_solve: fields must be 16-byte aligned");
    rmhmc_mass mm{c, nshift, alpha, sigma, 0.0};
    MassTerm m;
    RM_TRY(parse_mass(ctx, &mm, m));
    RM_TRY(ensure_links(ctx, U, stream));
    if (iters) *iters = 0;
    const size_t fs = field_elems(ctx);
    int status = RMHMC_OK;
    double* xw = nullptr;   // shared workspace of the shifted solutions when the caller wants none
    if (!xs && nshift > 0) {
        xw = (double*)workspace(ctx, "rs_xs", sizeof(double) * fs * nshift, &status);
        if (!xw) return status;
    }
    for (int f = 0; f < nfield; f++) {
        const double* bf = b + (size_t)f * fs;
        double* yf = y + (size_t)f * fs;
        double* x = xs ? xs + (size_t)f * nshift * fs : xw;
        int it = 0;
        RM_TRY(solve_shifts(ctx, m, bf, tol, maxiter, prec, x, &it, resid ? resid + (size_t)f * nshift : nullptr, stream));
        // y_f = c b_f + sum_j alpha_j x_fj (float64)
        RM_TRY(axpby64(ctx, c, bf, 0.0, nullptr, yf, fs, stream));
        for (int j = 0; j < nshift; j++) RM_TRY(axpby64(ctx, 1.0, yf, alpha[j], x + (size_t)j * fs, yf, fs, stream));
        if (iters) *iters += it;
    }
    return RMHMC_OK;
}
