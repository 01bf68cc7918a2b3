// Sec. 2, Eq. (3) for many fields at once: Y_f = a X_f + b H(X_f) + c W_f (f < nfield) with the hops in the
// adjoint form
//   H(X)^a(x) = sum_nu [ Ad(U_nu(x))_ab X^b(x+nu) + Ad(U_nu(x-nu))_ba X^b(x-nu) ],
// Ad(U)_ab = 2 Tr(T^a U T^b U^dag), so that every link is read and turned into its 8x8 adjoint matrix once
// per application and then applied to all 4 nfield operands of its hop (64 FMA each instead of 144 for
// U X U^dag).  Float32 only; this is the stencil of the batched Chebyshev recurrence (all spectral fields
// share one launch per step) and of multi-field lap_apply.
//
// Work of one block: a tile of kAdSites consecutive sites (lexicographic order).
//   phase 1: thread (hop, site) loads one link -- U_h(x) for the forward hops h < 4, U_{h-4}(x - h) for the
//            backward ones -- and stores Ad (forward) or Ad^T (backward) in shared memory, with the
//            neighbour site of that hop;
//   phase 2: thread (site, mu, half) accumulates rows 4 half .. 4 half + 3 of H(X_f)_mu for CH fields
//            at a time over the 8 hops, reading the adjoint rows from shared memory (bank-conflict-free
//            padding) and the neighbour values from global memory, then writes its quarter-row of Y_f and
//            adds the per-field dots <Y,Y>, <Y,X> to per-warp float64 sums (deterministic order).
#include "common.cuh"
#include "ops.cuh"

namespace rm {

constexpr int kAdSites = 32;                 // sites per tile
constexpr int kAdThreads = 256;              // 8 hops x 32 sites in phase 1; 32 sites x 4 mu x 2 halves in phase 2
constexpr int kAdHalf = 36;                  // floats per half record (4 rows x 8, padded by 4)
constexpr int kAdHop = 2 * kAdHalf;          // floats per (site, hop) record
constexpr int kAdSiteStride = 8 * kAdHop + 8;   // 584 floats: = 8 mod 32, so the 8 (site, half) records a warp
                                                // reads in one 128-bit load fall on 8 distinct bank quads
constexpr size_t kAdSmemFloats = (size_t)kAdSites * kAdSiteStride;
constexpr int kMaxDevices = 64;

// dynamic shared memory of one block: adjoint records, neighbour sites, per-warp float64 dots of nd fields
inline size_t ad_smem_bytes(int nd) {
    return kAdSmemFloats * sizeof(float) + kAdSites * 8 * sizeof(int) + (size_t)(kAdThreads / 32) * nd * 2 * sizeof(double);
}

// CH: fields per pass of phase 2; MINB: resident blocks the register budget is compiled for
template <int LF, bool HAS_W, bool DOTS, int CH, int MINB>
__global__ void __launch_bounds__(kAdThreads, MINB) k_lap_ad(Geom g, Links32 U, const float* __restrict__ X,
                                                        float* __restrict__ Y, const float* __restrict__ W, int nf,
                                                        float a, float b, float c, size_t fs, double* partials,
                                                        unsigned* counters, double* out, size_t slot_stride) {
    extern __shared__ __align__(16) float smem[];
    float* ad = smem;                                            // [kAdSites][kAdSiteStride]
    int* nbr = reinterpret_cast<int*>(smem + kAdSmemFloats);     // [kAdSites][8]
    double* dsum = reinterpret_cast<double*>(nbr + kAdSites * 8);   // [warps][nf][2] (DOTS)
    __shared__ double sh[2 * (kAdThreads / 32)];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (DOTS)
        for (int i = t; i < (kAdThreads / 32) * nf * 2; i += kAdThreads) dsum[i] = 0.0;
    const int ntile = (g.V + kAdSites - 1) / kAdSites;
    // phase-2 role of this thread
    const int ps = t >> 3, pmu = (t >> 1) & 3, phalf = t & 1;
    for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        // ---- phase 1: adjoint matrices of the 8 hops of every site in the tile
        {
            const int sl = t & (kAdSites - 1), hop = t >> 5;
            const int s = tile * kAdSites + sl;
            if (s < g.V) {
                const int dir = hop & 3;
                const int nb = hop < 4 ? step_site(g, s, dir, 1) : step_site(g, s, dir, -1);
                const mat3<float> u = LinkLoad<float, LF>::load(U, hop < 4 ? s : nb, dir);
                float* rec = ad + sl * kAdSiteStride + hop * kAdHop;
                if (hop < 4) {
                    // Ad row by row: column b lands in entry b of each row
                    adjoint_columns(u, [&](int bcol, const float (&col)[8]) {
#pragma unroll
                        for (int r = 0; r < 8; r++) rec[(r >> 2) * kAdHalf + (r & 3) * 8 + bcol] = col[r];
                    });
                } else {
                    // Ad^T: column b of Ad is row b of the record
                    adjoint_columns(u, [&](int bcol, const float (&col)[8]) {
                        float4* d = reinterpret_cast<float4*>(rec + (bcol >> 2) * kAdHalf + (bcol & 3) * 8);
                        d[0] = make_float4(col[0], col[1], col[2], col[3]);
                        d[1] = make_float4(col[4], col[5], col[6], col[7]);
                    });
                }
                nbr[sl * 8 + hop] = nb;
            }
        }
        __syncthreads();
        // ---- phase 2
        const int s = tile * kAdSites + ps;
        const bool active = s < g.V;
        const float* rec0 = ad + ps * kAdSiteStride + phalf * kAdHalf;
        const int* nb = nbr + ps * 8;
        const float* Xm = X + pmu * 8;
        // the (pass, hop) iterations are software-pipelined: the neighbour values of the next iteration are
        // loaded before the arithmetic of the current one
        auto load_x = [&](int f0, int hop, float (&x)[CH][8]) {
            const size_t n = (size_t)nb[hop] * 32;
#pragma unroll
            for (int q = 0; q < CH; q++) {
                if (active && f0 + q < nf) load8(Xm + (size_t)(f0 + q) * fs + n, x[q]);
                else
#pragma unroll
                    for (int k = 0; k < 8; k++) x[q][k] = 0.f;
            }
        };
        float xb[2][CH][8];
        load_x(0, 0, xb[0]);
        for (int f0 = 0; f0 < nf; f0 += CH) {
            float acc[CH][4];
#pragma unroll
            for (int q = 0; q < CH; q++)
#pragma unroll
                for (int r = 0; r < 4; r++) acc[q][r] = 0.f;
#pragma unroll
            for (int hop = 0; hop < 8; hop++) {
                // prefetch: the next hop of this pass, or hop 0 of the next pass
                if (hop < 7) load_x(f0, hop + 1, xb[(hop + 1) & 1]);
                else if (f0 + CH < nf) load_x(f0 + CH, 0, xb[0]);
                const float (&x)[CH][8] = xb[hop & 1];
                const float* rec = rec0 + hop * kAdHop;
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const float4 r0 = *reinterpret_cast<const float4*>(rec + r * 8);
                    const float4 r1 = *reinterpret_cast<const float4*>(rec + r * 8 + 4);
#pragma unroll
                    for (int q = 0; q < CH; q++) {
                        float v = acc[q][r];
                        v = fmaf(r0.x, x[q][0], v); v = fmaf(r0.y, x[q][1], v);
                        v = fmaf(r0.z, x[q][2], v); v = fmaf(r0.w, x[q][3], v);
                        v = fmaf(r1.x, x[q][4], v); v = fmaf(r1.y, x[q][5], v);
                        v = fmaf(r1.z, x[q][6], v); v = fmaf(r1.w, x[q][7], v);
                        acc[q][r] = v;
                    }
                }
            }
            // epilogue: the thread's 4 components of Y_f(s)_mu, and the dots
#pragma unroll
            for (int q = 0; q < CH; q++) {
                const int f = f0 + q;
                float yy = 0.f, yx = 0.f;
                if (active && f < nf) {
                    const size_t off = (size_t)f * fs + (size_t)s * 32 + pmu * 8 + phalf * 4;
                    const float4 xo = __ldg(reinterpret_cast<const float4*>(X + off));
                    float y[4] = {fmaf(b, acc[q][0], a * xo.x), fmaf(b, acc[q][1], a * xo.y),
                                  fmaf(b, acc[q][2], a * xo.z), fmaf(b, acc[q][3], a * xo.w)};
                    if (HAS_W) {
                        const float4 w = __ldg(reinterpret_cast<const float4*>(W + off));
                        y[0] = fmaf(c, w.x, y[0]); y[1] = fmaf(c, w.y, y[1]);
                        y[2] = fmaf(c, w.z, y[2]); y[3] = fmaf(c, w.w, y[3]);
                    }
                    *reinterpret_cast<float4*>(Y + off) = make_float4(y[0], y[1], y[2], y[3]);
                    if (DOTS) {
                        yy = fmaf(y[0], y[0], fmaf(y[1], y[1], fmaf(y[2], y[2], y[3] * y[3])));
                        yx = fmaf(y[0], xo.x, fmaf(y[1], xo.y, fmaf(y[2], xo.z, y[3] * xo.w)));
                    }
                }
                if (DOTS && f < nf) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        yy += __shfl_xor_sync(0xffffffffu, yy, o);
                        yx += __shfl_xor_sync(0xffffffffu, yx, o);
                    }
                    if (lane == 0) {
                        dsum[(warp * nf + f) * 2] += (double)yy;
                        dsum[(warp * nf + f) * 2 + 1] += (double)yx;
                    }
                }
            }
        }
        __syncthreads();   // the next tile overwrites the adjoint records
    }
    if (DOTS) {
        // per field: the warps' sums in warp order, then the deterministic grid sum
        for (int f = 0; f < nf; f++) {
            double v[2] = {0.0, 0.0};
            if (t == 0)
                for (int w = 0; w < kAdThreads / 32; w++) {
                    v[0] += dsum[(w * nf + f) * 2];
                    v[1] += dsum[(w * nf + f) * 2 + 1];
                }
            grid_sum_finish<2>(v, partials + f * slot_stride, counters + f, out + (size_t)f * 8, gridDim.x, blockIdx.x,
                               sh);
        }
    }
}

// launch shapes (fields per pass, blocks per SM), chosen per context by timing on first use
struct AdShape { int ch, minb; };
constexpr AdShape kAdShapes[3] = {{2, 3}, {3, 2}, {4, 2}};

template <int LF, bool HAS_W, bool DOTS, int CH, int MINB>
static int launch_ad_t(rmhmc_ctx* ctx, const float* X, float* Y, int nf, double a, double b, const float* W, double c,
                       int slot, cudaStream_t st) {
    if (DOTS && nf > kRedSlots) return set_err(ctx, RMHMC_EINVAL, "too many reduced fields");
    auto kern = k_lap_ad<LF, HAS_W, DOTS, CH, MINB>;
    const size_t smem = ad_smem_bytes(DOTS ? nf : 0);
    // the dynamic shared-memory limit of this instantiation, raised once per device to the largest size any
    // launch can ask for (kRedSlots reduced fields)
    static bool configured[kMaxDevices] = {};
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return set_err(ctx, RMHMC_EINVAL, "device index too large");
    if (!configured[ctx->device]) {
        RM_CHECK(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ad_smem_bytes(kRedSlots)));
        configured[ctx->device] = true;
    }
    int per_sm = 0;
    RM_CHECK(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAdThreads, smem));
    const int ntile = (ctx->g.V + kAdSites - 1) / kAdSites;
    const int grid = std::max(1, std::min(ntile, (int)ctx->num_sms * std::max(per_sm, 1)));
    const size_t ss = (size_t)ctx->max_blocks * 2;
    double* part = DOTS ? red_slot_partials(ctx, slot) : nullptr;
    unsigned* cnt = DOTS ? red_slot_counter(ctx, slot) : nullptr;
    double* out = DOTS ? red_slot_out(ctx, slot) : nullptr;
    kern<<<grid, kAdThreads, smem, st>>>(ctx->g, links32(ctx), X, Y, W, nf, (float)a, (float)b, (float)c, field_elems(ctx),
                                         part, cnt, out, ss);
    ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}

template <int LF, int CH, int MINB>
static int launch_ad_shape(rmhmc_ctx* ctx, const float* X, float* Y, int nf, double a, double b, const float* W,
                           double c, int slot, cudaStream_t st) {
    if (W) {
        if (slot >= 0) return launch_ad_t<LF, true, true, CH, MINB>(ctx, X, Y, nf, a, b, W, c, slot, st);
        return launch_ad_t<LF, true, false, CH, MINB>(ctx, X, Y, nf, a, b, W, c, slot, st);
    }
    if (slot >= 0) return launch_ad_t<LF, false, true, CH, MINB>(ctx, X, Y, nf, a, b, W, c, slot, st);
    return launch_ad_t<LF, false, false, CH, MINB>(ctx, X, Y, nf, a, b, W, c, slot, st);
}

template <int LF>
static int launch_ad_idx(rmhmc_ctx* ctx, int k, const float* X, float* Y, int nf, double a, double b, const float* W,
                         double c, int slot, cudaStream_t st) {
    if (k == 0) return launch_ad_shape<LF, 2, 3>(ctx, X, Y, nf, a, b, W, c, slot, st);
    if (k == 1) return launch_ad_shape<LF, 3, 2>(ctx, X, Y, nf, a, b, W, c, slot, st);
    return launch_ad_shape<LF, 4, 2>(ctx, X, Y, nf, a, b, W, c, slot, st);
}

// the shape for this link format: on first use every shape is timed (one warm-up and three timed plain
// applications of the caller's fields, written to the caller's output) and the fastest is kept
template <int LF>
static int ad_shape(rmhmc_ctx* ctx, const float* X, float* Y, int nf, cudaStream_t st, int* out) {
    const int key = 20000 + LF;
    auto it = ctx->tune.find(key);
    if (it != ctx->tune.end()) {
        *out = it->second.first;
        return RMHMC_OK;
    }
    cudaEvent_t e0, e1;
    RM_CHECK(ctx, cudaEventCreate(&e0));
    RM_CHECK(ctx, cudaEventCreate(&e1));
    float best = 1e30f;
    int bk = 0;
    char line[96];
    std::string rep;
    for (int k = 0; k < 3; k++) {
        RM_TRY(launch_ad_idx<LF>(ctx, k, X, Y, nf, 0.5, -0.0625, nullptr, 0.0, -1, st));
        RM_CHECK(ctx, cudaEventRecord(e0, st));
        for (int r = 0; r < 3; r++) RM_TRY(launch_ad_idx<LF>(ctx, k, X, Y, nf, 0.5, -0.0625, nullptr, 0.0, -1, st));
        RM_CHECK(ctx, cudaEventRecord(e1, st));
        RM_CHECK(ctx, cudaEventSynchronize(e1));
        float ms = 0.f;
        RM_CHECK(ctx, cudaEventElapsedTime(&ms, e0, e1));
        ms /= 3.f;
        snprintf(line, sizeof line, "%s%d/%d:%.4f", rep.empty() ? "" : " ", kAdShapes[k].ch, kAdShapes[k].minb, ms);
        rep += line;
        if (ms < best) { best = ms; bk = k; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tune[key] = {bk, nf};
    snprintf(line, sizeof line, "; adjoint LF%d (%d fields) -> %d fields/pass, %d blocks/SM [", LF, nf, kAdShapes[bk].ch,
             kAdShapes[bk].minb);
    ctx->tune_report += line + rep + "]";
    *out = bk;
    return RMHMC_OK;
}

template <int LF>
static int launch_ad_lf(rmhmc_ctx* ctx, const float* X, float* Y, int nf, double a, double b, const float* W, double c,
                        int slot, cudaStream_t st) {
    // the tuner writes Y, so a call that updates W in place (Y == W) takes the tuned shape if there is one and
    // the middle shape otherwise
    int k = 1;
    if (W != Y) RM_TRY(ad_shape<LF>(ctx, X, Y, nf, st, &k));
    else if (ctx->tune.count(20000 + LF)) k = ctx->tune[20000 + LF].first;
    return launch_ad_idx<LF>(ctx, k, X, Y, nf, a, b, W, c, slot, st);
}

int launch_lap_ad(rmhmc_ctx* ctx, int linkfmt, const float* X, float* Y, int nfield, double a, double b, const float* W,
                  double c, int slot, cudaStream_t st) {
    if (linkfmt == 12) return launch_ad_lf<12>(ctx, X, Y, nfield, a, b, W, c, slot, st);
    return launch_ad_lf<18>(ctx, X, Y, nfield, a, b, W, c, slot, st);
}

}  // namespace rm
