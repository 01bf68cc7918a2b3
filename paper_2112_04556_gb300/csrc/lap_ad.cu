// Sec. 2, Eq. (3) for many fields at once: Y_f = a X_f + b H(X_f) + c W_f (f < nfield) with the hops in the
// adjoint form
//   H(X)^a(x) = sum_nu [ Ad(U_nu(x))_ab X^b(x+nu) + Ad(U_nu(x-nu))_ba X^b(x-nu) ],
// Ad(U)_ab = 2 Tr(T^a U T^b U^dag), so that every link is read and turned into its 8x8 adjoint matrix once
// per application and then applied to all 4 nfield operands of its hop (64 FMA each instead of 144 for
// U X U^dag).  Float32 only; this is the stencil of the batched Chebyshev recurrence (all spectral fields
// share one launch per step) and of multi-field lap_apply.
//
// Work of one block: a tile of kAdSites consecutive sites; tiles are taken in the order (z block, t, position
// in the slab), slabs of bz whole xy-planes.  bz = L2 (the default) is the lexicographic order; a thinner slab
// keeps the t-neighbours of a slab in L2 until they are read again (fewer DRAM bytes: 1.99 against 2.64 GB
// read at 24^3 x 32 with 18 fields and bz = 12), at the cost of re-reading the z-neighbours at the block
// faces; in time neither order won consistently, so it is a pinned option (RMHMC_SHAPE_ADJOINT).
//   phase 1: thread (hop, site) loads one link -- U_h(x) for the forward hops h < 4, U_{h-4}(x - h) for the
//            backward ones -- and stores Ad (forward) or Ad^T (backward) in shared memory, with the
//            neighbour site of that hop (both as the columns of an adjoint matrix, Ad(U^dag) = Ad(U)^T);
//   phase 2: the 8 threads of a site own the 8 16-byte chunks of its 32 components (chunk j: component j/2,
//            colours 4 (j%2) .. 4 (j%2) + 3), so that one 128-bit load instruction of a warp reads 4 whole
//            128-byte lines (4 sites of one field).  Over the 8 hops a thread accumulates, CH fields at a time,
//            the products of the four matching columns of each adjoint matrix (from shared memory, padded so
//            that a warp's 128-bit reads hit distinct bank quads) with its chunk of the neighbour's value; the
//            two column halves of a component are summed by one lane exchange, each lane keeping the rows of
//            its own chunk.  Y_f(x) is written chunk by chunk, and the per-field dots <Y,Y>, <Y,X> go to
//            per-warp float64 sums (deterministic order).
#include "common.cuh"
#include "ops.cuh"

namespace rm {

constexpr int kAdSites = 32;                 // sites per tile
constexpr int kAdThreads = 256;              // 8 hops x 32 sites in phase 1; 32 sites x 8 chunks in phase 2
constexpr int kAdHop = 64;                   // floats per (site, hop) record: 8 rows x 8
constexpr int kAdSiteStride = 8 * kAdHop + 8;   // 520 floats: = 8 mod 32, so the 8 row halves (4 sites x 2) a
                                                // warp reads in one 128-bit load fall on distinct bank quads
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
                                                        float a, float b, float c, size_t fs, int bz,
                                                        double* partials, unsigned* counters, double* out,
                                                        size_t slot_stride) {
    extern __shared__ __align__(16) float smem[];
    float* ad = smem;                                            // [kAdSites][kAdSiteStride]
    int* nbr = reinterpret_cast<int*>(smem + kAdSmemFloats);     // [kAdSites][8]
    double* dsum = reinterpret_cast<double*>(nbr + kAdSites * 8);   // [warps][nf][2] (DOTS)
    __shared__ double sh[2 * (kAdThreads / 32)];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (DOTS)
        for (int i = t; i < (kAdThreads / 32) * nf * 2; i += kAdThreads) dsum[i] = 0.0;
    // phase-2 role of this thread: site, component, and the parity of its fields
    const int ps = t >> 3, pmu = (t >> 1) & 3, par = t & 1;
    // work units in the order (z block, t, tile): a slab is bz whole xy-planes at one t, cut into tiles of
    // kAdSites consecutive sites
    const int P = g.stride[2], V3 = g.stride[3];
    const int nts = (P * bz + kAdSites - 1) / kAdSites;
    const int nunit = nts * g.L[3] * ((g.L[2] + bz - 1) / bz);
    for (int u = blockIdx.x; u < nunit; u += gridDim.x) {
        const int jt = u % nts, r = u / nts, tt = r % g.L[3], z0 = (r / g.L[3]) * bz;
        const int first = jt * kAdSites;
        const int nvalid = min(kAdSites, P * min(bz, g.L[2] - z0) - first);
        if (nvalid <= 0) continue;   // a tile past the end of a thinner last z block (uniform over the block)
        const int base = tt * V3 + z0 * P + first;
        // ---- phase 1: adjoint matrices of the 8 hops of every site in the tile
        {
            const int sl = t & (kAdSites - 1), hop = t >> 5;
            const int s = base + sl;
            if (sl < nvalid) {
                const int dir = hop & 3;
                const int nb = hop < 4 ? step_site(g, s, dir, 1) : step_site(g, s, dir, -1);
                const mat3<float> u = LinkLoad<float, LF>::load(U, hop < 4 ? s : nb, dir);
                float* rec = ad + sl * kAdSiteStride + hop * kAdHop;
                // record row b = column b of Ad(V): V = U^dag for a forward hop, since Ad(U^dag) = Ad(U)^T gives
                // the rows of Ad(U); V = U for a backward hop, whose record is Ad(U)^T.  Whole rows are stored
                // as two 128-bit words.
                adjoint_columns(hop < 4 ? m_dag(u) : u, [&](int bcol, const float (&col)[8]) {
                    float4* d = reinterpret_cast<float4*>(rec + bcol * 8);
                    d[0] = make_float4(col[0], col[1], col[2], col[3]);
                    d[1] = make_float4(col[4], col[5], col[6], col[7]);
                });
                nbr[sl * 8 + hop] = nb;
            }
        }
        __syncthreads();
        // ---- phase 2
        const int s = base + ps;
        const bool active = ps < nvalid;
        const float* rec0 = ad + ps * kAdSiteStride;
        const int* nb = nbr + ps * 8;
        const float* Xm = X + pmu * 8;
        // fields of this thread: par, par + 2, par + 4, ...; pass p covers the CH fields par + 2 (p CH + q)
        const int mine = (nf - par + 1) / 2;
        // the (pass, hop) iterations are software-pipelined: the neighbour values of the next iteration are
        // loaded before the arithmetic of the current one
        auto load_x = [&](int q0, int hop, float (&x)[CH][8]) {
            const size_t n = (size_t)nb[hop] * 32;
#pragma unroll
            for (int q = 0; q < CH; q++) {
                if (active && q0 + q < mine) load8(Xm + (size_t)(par + 2 * (q0 + q)) * fs + n, x[q]);
                else
#pragma unroll
                    for (int k = 0; k < 8; k++) x[q][k] = 0.f;
            }
        };
        float xb[2][CH][8];
        load_x(0, 0, xb[0]);
        const int npass = (mine + CH - 1) / CH;
        const int npass_blk = ((nf + 1) / 2 + CH - 1) / CH;   // uniform over the block (for the dot shuffles)
        for (int p = 0; p < npass_blk; p++) {
            const int q0 = p * CH;
            float acc[CH][8];
#pragma unroll
            for (int q = 0; q < CH; q++)
#pragma unroll
                for (int r = 0; r < 8; r++) acc[q][r] = 0.f;
            if (p < npass) {
#pragma unroll
                for (int hop = 0; hop < 8; hop++) {
                    // prefetch: the next hop of this pass, or hop 0 of the next pass
                    if (hop < 7) load_x(q0, hop + 1, xb[(hop + 1) & 1]);
                    else if (q0 + CH < mine) load_x(q0 + CH, 0, xb[0]);
                    const float (&x)[CH][8] = xb[hop & 1];
                    const float* rec = rec0 + hop * kAdHop;
#pragma unroll
                    for (int r = 0; r < 8; r++) {
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
            }
            // epilogue: Y_f(s)_mu for the pass's fields, and the dots (every lane joins the shuffles)
#pragma unroll
            for (int q = 0; q < CH; q++) {
                const int fi = q0 + q;                 // index among this thread's fields
                const int f = par + 2 * fi;
                float yy = 0.f, yx = 0.f;
                if (active && fi < mine) {
                    const size_t off = (size_t)f * fs + (size_t)s * 32 + pmu * 8;
                    float xo[8], y[8];
                    load8(X + off, xo);
#pragma unroll
                    for (int r = 0; r < 8; r++) y[r] = fmaf(b, acc[q][r], a * xo[r]);
                    if (HAS_W) {
                        float w[8];
                        load8(W + off, w);
#pragma unroll
                        for (int r = 0; r < 8; r++) y[r] = fmaf(c, w[r], y[r]);
                    }
                    store8(Y + off, y);
                    if (DOTS) {
#pragma unroll
                        for (int r = 0; r < 8; r++) { yy = fmaf(y[r], y[r], yy); yx = fmaf(y[r], xo[r], yx); }
                    }
                }
                if (DOTS) {
                    // lanes of parity par hold field par + 2 fi: reduce each parity over its 16 lanes
#pragma unroll
                    for (int o = 16; o > 1; o >>= 1) {
                        yy += __shfl_xor_sync(0xffffffffu, yy, o);
                        yx += __shfl_xor_sync(0xffffffffu, yx, o);
                    }
                    if (lane < 2 && par + 2 * fi < nf) {
                        dsum[(warp * nf + f) * 2] += (double)yy;
                        dsum[(warp * nf + f) * 2 + 1] += (double)yx;
                    }
                }
            }
        }
        __syncthreads();   // the next unit overwrites the adjoint records
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
constexpr AdShape kAdShapes[2] = {{2, 3}, {3, 2}};

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
    const int bz = ctx->ad_slab > 0 ? ctx->ad_slab : ctx->g.L[2];
    const int P = ctx->g.stride[2];
    const int nunit = (P * bz + kAdSites - 1) / kAdSites * ctx->g.L[3] * ((ctx->g.L[2] + bz - 1) / bz);
    const int grid = std::max(1, std::min(nunit, (int)ctx->num_sms * std::max(per_sm, 1)));
    const size_t ss = (size_t)ctx->max_blocks * 2;
    double* part = DOTS ? red_slot_partials(ctx, slot) : nullptr;
    unsigned* cnt = DOTS ? red_slot_counter(ctx, slot) : nullptr;
    double* out = DOTS ? red_slot_out(ctx, slot) : nullptr;
    kern<<<grid, kAdThreads, smem, st>>>(ctx->g, links32(ctx), X, Y, W, nf, (float)a, (float)b, (float)c, field_elems(ctx),
                                         bz, part, cnt, out, ss);
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
    return launch_ad_shape<LF, 3, 2>(ctx, X, Y, nf, a, b, W, c, slot, st);
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
    for (int k = 0; k < 2; k++) {
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
