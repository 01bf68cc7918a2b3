// Float64-accurate true residuals r_f = b - (A + sigma_f) x_f computed with float32 arithmetic, for the
// reliable updates of the mixed-precision shifted solves (Sec. 3, Eq. 6; the residual check of the
// rational mass term).
//
// GB300 executes float64 at 1/62 of the float32 rate, so the float64 stencil (4608 float64 FMA per site
// and field) costs more than every other part of a Hamiltonian evaluation.  Here:
//  * each link's adjoint matrix Ad(U)_cb = 2 Re Tr(T^c U T^b U^dag) (8x8 real, so that
//    U X U^dag = sum_c (Ad x)_c T^c for X = sum_b x_b T^b) is formed once in float64, scaled by 1/16
//    and stored as a pair of float32 matrices (hi + lo, 48 significant bits);
//  * x_f is split once into float32 pairs (x_hi + x_lo);
//  * every residual component is accumulated as an unevaluated float32 sum (s, c): the exact products
//    hi*hi enter through an error-free product (fma) and an error-free sum (Knuth's TwoSum), the
//    products hi*lo and lo*hi go to c, and lo*lo (2^-48 relative) is dropped.  This is the compensated
//    dot product "Dot2" of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005), whose result is as
//    accurate as if computed in twice the working precision.
// The residual is returned rounded to float32 (the correction solve's right-hand side) together with
// its float64 squared norm.
#include "krylov.cuh"

namespace rm {

// ------------------------------------------------------------------------------------------------
// adjoint table: [V][4][2][64] float32 (hi row-major 8x8 of Ad(U)/16, then lo)
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_adjoint_table(Links64 U, int V, float* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int nu = blockIdx.y;
    if (s >= V) return;
    const mat3<double> u = LinkLoad<double, 18>::load(U, s, nu);
    float* o = out + ((size_t)s * 4 + nu) * 128;
#pragma unroll
    for (int b = 0; b < 8; b++) {
        double e[8];
#pragma unroll
        for (int a = 0; a < 8; a++) e[a] = a == b ? 1.0 : 0.0;
        herm<double> H = h_zero<double>();
        acc_uxud(H, u, coef_to_herm2(e));   // U (2 T^b) U^dag = sum_c Ad_cb (2 T^c)
        double col[8];
        herm2_to_coef(H, col);
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const double v = col[c] * 0.0625;
            const float hi = (float)v;
            o[c * 8 + b] = hi;
            o[64 + c * 8 + b] = (float)(v - (double)hi);
        }
    }
}

// x (float64 [nf][V][4][8]) -> [nf][V][4][16] float32: hi[8] then lo[8] per component
__global__ void k_split_pairs(const double* __restrict__ x, float* __restrict__ out, size_t n8) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += (size_t)gridDim.x * blockDim.x) {
        double v[8];
        load8(x + i * 8, v);
        float h[8], l[8];
#pragma unroll
        for (int a = 0; a < 8; a++) {
            h[a] = (float)v[a];
            l[a] = (float)(v[a] - (double)h[a]);
        }
        store8(out + i * 16, h);
        store8(out + i * 16 + 8, l);
    }
}

// (s, c) += a * b for float32 a, b: the rounded product goes through TwoSum into s, both rounding
// errors into c
__device__ __forceinline__ void dot2_acc(float a, float b, float& s, float& c) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(q, e));
}
__device__ __forceinline__ void ld_pair(const float* p, float (&h)[8], float (&l)[8]) {
    load8(p, h);
    load8(p + 8, l);
}

// one lane per (site, component mu, field f); lanes of one site are adjacent (team of 4 nf) so the
// adjoint rows they read coincide.  r (float32 [nf][V][4][8]).
__global__ void __launch_bounds__(kBlock) k_resid_df(Geom g, const float* __restrict__ Ad, const float* __restrict__ xs,
                                                      const double* __restrict__ b, const double* __restrict__ sig, int nf,
                                                      size_t fs, float* __restrict__ r) {
    const int team = 4 * nf;
    // grid-stride over lanes, carrying (site, rem) = divmod(lane, team) incrementally
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int sq = (int)(stride / team), sr = (int)(stride % team);
    const long long lane0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int site = (int)(lane0 / team), rem = (int)(lane0 % team);
    for (; site < g.V; site += sq, rem += sr, site += rem >= team ? 1 : 0, rem -= rem >= team ? team : 0) {
        const int mu = rem & 3, f = rem >> 2;
        const float* xf = xs + (size_t)f * fs * 2;
        float s[8], c[8];
        {
            // b - (sigma_f + 1/2) x_f(site)
            double bb[8];
            load8(b + (size_t)site * 32 + mu * 8, bb);
            float xh[8], xl[8];
            ld_pair(xf + ((size_t)site * 4 + mu) * 16, xh, xl);
            const double dg = -(sig[f] + 0.5);
            const float dh = (float)dg, dl = (float)(dg - (double)dh);
#pragma unroll
            for (int a = 0; a < 8; a++) {
                const float bh = (float)bb[a];
                s[a] = bh;
                c[a] = (float)(bb[a] - (double)bh);
                dot2_acc(dh, xh[a], s[a], c[a]);
                c[a] = __fmaf_rn(dh, xl[a], __fmaf_rn(dl, xh[a], c[a]));
            }
        }
        int fwd[4], bwd[4];
        neighbours(g, site, fwd, bwd);
#pragma unroll 1
        for (int nu = 0; nu < 4; nu++) {
            // forward hop: + Ad(U_nu(site)) x(site + nu) / 16
            {
                float xh[8], xl[8];
                ld_pair(xf + ((size_t)fwd[nu] * 4 + mu) * 16, xh, xl);
                const float* R = Ad + ((size_t)site * 4 + nu) * 128;
#pragma unroll
                for (int cc = 0; cc < 8; cc++) {
                    float rh[8], rl[8];
                    load8(R + cc * 8, rh);
                    load8(R + 64 + cc * 8, rl);
                    float lo = 0.f;
#pragma unroll
                    for (int k = 0; k < 8; k++) {
                        dot2_acc(rh[k], xh[k], s[cc], c[cc]);
                        lo = __fmaf_rn(rh[k], xl[k], __fmaf_rn(rl[k], xh[k], lo));
                    }
                    c[cc] = __fadd_rn(c[cc], lo);
                }
            }
            // backward hop: + Ad(U_nu(site - nu))^T x(site - nu) / 16
            {
                float xh[8], xl[8];
                ld_pair(xf + ((size_t)bwd[nu] * 4 + mu) * 16, xh, xl);
                const float* R = Ad + ((size_t)bwd[nu] * 4 + nu) * 128;
                float lo[8];
#pragma unroll
                for (int cc = 0; cc < 8; cc++) lo[cc] = 0.f;
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    float rh[8], rl[8];
                    load8(R + k * 8, rh);
                    load8(R + 64 + k * 8, rl);
#pragma unroll
                    for (int cc = 0; cc < 8; cc++) {
                        dot2_acc(rh[cc], xh[k], s[cc], c[cc]);
                        lo[cc] = __fmaf_rn(rh[cc], xl[k], __fmaf_rn(rl[cc], xh[k], lo[cc]));
                    }
                }
#pragma unroll
                for (int cc = 0; cc < 8; cc++) c[cc] = __fadd_rn(c[cc], lo[cc]);
            }
        }
        float out[8];
#pragma unroll
        for (int a = 0; a < 8; a++) out[a] = __fadd_rn(s[a], c[a]);
        store8(r + (size_t)f * fs + (size_t)site * 32 + mu * 8, out);
    }
}

// squared norms of nf float32 fields (float64 sums, deterministic), field f in blockIdx.y
__global__ void __launch_bounds__(kBlock) k_norm2_fields(const float* __restrict__ x, size_t fs, double* partials,
                                                          unsigned* counters, double* out, size_t slot_stride) {
    __shared__ double sh[kBlock / 32];
    const int f = blockIdx.y;
    const float4* p = reinterpret_cast<const float4*>(x + (size_t)f * fs);
    double acc = 0.0;
    float accf = 0.f;
    int cnt = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < fs / 4; i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = p[i];
        accf = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, accf))));
        if (++cnt == 64) { acc += (double)accf; accf = 0.f; cnt = 0; }
    }
    acc += (double)accf;
    double v[1] = {acc};
    block_sum<1>(v, sh);
    grid_sum_finish<1>(v, partials + f * slot_stride, counters + f, out + (size_t)f * 8, gridDim.x, blockIdx.x, sh);
}

int adjoint_table(rmhmc_ctx* ctx, float** tab, cudaStream_t st) {
    int status = RMHMC_OK;
    const unsigned long long ws = ctx->ws_gen;
    float* t = (float*)workspace(ctx, "rd_adjoint", sizeof(float) * (size_t)ctx->g.V * 4 * 128, &status);
    if (!t) return status;
    *tab = t;
    // the table of the current links is kept until they change (a heatbath and the Hamiltonian that follows
    // share it)
    if (ctx->adj_gen == ctx->link_gen && ws == ctx->ws_gen) return RMHMC_OK;
    const dim3 grid(site_blocks(ctx), 4);
    k_adjoint_table<<<grid, kBlock, 0, st>>>(links64(ctx), ctx->g.V, t); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    ctx->adj_gen = ctx->link_gen;
    return RMHMC_OK;
}

int resid_df(rmhmc_ctx* ctx, const float* tab, const double* b, const double* x, int nf, const double* sigma, float* r,
             double* norm2, cudaStream_t st) {
    if (nf > kRedSlots - kSlotResid) return set_err(ctx, RMHMC_EINVAL, "too many shifts for one residual launch");
    int status = RMHMC_OK;
    const size_t fs = field_elems(ctx);
    float* xs = (float*)workspace(ctx, "rd_pairs", sizeof(float) * fs * 2 * (size_t)nf, &status);
    double* dsig = (double*)workspace(ctx, "rd_sig", sizeof(double) * 64, &status);
    if (!xs || !dsig) return status;
    RM_TRY(upload(ctx, dsig, sigma, sizeof(double) * nf, st));
    const size_t n8 = fs / 8 * (size_t)nf;
    k_split_pairs<<<capped_grid(ctx, n8, kBlock), kBlock, 0, st>>>(x, xs, n8); ++ctx->launches;
    const size_t lanes = (size_t)ctx->g.V * 4 * nf;
    k_resid_df<<<capped_grid(ctx, lanes, kBlock), kBlock, 0, st>>>(ctx->g, tab, xs, b, dsig, nf, fs, r);
    ++ctx->launches;
    const dim3 grid(capped_grid(ctx, fs / 4, kBlock), nf);
    k_norm2_fields<<<grid, kBlock, 0, st>>>(r, fs, red_slot_partials(ctx, kSlotResid), red_slot_counter(ctx, kSlotResid),
                                            red_slot_out(ctx, kSlotResid), (size_t)ctx->max_blocks * 2); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    std::vector<double> out((size_t)nf * 8);
    RM_TRY(fetch(ctx, red_slot_out(ctx, kSlotResid), out.data(), (int)out.size(), st));
    for (int f = 0; f < nf; f++) norm2[f] = out[(size_t)f * 8];
    return RMHMC_OK;
}

}  // namespace rm
