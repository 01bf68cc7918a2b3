// Sec. 2, Eq. (3) for one field, link by link: every link U_nu(x) is turned into its adjoint matrix
// Ad = Ad(U_nu(x)) once and serves both hops that cross it,
//   forward  (to x):      F = Ad X(x+nu)      (U X(x+nu) U^dag in coefficients)
//   backward (to x+nu):   B = Ad^T X(x)       (U^dag X(x) U),
// so that H(X)(x) = sum_nu [F_nu(x) + B_nu(x-nu)] costs 4 adjoint builds and 8 x 4 8x8 products per site
// instead of 8 x 4 3x3 conjugations (about 3600 against 4700 FP32 operations per site).
//
// The backward contributions travel to the neighbouring site, so the lattice is cut into 4D-blocked tiles
// that sweep through time: a block owns an xyz box of sites (up to 8 x 4 x 2) and walks its t-range one
// slice at a time.  Four threads per site, one per link direction nu.  Per slice:
//   * the own field X(x) is staged in shared memory (transposed per colour component);
//   * thread (x, nu) streams the rows of Ad(U_nu(x)) -- built as the columns of Ad(U^dag) -- and forms the
//     forward rows (to shared memory, summed over nu later) and accumulates B in registers;
//   * B goes to the slot of the target site in shared memory when the target lies in the box, and to a
//     double-buffered slot for the next slice when nu = t;
//   * the box's low faces take their backward contributions from links outside the box: extra threads
//     recompute those (the halo), and the first slice of a t-range recomputes its t-halo;
//   * thread (x, mu) then sums its component and applies the epilogue (lap_apply: Y = a X + b H; the CG
//     stencil: q = (0.5 + sigma0) r - H(r)/16 + beta q_old with the dot <r, q>).
// Every slot is written exactly once per slice, and every sum has a fixed order (deterministic results).
#include "common.cuh"
#include "ops.cuh"
#include "tune.cuh"

namespace rm {

constexpr int kLcSites = 64;                 // sites per box
constexpr int kLcThreads = 4 * kLcSites;     // one thread per (site, link direction)
constexpr int kLcBox[3] = {8, 4, 2};         // box extents in x, y, z (clipped to the lattice)
constexpr int kLcTLen = 8;                   // slices per t-range
// shared-memory layout (floats); the paddings keep the 128-bit reads and the scalar writes of a warp on
// distinct bank quads
constexpr int kLcXO = 36;                    // own field per site: [a][mu] (8 x 4) + 4
constexpr int kLcFS = 164;                   // forward rows per site: [mu][a][nu] at mu stride 36, + pad (= 4 mod 32)
constexpr int kLcFmu = 36;
constexpr int kLcBS = 100;                   // backward slots per site: [d = x, y, z][mu][8] + 4
constexpr int kLcBT = 36;                    // t-backward slot per site: [mu][8] + 4
constexpr int kLcSmemFloats = kLcSites * (kLcXO + kLcFS + kLcBS + 2 * kLcBT);

struct LcGeom {
    int b[3];       // box extents
    int nb[3];      // boxes per direction
    int full[3];    // the box spans the whole extent (its neighbours wrap inside the box)
    int nt;         // t-ranges
};

inline LcGeom lc_geom(const Geom& g) {
    LcGeom lg{};
    for (int d = 0; d < 3; d++) {
        lg.b[d] = std::min(kLcBox[d], g.L[d]);
        lg.nb[d] = (g.L[d] + lg.b[d] - 1) / lg.b[d];
        lg.full[d] = lg.b[d] >= g.L[d];
    }
    lg.nt = (g.L[3] + kLcTLen - 1) / kLcTLen;
    return lg;
}
inline int lc_blocks(const Geom& g) {
    const LcGeom lg = lc_geom(g);
    return lg.nb[0] * lg.nb[1] * lg.nb[2] * lg.nt;
}

// B = Ad(u)^T x for the four components (x[mu][a] in registers), rows of Ad streamed
template <class RowSink>
__device__ __forceinline__ void lc_rows(const mat3<float>& u, RowSink&& sink) {
    adjoint_columns(m_dag(u), sink);   // column a of Ad(U^dag) is row a of Ad(U)
}

// MODE 0: Y = a X + b H(X).  MODE 1: q = c0 r + b H(r) + beta q_old (k > 0), gamma = <r, q> (CG stencil;
// X = r_k is basis vector k of R, flags/vals as in k_cg_A)
template <int LF, int MODE>
__global__ void __launch_bounds__(kLcThreads, 2) k_lap_lc(Geom g, LcGeom lg, Links32 U, const float* __restrict__ Xin,
                                                          float* __restrict__ Y, float a, float b, size_t fs,
                                                          const int* __restrict__ flags, double* vals, int maxit,
                                                          double* partials, unsigned* counter) {
    extern __shared__ __align__(16) float sm[];
    float* XO = sm;                                   // [site][kLcXO]
    float* FS = XO + kLcSites * kLcXO;                // [site][kLcFS]
    float* BS = FS + kLcSites * kLcFS;                // [site][kLcBS]
    float* BT = BS + kLcSites * kLcBS;                // [2][site][kLcBT]
    __shared__ double sh[kLcThreads / 32];
    const float* X = Xin;
    float beta = 0.f;
    int k = 0;
    if (MODE == 1) {
        if (flags[0]) return;
        k = flags[1];
        X = Xin + (size_t)k * fs;
        if (k > 0) beta = (float)vals[(maxit + 1) + 2 * maxit + (k - 1)];
    }
    const int tid = threadIdx.x, s = tid >> 2, nu = tid & 3;
    // box and t-range of this block
    int bi = blockIdx.x;
    const int tr = bi % lg.nt; bi /= lg.nt;
    const int bxi = bi % lg.nb[0]; bi /= lg.nb[0];
    const int byi = bi % lg.nb[1]; bi /= lg.nb[1];
    const int bzi = bi;
    // box origin and actual extents (the last box along a direction may be shorter); scalars throughout, so
    // that no array is indexed at run time (which would place it in local memory)
    const int c0x = bxi * lg.b[0], c0y = byi * lg.b[1], c0z = bzi * lg.b[2];
    const int ex = min(lg.b[0], g.L[0] - c0x), ey = min(lg.b[1], g.L[1] - c0y), ez = min(lg.b[2], g.L[2] - c0z);
    const bool fx = lg.full[0], fy = lg.full[1], fz = lg.full[2];
    const int nsite = ex * ey * ez;
    const int t0 = tr * kLcTLen, t1 = min(g.L[3], t0 + kLcTLen);
    const bool live = s < nsite;
    int ix = 0, iy = 0, iz = 0;
    if (live) { ix = s % ex; iy = (s / ex) % ey; iz = s / (ex * ey); }
    const int gx = c0x + ix, gy = c0y + iy, gz = c0z + iz;
    const int xyz = gx + g.L[0] * (gy + g.L[1] * gz);
    const int slice = g.stride[3];
    // local index of the box site one step forward along d < 3 (-1 when it lies outside the box)
    auto fwd_local = [&](int d) {
        int jx = ix, jy = iy, jz = iz;
        if (d == 0) { jx++; if (jx >= ex) { if (!fx) return -1; jx = 0; } }
        else if (d == 1) { jy++; if (jy >= ey) { if (!fy) return -1; jy = 0; } }
        else { jz++; if (jz >= ez) { if (!fz) return -1; jz = 0; } }
        return jx + ex * (jy + ey * jz);
    };
    // the xyz part of the site one step forward along d < 3, periodic
    auto fwd_xyz = [&](int d) {
        if (d == 0) return gx + 1 == g.L[0] ? xyz - gx : xyz + 1;
        if (d == 1) return gy + 1 == g.L[1] ? xyz - gy * g.stride[1] : xyz + g.stride[1];
        return gz + 1 == g.L[2] ? xyz - gz * g.stride[2] : xyz + g.stride[2];
    };
    // halo tasks of a slice: the low faces of the box along x, y, z that are not full (one link each)
    const int hx = fx ? 0 : ey * ez, hy = fy ? 0 : ex * ez, hz = fz ? 0 : ex * ey;
    const int nhalo = hx + hy + hz;
    // B = Ad(U_d(site))^T X(site) into dst[mu * 8 + b]
    auto backward_only = [&](int lsite, int d, float* dst) {
        const mat3<float> u = LinkLoad<float, LF>::load(U, lsite, d);
        float xo[4][8];
#pragma unroll
        for (int m = 0; m < 4; m++) load8(X + (size_t)lsite * 32 + m * 8, xo[m]);
        float B[4][8];
#pragma unroll
        for (int m = 0; m < 4; m++)
#pragma unroll
            for (int c = 0; c < 8; c++) B[m][c] = 0.f;
        lc_rows(u, [&](int ra, const float (&row)[8]) {
#pragma unroll
            for (int m = 0; m < 4; m++)
#pragma unroll
                for (int c = 0; c < 8; c++) B[m][c] = fmaf(row[c], xo[m][ra], B[m][c]);
        });
#pragma unroll
        for (int m = 0; m < 4; m++) {
            float4* q = reinterpret_cast<float4*>(dst + m * 8);
            q[0] = make_float4(B[m][0], B[m][1], B[m][2], B[m][3]);
            q[1] = make_float4(B[m][4], B[m][5], B[m][6], B[m][7]);
        }
    };
    float dot = 0.f;
    int cur = 0;
    // t-halo: B_t of the links U_t(x, t0 - 1) for the first slice
    if (nu == 0 && live) {
        const int tp = t0 == 0 ? g.L[3] - 1 : t0 - 1;
        backward_only(xyz + tp * slice, 3, BT + (size_t)s * kLcBT);
    }
    for (int t = t0; t < t1; t++) {
        const int x = xyz + t * slice;
        // own field, transposed: XO[s][a * 4 + mu]
        if (live) {
            float v[8];
            load8(X + (size_t)x * 32 + nu * 8, v);
#pragma unroll
            for (int c = 0; c < 8; c++) XO[s * kLcXO + c * 4 + nu] = v[c];
        }
        __syncthreads();
        if (live) {
            // the link U_nu(x) and the field one step forward
            const int xf_site = nu < 3 ? fwd_xyz(nu) + t * slice : xyz + (t + 1 == g.L[3] ? 0 : t + 1) * slice;
            const mat3<float> u = LinkLoad<float, LF>::load(U, x, nu);
            float xf[4][8];
#pragma unroll
            for (int m = 0; m < 4; m++) load8(X + (size_t)xf_site * 32 + m * 8, xf[m]);
            float B[4][8];
#pragma unroll
            for (int m = 0; m < 4; m++)
#pragma unroll
                for (int c = 0; c < 8; c++) B[m][c] = 0.f;
            float* fs_out = FS + s * kLcFS + nu;
            const float* xo = XO + s * kLcXO;
            lc_rows(u, [&](int ra, const float (&row)[8]) {
                // forward row ra: F[mu][ra] = row . X(x+nu)_mu
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    float f = 0.f;
#pragma unroll
                    for (int c = 0; c < 8; c++) f = fmaf(row[c], xf[m][c], f);
                    fs_out[m * kLcFmu + ra * 4] = f;
                }
                // backward: B[mu][c] += Ad[ra][c] X(x)_mu[ra]
                const float4 xq = *reinterpret_cast<const float4*>(xo + ra * 4);
                const float xm[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
                for (int m = 0; m < 4; m++)
#pragma unroll
                    for (int c = 0; c < 8; c++) B[m][c] = fmaf(row[c], xm[m], B[m][c]);
            });
            float* dst = nullptr;
            if (nu == 3) {
                dst = BT + (size_t)((cur ^ 1) * kLcSites + s) * kLcBT;
            } else {
                const int tl = fwd_local(nu);
                if (tl >= 0) dst = BS + tl * kLcBS + nu * 32;
            }
            if (dst) {
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    float4* q = reinterpret_cast<float4*>(dst + m * 8);
                    q[0] = make_float4(B[m][0], B[m][1], B[m][2], B[m][3]);
                    q[1] = make_float4(B[m][4], B[m][5], B[m][6], B[m][7]);
                }
            }
        }
        // halo: backward contributions into the box's low faces from links outside it
        for (int h = tid; h < nhalo; h += kLcThreads) {
            // face site (coordinate d = 0 in the box) and the lattice site one step below it along d
            int d, jx, jy, jz;
            if (h < hx) { d = 0; jx = 0; jy = h % ey; jz = h / ey; }
            else if (h < hx + hy) { d = 1; const int r = h - hx; jy = 0; jx = r % ex; jz = r / ex; }
            else { d = 2; const int r = h - hx - hy; jz = 0; jx = r % ex; jy = r / ex; }
            const int ls = jx + ex * (jy + ey * jz);
            int bx = c0x + jx, by = c0y + jy, bz = c0z + jz;
            if (d == 0) bx = bx == 0 ? g.L[0] - 1 : bx - 1;
            else if (d == 1) by = by == 0 ? g.L[1] - 1 : by - 1;
            else bz = bz == 0 ? g.L[2] - 1 : bz - 1;
            const int site = bx + g.L[0] * (by + g.L[1] * bz) + t * slice;
            backward_only(site, d, BS + ls * kLcBS + d * 32);
        }
        __syncthreads();
        // sum per (site, mu = nu) and the epilogue
        if (live) {
            const int m = nu;
            float H[8];
            const float* fr = FS + s * kLcFS + m * kLcFmu;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const float4 q = *reinterpret_cast<const float4*>(fr + c * 4);
                H[c] = (q.x + q.y) + (q.z + q.w);
            }
            const float* bt = BT + (size_t)(cur * kLcSites + s) * kLcBT + m * 8;
            const float* b0 = BS + s * kLcBS + m * 8;
#pragma unroll
            for (int c = 0; c < 8; c++) H[c] += ((b0[c] + b0[32 + c]) + b0[64 + c]) + bt[c];
            float xo[8], y[8];
#pragma unroll
            for (int c = 0; c < 8; c++) xo[c] = XO[s * kLcXO + c * 4 + m];
            float* out = Y + (size_t)x * 32 + m * 8;
            if (MODE == 0) {
#pragma unroll
                for (int c = 0; c < 8; c++) y[c] = fmaf(b, H[c], a * xo[c]);
            } else {
                if (k > 0) {
                    float qo[8];
                    load8(out, qo);
#pragma unroll
                    for (int c = 0; c < 8; c++) y[c] = fmaf(beta, qo[c], fmaf(b, H[c], a * xo[c]));
                } else {
#pragma unroll
                    for (int c = 0; c < 8; c++) y[c] = fmaf(b, H[c], a * xo[c]);
                }
#pragma unroll
                for (int c = 0; c < 8; c++) dot = fmaf(xo[c], y[c], dot);
            }
            store8(out, y);
        }
        cur ^= 1;
        __syncthreads();
    }
    if (MODE == 1) {
        float fv[1] = {dot};
        block_sum_f<1>(fv, sh);
        double v[1] = {0.0};
        if (threadIdx.x == 0)
            for (int w = 0; w < kLcThreads / 32; w++) v[0] += sh[w];
        double* gamma = vals + (maxit + 1);
        double* alpha = gamma + maxit;
        double res[1];
        if (grid_sum_finish<1>(v, partials, counter, res, gridDim.x, blockIdx.x, sh)) {
            gamma[k] = res[0];
            alpha[k] = vals[k] / res[0];
        }
    }
}

template <int LF, int MODE>
static int launch_lc_t(rmhmc_ctx* ctx, const float* X, float* Y, double a, double b, const int* flags, double* vals,
                       int maxit, double* partials, unsigned* counter, cudaStream_t st) {
    auto kern = k_lap_lc<LF, MODE>;
    static bool configured[64] = {};
    const size_t smem = sizeof(float) * kLcSmemFloats;
    if (ctx->device < 0 || ctx->device >= 64) return set_err(ctx, RMHMC_EINVAL, "device index too large");
    if (!configured[ctx->device]) {
        RM_CHECK(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured[ctx->device] = true;
    }
    const int grid = lc_blocks(ctx->g);
    if (MODE == 1 && grid > ctx->max_blocks) return set_err(ctx, RMHMC_EINVAL, "link-centric grid above the reduction slots");
    kern<<<grid, kLcThreads, smem, st>>>(ctx->g, lc_geom(ctx->g), links32(ctx), X, Y, (float)a, (float)b,
                                                       field_elems(ctx), flags, vals, maxit, partials, counter);
    ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}

int launch_lap_lc(rmhmc_ctx* ctx, int linkfmt, const float* X, float* Y, double a, double b, cudaStream_t st) {
    if (linkfmt == 12) return launch_lc_t<12, 0>(ctx, X, Y, a, b, nullptr, nullptr, 0, nullptr, nullptr, st);
    return launch_lc_t<18, 0>(ctx, X, Y, a, b, nullptr, nullptr, 0, nullptr, nullptr, st);
}

int launch_cg_lc(rmhmc_ctx* ctx, const float* R, float* q, double diag, const int* flags, double* vals, int maxit,
                 double* partials, unsigned* counter, cudaStream_t st) {
    return launch_lc_t<18, 1>(ctx, R, q, diag, -0.0625, flags, vals, maxit, partials, counter, st);
}

}  // namespace rm
