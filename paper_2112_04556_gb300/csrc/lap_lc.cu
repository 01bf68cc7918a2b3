// Sec. 2, Eq. (3) for one field, link by link: every link U_nu(x) is turned into its adjoint matrix
// Ad = Ad(U_nu(x)) once and serves both hops that cross it,
//   forward  (to x):      F = Ad X(x+nu)      (U X(x+nu) U^dag in coefficients)
//   backward (to x+nu):   B = Ad^T X(x)       (U^dag X(x) U),
// so that H(X)(x) = sum_nu [F_nu(x) + B_nu(x-nu)] costs 4 adjoint builds and 8 x 4 8x8 products per site
// instead of 8 x 4 3x3 conjugations (about 3600 against 4700 FP32 operations per site).
//
// The backward contributions travel to the neighbouring site, so the lattice is cut into 4D-blocked tiles
// that sweep through time: a block owns an xyz box of sites (up to 8 x 4 x 2) and walks its t-range one
// slice at a time, four threads per site (one per link direction nu).  Per slice:
//   * the field of the box and of its one-site halo (the sites one step beyond each face) sits in shared
//     memory, copied in asynchronously (cp.async) while the previous slice computes (double buffer);
//   * the links of the slice were loaded into registers during the previous slice's epilogue, and so was
//     X(x, t+1) for the t-direction thread;
//   * halo first: the box's low faces get their backward contributions from links outside the box, each
//     such link split over four threads by field component so that every thread has at most one task;
//   * thread (x, nu) streams the rows of Ad(U_nu(x)) (the columns of Ad(U^dag)); each forward row is summed
//     over the four link directions of the site with a fixed 3-shuffle transpose-sum, and B accumulates in
//     registers and goes to the shared slot of the target site (the next slice's slot when nu = t);
//   * thread (x, mu) applies the epilogue (lap_apply: Y = a X + b H; the CG stencil:
//     q = (0.5 + sigma0) r - H(r)/16 + beta q_old with the dot <r, q>).
// Every slot is written exactly once per slice, and every sum has a fixed order (deterministic results).
#include "common.cuh"
#include "ops.cuh"
#include "tune.cuh"

namespace rm {

constexpr int kLcSites = 64;                 // sites per box
constexpr int kLcThreads = 4 * kLcSites;     // one thread per (site, link direction)
constexpr int kLcBox[3] = {8, 4, 2};         // box extents in x, y, z (clipped to the lattice)
constexpr int kLcTLen = 8;                   // slices per t-range
constexpr int kLcFaceMax = 8 + 16 + 32;      // face sites of the largest box (4x2 + 8x2 + 8x4)
constexpr int kLcSlots = kLcSites + 2 * kLcFaceMax;   // field slots: box, high-face and low-face neighbours
// shared-memory layout (floats); the paddings keep a warp's 128-bit reads on distinct bank quads
constexpr int kLcRow = 36;                   // field slot: [mu][a] (32) + 4
constexpr int kLcBS = 100;                   // backward slots per site: [d = x, y, z][mu][8] + 4
constexpr int kLcBT = 36;                    // t-backward slot per site: [mu][8] + 4
constexpr int kLcSmemFloats = 2 * kLcSlots * kLcRow + kLcSites * kLcBS + 2 * kLcSites * kLcBT + kLcSlots;

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

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// rows of Ad(u), streamed (column a of Ad(u^dag) is row a of Ad(u))
template <class RowSink>
__device__ __forceinline__ void lc_rows(const mat3<float>& u, RowSink&& sink) {
    adjoint_columns(m_dag(u), sink);
}

// sum over the four link-direction lanes of a site of f[mu], returned in the lane whose nu equals mu
// (fixed order: pairs across bit 1 first, then across bit 0)
__device__ __forceinline__ float quad_transpose_sum(const float (&f)[4], int nu) {
    const bool hi = nu & 2, odd = nu & 1;
    const float r0 = __shfl_xor_sync(0xffffffffu, hi ? f[0] : f[2], 2);
    const float r1 = __shfl_xor_sync(0xffffffffu, hi ? f[1] : f[3], 2);
    const float k0 = (hi ? f[2] : f[0]) + r0, k1 = (hi ? f[3] : f[1]) + r1;
    const float r = __shfl_xor_sync(0xffffffffu, odd ? k0 : k1, 1);
    return (odd ? k1 : k0) + r;
}

// MODE 0: Y = a X + b H(X).  MODE 1: q = a r + b H(r) + beta q_old (k > 0), gamma = <r, q> (CG stencil;
// X = r_k is basis vector k of R, flags/vals as in k_cg_A)
template <int LF, int MODE>
__global__ void __launch_bounds__(kLcThreads, 1) k_lap_lc(Geom g, LcGeom lg, Links32 U, const float* __restrict__ Xin,
                                                          float* __restrict__ Y, float a, float b, size_t fs,
                                                          const int* __restrict__ flags, double* vals, int maxit,
                                                          double* partials, unsigned* counter) {
    extern __shared__ __align__(16) float sm[];
    float* XO = sm;                                       // [2][kLcSlots][kLcRow]
    float* BS = XO + 2 * kLcSlots * kLcRow;               // [site][kLcBS]
    float* BT = BS + kLcSites * kLcBS;                    // [2][site][kLcBT]
    int* slot_xyz = reinterpret_cast<int*>(BT + 2 * kLcSites * kLcBT);   // [kLcSlots]: xyz part of each slot's site
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
    const int slice = g.stride[3];
    const int Lt = g.L[3];
    // face sizes (0 along a direction the box spans) and their offsets in the slot list
    const int hx = fx ? 0 : ey * ez, hy = fy ? 0 : ex * ez, hz = fz ? 0 : ex * ey;
    const int nhalo = hx + hy + hz;
    const int hiB = kLcSites, loB = kLcSites + nhalo;     // first high-face and low-face slot
    // xyz index of the lattice site at box coordinates (jx, jy, jz) shifted by n along d (periodic)
    auto site_xyz = [&](int jx, int jy, int jz, int d, int n) {
        int gx = c0x + jx, gy = c0y + jy, gz = c0z + jz;
        if (d == 0) { gx += n; gx = gx < 0 ? gx + g.L[0] : gx >= g.L[0] ? gx - g.L[0] : gx; }
        else if (d == 1) { gy += n; gy = gy < 0 ? gy + g.L[1] : gy >= g.L[1] ? gy - g.L[1] : gy; }
        else if (d == 2) { gz += n; gz = gz < 0 ? gz + g.L[2] : gz >= g.L[2] ? gz - g.L[2] : gz; }
        return gx + g.L[0] * (gy + g.L[1] * gz);
    };
    // face index f (< hx, hy or hz) of direction d -> box coordinates of the face site (i_d = i)
    auto face_site = [&](int d, int f, int i, int& jx, int& jy, int& jz) {
        if (d == 0) { jx = i; jy = f % ey; jz = f / ey; }
        else if (d == 1) { jy = i; jx = f % ex; jz = f / ex; }
        else { jz = i; jx = f % ex; jy = f / ex; }
    };
    // slot table: box sites, then the sites one step beyond the high faces, then one step below the low faces
    for (int sl = tid; sl < kLcSlots; sl += kLcThreads) {
        int v = -1;
        if (sl < nsite) {
            v = site_xyz(sl % ex, (sl / ex) % ey, sl / (ex * ey), 3, 0);
        } else if (sl >= hiB && sl < hiB + 2 * nhalo) {
            const bool high = sl < loB;
            int f = sl - (high ? hiB : loB), d = 0;
            if (f >= hx) { f -= hx; d = 1; if (f >= hy) { f -= hy; d = 2; } }
            const int ed = d == 0 ? ex : d == 1 ? ey : ez;
            int jx, jy, jz;
            face_site(d, f, high ? ed - 1 : 0, jx, jy, jz);
            v = site_xyz(jx, jy, jz, d, high ? 1 : -1);
        }
        slot_xyz[sl] = v;
    }
    __syncthreads();
    // copy the field of slice t into buffer buf (asynchronous)
    auto stage = [&](int t, int buf) {
        float* dst = XO + buf * kLcSlots * kLcRow;
        for (int idx = tid; idx < kLcSlots * 8; idx += kLcThreads) {
            const int sl = idx >> 3, c = idx & 7;
            const int v = slot_xyz[sl];
            if (v >= 0) cp_async16(dst + sl * kLcRow + c * 4, X + ((size_t)v + (size_t)t * slice) * 32 + c * 4);
        }
    };
    // this thread's site (dead threads of a partial box compute on site 0 and store nothing)
    const bool live = s < nsite;
    const int sx = live ? s : 0;
    const int ix = sx % ex, iy = (sx / ex) % ey, iz = sx / (ex * ey);
    const int xyz = slot_xyz[sx];
    // slot of the forward neighbour along d < 3, and whether it is a box site (its B lands in this box)
    int nb_slot = 0, tgt_local = -1;
    if (nu < 3) {
        const int ed = nu == 0 ? ex : nu == 1 ? ey : ez;
        const bool fd = nu == 0 ? fx : nu == 1 ? fy : fz;
        const int id = nu == 0 ? ix : nu == 1 ? iy : iz;
        if (id + 1 < ed || fd) {
            const int jx = nu == 0 ? (id + 1 < ed ? ix + 1 : 0) : ix;
            const int jy = nu == 1 ? (id + 1 < ed ? iy + 1 : 0) : iy;
            const int jz = nu == 2 ? (id + 1 < ed ? iz + 1 : 0) : iz;
            tgt_local = jx + ex * (jy + ey * jz);
            nb_slot = tgt_local;
        } else {
            const int off = nu == 0 ? 0 : nu == 1 ? hx : hx + hy;
            const int f = nu == 0 ? iy + ey * iz : nu == 1 ? ix + ex * iz : ix + ex * iy;
            nb_slot = hiB + off + f;
        }
    }
    // halo task of this thread: link hl of the low faces, component hmu
    const bool has_halo = tid < 4 * nhalo;
    int h_d = 0, h_local = 0, h_slot = 0, h_xyz = 0;
    const int hmu = tid & 3;
    if (has_halo) {
        int f = tid >> 2;
        h_slot = loB + f;
        if (f >= hx) { f -= hx; h_d = 1; if (f >= hy) { f -= hy; h_d = 2; } }
        int jx, jy, jz;
        face_site(h_d, f, 0, jx, jy, jz);
        h_local = jx + ex * (jy + ey * jz);
        h_xyz = slot_xyz[h_slot];
    }
    // first slice: field (synchronous), t-halo B_t(x, t0 - 1) split by component, prefetched registers
    stage(t0, t0 & 1);
    {
        const int tp = t0 == 0 ? Lt - 1 : t0 - 1;
        const int m = nu;   // component of the t-halo task
        const mat3<float> u = LinkLoad<float, LF>::load(U, xyz + tp * slice, 3);
        float xm[8];
        load8(X + ((size_t)xyz + (size_t)tp * slice) * 32 + m * 8, xm);
        float Bm[8];
#pragma unroll
        for (int c = 0; c < 8; c++) Bm[c] = 0.f;
        lc_rows(u, [&](int ra, const float (&row)[8]) {
#pragma unroll
            for (int c = 0; c < 8; c++) Bm[c] = fmaf(row[c], xm[ra], Bm[c]);
        });
        if (live) {
            float4* q = reinterpret_cast<float4*>(BT + (size_t)((t0 & 1) * kLcSites + s) * kLcBT + m * 8);
            q[0] = make_float4(Bm[0], Bm[1], Bm[2], Bm[3]);
            q[1] = make_float4(Bm[4], Bm[5], Bm[6], Bm[7]);
        }
    }
    mat3<float> u = LinkLoad<float, LF>::load(U, xyz + t0 * slice, nu);
    mat3<float> uh;
    if (has_halo) uh = LinkLoad<float, LF>::load(U, h_xyz + t0 * slice, h_d);
    float xf[4][8];
    if (nu == 3) {
        const int tn = t0 + 1 == Lt ? 0 : t0 + 1;
#pragma unroll
        for (int m = 0; m < 4; m++) load8(X + ((size_t)xyz + (size_t)tn * slice) * 32 + m * 8, xf[m]);
    }
    cp_async_wait_all();
    __syncthreads();
    float dot = 0.f;
    for (int t = t0; t < t1; t++) {
        const int cur = t & 1;
        const float* XC = XO + cur * kLcSlots * kLcRow;
        if (t + 1 < t1) stage(t + 1, cur ^ 1);
        // ---- halo: B_d of the low-face links, component hmu
        if (has_halo) {
            float xm[8], Bm[8];
            {
                const float4* p = reinterpret_cast<const float4*>(XC + h_slot * kLcRow + hmu * 8);
                const float4 v0 = p[0], v1 = p[1];
                xm[0] = v0.x; xm[1] = v0.y; xm[2] = v0.z; xm[3] = v0.w; xm[4] = v1.x; xm[5] = v1.y; xm[6] = v1.z; xm[7] = v1.w;
            }
#pragma unroll
            for (int c = 0; c < 8; c++) Bm[c] = 0.f;
            lc_rows(uh, [&](int ra, const float (&row)[8]) {
#pragma unroll
                for (int c = 0; c < 8; c++) Bm[c] = fmaf(row[c], xm[ra], Bm[c]);
            });
            float4* q = reinterpret_cast<float4*>(BS + h_local * kLcBS + h_d * 32 + hmu * 8);
            q[0] = make_float4(Bm[0], Bm[1], Bm[2], Bm[3]);
            q[1] = make_float4(Bm[4], Bm[5], Bm[6], Bm[7]);
        }
        // ---- main: the link U_nu(x); forward rows summed over nu into Hs, backward B to the target slot
        if (nu < 3) {
#pragma unroll
            for (int m = 0; m < 4; m++) {
                const float4* p = reinterpret_cast<const float4*>(XC + nb_slot * kLcRow + m * 8);
                const float4 v0 = p[0], v1 = p[1];
                xf[m][0] = v0.x; xf[m][1] = v0.y; xf[m][2] = v0.z; xf[m][3] = v0.w;
                xf[m][4] = v1.x; xf[m][5] = v1.y; xf[m][6] = v1.z; xf[m][7] = v1.w;
            }
        }
        float B[4][8], Hs[8];
#pragma unroll
        for (int m = 0; m < 4; m++)
#pragma unroll
            for (int c = 0; c < 8; c++) B[m][c] = 0.f;
        const float* xo = XC + sx * kLcRow;
        lc_rows(u, [&](int ra, const float (&row)[8]) {
            float f[4];
#pragma unroll
            for (int m = 0; m < 4; m++) {
                float v = 0.f;
#pragma unroll
                for (int c = 0; c < 8; c++) v = fmaf(row[c], xf[m][c], v);
                f[m] = v;
            }
            Hs[ra] = quad_transpose_sum(f, nu);
#pragma unroll
            for (int m = 0; m < 4; m++) {
                const float xm = xo[m * 8 + ra];
#pragma unroll
                for (int c = 0; c < 8; c++) B[m][c] = fmaf(row[c], xm, B[m][c]);
            }
        });
        float* dst = nullptr;
        if (live) {
            if (nu == 3) dst = BT + (size_t)((cur ^ 1) * kLcSites + s) * kLcBT;
            else if (tgt_local >= 0) dst = BS + tgt_local * kLcBS + nu * 32;
        }
        if (dst) {
#pragma unroll
            for (int m = 0; m < 4; m++) {
                float4* q = reinterpret_cast<float4*>(dst + m * 8);
                q[0] = make_float4(B[m][0], B[m][1], B[m][2], B[m][3]);
                q[1] = make_float4(B[m][4], B[m][5], B[m][6], B[m][7]);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        // ---- epilogue for component mu = nu; the next slice's links (and X(x, t+2) for nu = t) are loaded first
        const int x = xyz + t * slice;
        float qo[8];
        if (MODE == 1 && k > 0 && live) load8(Y + (size_t)x * 32 + nu * 8, qo);
        if (t + 1 < t1) {
            u = LinkLoad<float, LF>::load(U, xyz + (t + 1) * slice, nu);
            if (has_halo) uh = LinkLoad<float, LF>::load(U, h_xyz + (t + 1) * slice, h_d);
            if (nu == 3) {
                const int tn = t + 2 >= Lt ? t + 2 - Lt : t + 2;
#pragma unroll
                for (int m = 0; m < 4; m++) load8(X + ((size_t)xyz + (size_t)tn * slice) * 32 + m * 8, xf[m]);
            }
        }
        if (live) {
            const int m = nu;
            const float* bt = BT + (size_t)(cur * kLcSites + s) * kLcBT + m * 8;
            const float* b0 = BS + s * kLcBS + m * 8;
            const float* xs = XC + s * kLcRow + m * 8;
            float y[8];
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const float h = Hs[c] + (((b0[c] + b0[32 + c]) + b0[64 + c]) + bt[c]);
                y[c] = fmaf(b, h, a * xs[c]);
            }
            if (MODE == 1) {
                if (k > 0)
#pragma unroll
                    for (int c = 0; c < 8; c++) y[c] = fmaf(beta, qo[c], y[c]);
#pragma unroll
                for (int c = 0; c < 8; c++) dot = fmaf(xs[c], y[c], dot);
            }
            store8(Y + (size_t)x * 32 + m * 8, y);
        }
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
