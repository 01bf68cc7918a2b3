// Shared runtime pieces of the library: context, status handling, lattice geometry, link views,
// deterministic float64 reductions and the workspace pool.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "../../include/rmhmc.h"
#include "su3.cuh"

namespace rm {

constexpr int kBlock = 128;           // threads per block of the site kernels
constexpr int kBlockMin = 64;         // smallest block of a tuned stencil launch
constexpr int kBlockMax = 256;        // largest block of a tuned stencil launch
constexpr int kRedSlots = 256;        // reduction slots per context (one per concurrent sum)

// ------------------------------------------------------------------------------------------------
// lattice geometry
// ------------------------------------------------------------------------------------------------
struct Geom {
    int L[4];
    int stride[4];
    int V;
    // division by L[d] as a multiply-high and shift (Granlund-Montgomery round-up method, exact for
    // numerators below 2^31 and therefore for every site index): q = (umulhi(mag, n) + n) >> shr
    unsigned mag[4];
    int shr[4];
};

__host__ inline void geom_init_divmod(Geom& g) {
    for (int d = 0; d < 4; d++) {
        int l = 0;
        while ((1u << l) < (unsigned)g.L[d]) l++;
        const unsigned long long m = ((1ull << 32) * ((1ull << l) - (unsigned long long)g.L[d])) / (unsigned long long)g.L[d] + 1ull;
        g.mag[d] = (unsigned)(m & 0xffffffffull);
        g.shr[d] = l;
    }
}

__device__ __forceinline__ int fast_div(const Geom& g, int n, int d) {
    return (int)((__umulhi(g.mag[d], (unsigned)n) + (unsigned)n) >> g.shr[d]);
}

__device__ __forceinline__ void neighbours(const Geom& g, int s, int fwd[4], int bwd[4]) {
    int r = s;
#pragma unroll
    for (int d = 0; d < 4; d++) {
        const int q = fast_div(g, r, d);
        const int c = r - q * g.L[d];
        r = q;
        fwd[d] = (c == g.L[d] - 1) ? s - c * g.stride[d] : s + g.stride[d];
        bwd[d] = (c == 0) ? s + (g.L[d] - 1) * g.stride[d] : s - g.stride[d];
    }
}

__device__ __forceinline__ void site_coords(const Geom& g, int s, int c[4]) {
#pragma unroll
    for (int d = 0; d < 4; d++) {
        const int q = fast_div(g, s, d);
        c[d] = s - q * g.L[d];
        s = q;
    }
}

// neighbour of site s one step (n = +1 or -1) along direction d, periodic
__device__ __forceinline__ int step_site(const Geom& g, int s, int d, int n) {
    int r = s, c = 0;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const int q = fast_div(g, r, e);
        if (e == d) c = r - q * g.L[e];
        r = q;
    }
    if (n > 0) return c == g.L[d] - 1 ? s - c * g.stride[d] : s + g.stride[d];
    return c == 0 ? s + (g.L[d] - 1) * g.stride[d] : s - g.stride[d];
}

// site reached from coordinates c by n steps along direction d (periodic), without changing c
__device__ __forceinline__ int shifted(const Geom& g, const int c[4], int d, int n) {
    int s = 0;
#pragma unroll
    for (int e = 3; e >= 0; e--) {
        int ce = c[e];
        if (e == d) { ce = (ce + n) % g.L[e]; if (ce < 0) ce += g.L[e]; }
        s = s * g.L[e] + ce;
    }
    return s;
}

// ------------------------------------------------------------------------------------------------
// internal link layouts
//   FP64: u64[(mu*9 + 3i + j) * V + s]            double2 (re, im)
//   FP32: u32a[(mu*3 + r) * V + s]  float4, r=0: (u00,u01) r=1: (u02,u10) r=2: (u11,u12)
//         u32b[(mu*3 + j) * V + s]  float2, u2j (third row; unused by the 12-real format)
// ------------------------------------------------------------------------------------------------
struct Links64 { const double2* u; int V; };
struct Links32 { const float4* a; const float2* b; int V; };

template <typename T, int LF> struct LinkLoad;

template <int LF> struct LinkLoad<double, LF> {
    __device__ __forceinline__ static mat3<double> load(const Links64& U, int s, int mu) {
        mat3<double> m;
        const int rows = LF == 12 ? 2 : 3;
#pragma unroll
        for (int i = 0; i < rows; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const double2 v = __ldg(&U.u[(size_t)(mu * 9 + 3 * i + j) * U.V + s]);
                m.e[i][j] = cmk(v.x, v.y);
            }
        if (LF == 12) {
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
                cplx<double> c = csub(cmul(m.e[0][j1], m.e[1][j2]), cmul(m.e[0][j2], m.e[1][j1]));
                m.e[2][j] = cconj(c);
            }
        }
        return m;
    }
};

template <int LF> struct LinkLoad<float, LF> {
    __device__ __forceinline__ static mat3<float> load(const Links32& U, int s, int mu) {
        mat3<float> m;
        const float4 r0 = __ldg(&U.a[(size_t)(mu * 3 + 0) * U.V + s]);
        const float4 r1 = __ldg(&U.a[(size_t)(mu * 3 + 1) * U.V + s]);
        const float4 r2 = __ldg(&U.a[(size_t)(mu * 3 + 2) * U.V + s]);
        m.e[0][0] = cmk(r0.x, r0.y); m.e[0][1] = cmk(r0.z, r0.w);
        m.e[0][2] = cmk(r1.x, r1.y); m.e[1][0] = cmk(r1.z, r1.w);
        m.e[1][1] = cmk(r2.x, r2.y); m.e[1][2] = cmk(r2.z, r2.w);
        if (LF == 12) {
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
                cplx<float> c = csub(cmul(m.e[0][j1], m.e[1][j2]), cmul(m.e[0][j2], m.e[1][j1]));
                m.e[2][j] = cconj(c);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const float2 v = __ldg(&U.b[(size_t)(mu * 3 + j) * U.V + s]);
                m.e[2][j] = cmk(v.x, v.y);
            }
        }
        return m;
    }
};

// ------------------------------------------------------------------------------------------------
// field component access: AoS [V][4][8]
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void load8(const double* p, double* x) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < 4; i++) { double2 v = __ldg(q + i); x[2 * i] = v.x; x[2 * i + 1] = v.y; }
}
__device__ __forceinline__ void load8(const float* p, float* x) {
    const float4* q = reinterpret_cast<const float4*>(p);
    float4 a = __ldg(q), b = __ldg(q + 1);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}
// eight floats with one 256-bit read-only global load (sm_100 and later).  p must be 32-byte aligned (callers
// check it, or pass the context's own buffers) and no thread may write the data during the kernel before
// this read.
__device__ __forceinline__ void load8_v8(const float* p, float* x) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]), "=f"(x[4]), "=f"(x[5]), "=f"(x[6]), "=f"(x[7])
        : "l"(p));
}
__device__ __forceinline__ void store8(double* p, const double* x) {
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int i = 0; i < 4; i++) q[i] = make_double2(x[2 * i], x[2 * i + 1]);
}
__device__ __forceinline__ void store8(float* p, const float* x) {
    float4* q = reinterpret_cast<float4*>(p);
    q[0] = make_float4(x[0], x[1], x[2], x[3]);
    q[1] = make_float4(x[4], x[5], x[6], x[7]);
}

// ------------------------------------------------------------------------------------------------
// deterministic reductions: every block writes its partial sums to a slot array; the last block
// to finish (ticket counter) adds them in block order in float64 and writes the result.
// ------------------------------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* sh /* N * (kBlock/32) */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int n = 0; n < N; n++) {
        double x = v[n];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[n * (blockDim.x >> 5) + warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int n = 0; n < N; n++) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[n * (blockDim.x >> 5) + w];
            v[n] = s;
        }
    }
}

// float partials summed within a warp in float, then across warps and blocks in double
template <int N>
__device__ __forceinline__ void block_sum_f(float (&v)[N], double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int n = 0; n < N; n++) {
        float x = v[n];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[n * (blockDim.x >> 5) + warp] = (double)x;
    }
    __syncthreads();
}

// Called by EVERY thread of every block; v[] holds the block's N sums in thread 0.  partials:
// [nblocks][N] for this reduction, counter: its ticket.  The last block to arrive adds all partials:
// thread t takes blocks t, t + blockDim, ... in that order, then a fixed shuffle/shared-memory tree, so
// the result does not depend on scheduling.  Returns true in thread 0 of the last block, with out[0..N-1]
// written; sh needs N * (blockDim / 32) doubles.
template <int N>
__device__ __forceinline__ bool grid_sum_finish(const double* v, double* partials, unsigned* counter, double* out,
                                                int nblocks, int bid, double* sh) {
    __shared__ int am_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int n = 0; n < N; n++) partials[(size_t)bid * N + n] = v[n];
        __threadfence();
        const unsigned ticket = atomicAdd(counter, 1u);
        am_last = ticket == (unsigned)(nblocks - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double t[N];
#pragma unroll
    for (int n = 0; n < N; n++) t[n] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int n = 0; n < N; n++) t[n] += __ldcg(partials + (size_t)b * N + n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int n = 0; n < N; n++) {
        double x = t[n];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[n * nw + warp] = x;
    }
    __syncthreads();
    if (threadIdx.x != 0) return false;
#pragma unroll
    for (int n = 0; n < N; n++) {
        double x = 0.0;
        for (int w = 0; w < nw; w++) x += sh[n * nw + w];
        out[n] = x;
    }
    *counter = 0u;
    return true;
}

// ------------------------------------------------------------------------------------------------
// buffer of device memory owned by the context
// ------------------------------------------------------------------------------------------------
struct DevBuf { void* p = nullptr; size_t bytes = 0; };

}  // namespace rm

// ------------------------------------------------------------------------------------------------
// the context
// ------------------------------------------------------------------------------------------------
struct rmhmc_ctx {
    int device = 0;
    rm::Geom g{};
    std::string err;
    // links
    double2* u64 = nullptr;
    float4* u32a = nullptr;
    float2* u32b = nullptr;
    bool links_valid = false;
    unsigned long long link_gen = 1;   // bumped whenever the internal link copies change
    unsigned long long adj_gen = 0;    // link_gen the adjoint table was built for
    // reductions
    double* red_partials = nullptr;   // [kRedSlots][max_blocks * 2]
    unsigned* red_counters = nullptr; // [kRedSlots]
    double* red_out = nullptr;        // [kRedSlots][8]
    int max_blocks = 0;
    double* h_pinned = nullptr;       // pinned host staging (kPinned doubles)
    // workspace pool
    std::map<std::string, rm::DevBuf> bufs;
    size_t num_sms = 0;
    // pinned upload ring (kRingSlots slots of kRingBytes) and the events that guard slot reuse
    char* ring = nullptr;
    cudaEvent_t ring_ev[4] = {};
    unsigned ring_idx = 0;
    // events of the look-behind convergence check of the Krylov loop, and the iteration count of the
    // last run per (precision, shift, tolerance, cap)
    cudaEvent_t kr_ev[2] = {};
    std::map<std::string, int> kr_pred;
    // CUDA graph of the molecular dynamics: executable, the parameters and workspace generation it was
    // captured for, capture streams, and whether graphs are used (fallback reason when not)
    cudaGraphExec_t md_exec = nullptr;
    std::string md_key;
    unsigned long long md_gen = 0;
    unsigned long long ws_gen = 0;      // bumped whenever a workspace buffer is (re)allocated
    cudaStream_t cap_st[3] = {};
    bool use_graphs = true;
    std::string graph_note;
    // autotuned stencil shapes per (precision bytes * 100 + link format): components per lane, block size
    std::map<int, std::pair<int, int>> tune;
    // kernel of the kinetic-force contraction (rmhmc_set_stencil_shape, RMHMC_SHAPE_KFORCE): 0 four lanes per link,
    // own basis rows from global memory (the fastest at 32^4: 9.9 ms per kinetic evaluation against 11.2 and
    // 11.5 ms); 1 the same with the rows staged in shared memory; 2 eight lanes per link
    int lg_mode = 0;
    // float64 link update in float-float arithmetic (rmhmc_set_stencil_shape, RMHMC_SHAPE_LINKUPDATE)
    bool link_update_ff = true;
    // z-extent of the multi-field adjoint kernel's slabs (rmhmc_set_stencil_shape, RMHMC_SHAPE_ADJOINT); 0 chosen
    // from the lattice and the field count
    int ad_slab = 0;
    // incremented by every rmhmc_set_stencil_shape: part of the key of a captured trajectory graph
    int shape_gen = 0;
    std::string tune_report;
    // counters: kernels launched; optional timing of the conjugate-gradient stencil launches
    long long launches = 0;
    long long krylov_iters = 0;
    bool prof = false;
    long long prof_count = 0;
    double prof_ms = 0.0;
    cudaEvent_t* prof_ev = nullptr;   // 2 * kProfEvents events, created when profiling is switched on
};

namespace rm {

constexpr int kPinned = 1 << 16;
constexpr int kRingSlots = 4;
constexpr int kProfEvents = 256;
constexpr size_t kRingBytes = 1 << 20;
// copy host bytes to device memory asynchronously through the pinned ring
int upload(rmhmc_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st);

int set_err(rmhmc_ctx* ctx, int code, const char* fmt, ...);
int cuda_check(rmhmc_ctx* ctx, cudaError_t e, const char* what);
void* workspace(rmhmc_ctx* ctx, const char* name, size_t bytes, int* status);
int import_links(rmhmc_ctx* ctx, const double* U, cudaStream_t st);
int ensure_links(rmhmc_ctx* ctx, const double* U, cudaStream_t st);
inline size_t field_elems(const rmhmc_ctx* ctx) { return (size_t)ctx->g.V * 32; }
inline int site_blocks(const rmhmc_ctx* ctx) { return (ctx->g.V + kBlock - 1) / kBlock; }
// blocks of the stencil kernels: four lanes per site (one per field component mu)
inline int lane_blocks(const rmhmc_ctx* ctx) { return (int)(((size_t)ctx->g.V * 4 + kBlock - 1) / kBlock); }
// grids of the reduced kernels hold at most one full wave (2048 threads per SM) and stride over the rest:
// the deterministic final sum then has at most 16 * SMs block partials.  Above one wave the grid is trimmed
// so that every thread strides the same number of times (no tail pass with a partly idle grid, whose blocks
// would wait at the final reduction)
inline int capped_grid(const rmhmc_ctx* ctx, size_t threads, int block) {
    const size_t need = (threads + block - 1) / block;
    const size_t cap = (size_t)ctx->num_sms * (2048 / block);
    if (need <= cap) return (int)std::max<size_t>(1, need);
    const size_t passes = (need + cap - 1) / cap;
    const size_t sms = std::max<size_t>(1, ctx->num_sms);
    const size_t g = (need + passes - 1) / passes;
    return (int)std::min(cap, (g + sms - 1) / sms * sms);   // whole blocks per SM
}
inline Links64 links64(const rmhmc_ctx* ctx) { return Links64{ctx->u64, ctx->g.V}; }
inline Links32 links32(const rmhmc_ctx* ctx) { return Links32{ctx->u32a, ctx->u32b, ctx->g.V}; }
double* red_slot_partials(rmhmc_ctx* ctx, int slot);
unsigned* red_slot_counter(rmhmc_ctx* ctx, int slot);
double* red_slot_out(rmhmc_ctx* ctx, int slot);
// copy n doubles from device to host through pinned memory and synchronise the stream
int fetch(rmhmc_ctx* ctx, const double* dsrc, double* hdst, int n, cudaStream_t st);

}  // namespace rm

#define RM_CHECK(ctx, call)                                                  \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return rm::cuda_check((ctx), e_, #call);      \
    } while (0)
#define RM_LAUNCH_CHECK(ctx) RM_CHECK(ctx, cudaGetLastError())
#define RM_TRY(x)                     \
    do {                              \
        int s_ = (x);                 \
        if (s_ != RMHMC_OK) return s_; \
    } while (0)
