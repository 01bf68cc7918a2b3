// Gauge action (Sec. 2: Wilson plaquettes plus weighted 1x2 rectangles) and average plaquette without
// any allocation: a variant of the action reduction of gauge.cu for callers that may not allocate
// device memory.
//
// Who needs this: a caller whose device memory is entirely handed out by another allocator (a framework's
// caching pool that reserved the whole GPU up front), so that a context's workspace cannot be created, or
// a caller on a latency-critical path that must not call cudaMalloc/cudaFree because they synchronise the
// device.  Such a caller passes the links and a two-double output buffer it already owns; the only scratch
// is the file-scope device array below.
//
// The scratch holds kNoAllocBlocks block partials and a ticket counter.  It is shared by every call in
// the process and keeps the previous call's contents: each call zeroes the counter before its kernel,
// and two calls that overlap on the GPU (different streams, no ordering) race on it and must not be
// issued.  Each GPU that loads the library keeps this ~64 KB array until the process exits.  The device
// address of the array is looked up once per device (cudaGetSymbolAddress) by the first call made with
// that device current; make that first call before any stream capture.
#include <mutex>

#include "common.cuh"

namespace rm {

constexpr int kNoAllocBlocks = 4096;     // fixed grid: blocks stride over the lattice
constexpr int kNoAllocThreads = 128;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocBlocks * 2 + 32];

// links in the canonical layout [V][4][3][3] complex128
struct CanonLinks {
    const double* U;
    __device__ __forceinline__ mat3<double> operator()(int s, int mu) const {
        mat3<double> m;
        const double2* p = reinterpret_cast<const double2*>(U + ((size_t)s * 4 + mu) * 18);
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const double2 z = p[3 * i + j];
                m.e[i][j] = cmk(z.x, z.y);
            }
        return m;
    }
};

__device__ __forceinline__ int na_site(const Geom& g, const int c[4], int d1, int n1, int d2, int n2) {
    int s = 0;
#pragma unroll
    for (int e = 3; e >= 0; e--) {
        int v = c[e] + (e == d1 ? n1 : 0) + (e == d2 ? n2 : 0);
        if (v >= g.L[e]) v -= g.L[e];
        if (v >= g.L[e]) v -= g.L[e];
        if (v < 0) v += g.L[e];
        s = s * g.L[e] + v;
    }
    return s;
}

// S = beta sum_x [c0 sum_{mu<nu} (1 - ReTr P/3) + c1 sum_{mu!=nu} (1 - ReTr R/3)] and the plaquette sum;
// partials and the ticket counter live in the caller-supplied scratch
__global__ void __launch_bounds__(kNoAllocThreads) k_action_noalloc(Geom g, CanonLinks U, double beta, double c0,
                                                                     double c1, double* scratch, double* out) {
    __shared__ double sh[2 * (kNoAllocThreads / 32)];
    double act = 0.0, plaq = 0.0;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.V; x += gridDim.x * blockDim.x) {
        int c[4];
        site_coords(g, x, c);
        double ax = 0.0;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = 0; nu < 4; nu++) {
                if (mu == nu) continue;
                const int xpm = na_site(g, c, mu, 1, nu, 0);
                const int xpn = na_site(g, c, nu, 1, mu, 0);
                if (mu < nu) {
                    mat3<double> p = m_mul(U(x, mu), U(xpm, nu));
                    p = m_mul_nd(p, U(xpn, mu));
                    const double rt = re_trace(m_mul_nd(p, U(x, nu))) / 3.0;
                    plaq += rt;
                    ax += c0 * (1.0 - rt);
                }
                if (c1 != 0.0) {
                    const int x2m = na_site(g, c, mu, 2, nu, 0);
                    const int xpmpn = na_site(g, c, mu, 1, nu, 1);
                    mat3<double> r = m_mul(U(x, mu), U(xpm, mu));
                    r = m_mul(r, U(x2m, nu));
                    r = m_mul_nd(r, U(xpmpn, mu));
                    r = m_mul_nd(r, U(xpn, mu));
                    ax += c1 * (1.0 - re_trace(m_mul_nd(r, U(x, nu))) / 3.0);
                }
            }
        act += beta * ax;
    }
    double v[2] = {act, plaq};
    block_sum<2>(v, sh);
    unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNoAllocBlocks * 2);
    double res[2];
    if (grid_sum_finish<2>(v, scratch, counter, res, gridDim.x, blockIdx.x, sh)) {
        out[0] = res[0];
        out[1] = res[1] / (6.0 * g.V);
    }
}

static std::mutex g_noalloc_mutex;
static double* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// device address of the scratch array on the current device (looked up once per device)
static int noalloc_scratch(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RMHMC_ECUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return RMHMC_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return RMHMC_ECUDA;
        g_noalloc_ptr[dev] = (double*)p;
    }
    *out = g_noalloc_ptr[dev];
    return RMHMC_OK;
}

}  // namespace rm

using namespace rm;

extern "C" int rmhmc_action_noalloc(const int dims[4], const double* U, double beta, double c1, double* out,
                                    cudaStream_t stream) {
    if (!dims || !U || !out) return RMHMC_EINVAL;
    // the largest lattice: 2^26 sites; each partial product is checked, so no extent overflows it
    long long V = 1;
    for (int d = 0; d < 4; d++) {
        if (dims[d] < 2 || dims[d] > (1 << 26)) return RMHMC_EINVAL;
        V *= dims[d];
        if (V > (1ll << 26)) return RMHMC_EINVAL;
    }
    if ((uintptr_t)U % 16) return RMHMC_EINVAL;
    Geom g{};
    for (int d = 0; d < 4; d++) g.L[d] = dims[d];
    g.stride[0] = 1;
    for (int d = 1; d < 4; d++) g.stride[d] = g.stride[d - 1] * dims[d - 1];
    g.V = (int)V;
    geom_init_divmod(g);
    double* scratch = nullptr;
    const int st = noalloc_scratch(&scratch);
    if (st != RMHMC_OK) return st;
    // the ticket counter must start at zero whatever the previous call left
    if (cudaMemsetAsync(scratch + kNoAllocBlocks * 2, 0, sizeof(unsigned), stream) != cudaSuccess) return RMHMC_ECUDA;
    const int blocks = (int)std::min<long long>(kNoAllocBlocks, (V + kNoAllocThreads - 1) / kNoAllocThreads);
    k_action_noalloc<<<blocks, kNoAllocThreads, 0, stream>>>(g, CanonLinks{U}, beta, 1.0 - 8.0 * c1, c1, scratch, out);
    if (cudaGetLastError() != cudaSuccess) return RMHMC_ECUDA;
    return RMHMC_OK;
}
