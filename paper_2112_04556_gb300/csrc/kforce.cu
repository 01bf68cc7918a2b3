// Kinetic (mass-term) force, Sec. 3 (the force F_M below Eq. 5), and the link-adjoint of the
// Laplacian stencil it is built from.
//
// With T = 1/2 |R(A) P|^2, R(lam) = c + sum_j alpha_j/(lam + sigma_j):
//   dT = -sum_j alpha_j <Z_j, (dA) X_j>,  X_j = (A+sigma_j)^{-1} P,  Z_j = (A+sigma_j)^{-1} R(A) P,
// so F_K = -dT/dw = sum_j alpha_j <Z_j, (dA/dw) X_j>.  Only two hops of A contain U = U_nu(y): the
// forward hop at y and the backward hop at y+nu.  With W1 = U X(y+nu) U^dag, W2 = U Z(y+nu) U^dag,
//   d<Z, A X>/dw^a = -(1/16) 2i sum_mu Tr(T^a D),   D = [W1, Z(y)] - [X(y), W2] = M - M^dag,
//   M = W1 Z(y) - X(y) W2,
// and with K = -i D:  d<Z, A X>/dw^a = (1/16) sum_mu Tr(lambda^a K) = (1/8) sum_mu coef_a(M)
// where coef_a(M) = Tr(lambda^a (-i)(M - M^dag)/2) (antiherm_coef).
#include <algorithm>

#include "krylov.cuh"
#include "ops.cuh"
#include "stencil.cuh"

namespace rm {

constexpr int kMaxPairs = 24;
struct PairWeights { double w[kMaxPairs]; };

// one lane per (site y, link direction nu, field component mu); the four component lanes of a link are
// adjacent and their partial derivatives are summed with two butterfly shuffles
template <typename T, int LF>
__global__ void __launch_bounds__(kBlock) k_link_grad(Geom g, typename LinksOf<T>::type U, const T* __restrict__ X,
                                                       const T* __restrict__ Z, size_t fs, int nf, PairWeights w,
                                                       double* __restrict__ G) {
    const int lane = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = lane >> 2, mu = lane & 3;
    const int nu = blockIdx.y;
    const bool live = y < g.V;
    T k[8];
#pragma unroll
    for (int a = 0; a < 8; a++) k[a] = T(0);
    if (live) {
        int fwd[4], bwd[4];
        neighbours(g, y, fwd, bwd);
        const int yp = fwd[nu];
        const mat3<T> u = LinkLoad<T, LF>::load(U, y, nu);
        for (int f = 0; f < nf; f++) {
            const T wf = (T)w.w[f];
            const T* Xf = X + f * fs;
            const T* Zf = Z + f * fs;
            T xb[8];
            load8(Xf + (size_t)yp * 32 + mu * 8, xb);
            herm<T> W1 = h_zero<T>();
            acc_uxud(W1, u, coef_to_herm2(xb));          // 2 W1
            load8(Zf + (size_t)yp * 32 + mu * 8, xb);
            herm<T> W2 = h_zero<T>();
            acc_uxud(W2, u, coef_to_herm2(xb));          // 2 W2
            load8(Zf + (size_t)y * 32 + mu * 8, xb);
            const mat3<T> Zy = herm_full(coef_to_herm2(xb));   // 2 Z(y)
            load8(Xf + (size_t)y * 32 + mu * 8, xb);
            const mat3<T> Xy = herm_full(coef_to_herm2(xb));   // 2 X(y)
            mat3<T> M = m_mul(herm_full(W1), Zy);              // 4 W1 Z
            const mat3<T> M2 = m_mul(Xy, herm_full(W2));       // 4 X W2
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) M.e[i][j] = csub(M.e[i][j], M2.e[i][j]);
            T kk[8];
            antiherm_coef(M, kk);                               // 4 coef(M)
#pragma unroll
            for (int a = 0; a < 8; a++) k[a] = fma(wf, kk[a], k[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 8; a++) {
        k[a] += __shfl_xor_sync(0xffffffffu, k[a], 1);
        k[a] += __shfl_xor_sync(0xffffffffu, k[a], 2);
    }
    if (live && mu == 0) {
        double* out = G + (size_t)y * 32 + nu * 8;
        // d<Z,AX>/dw = (1/8) coef(M) and the doubled expansions gave 4 coef(M): scale by 1/32
#pragma unroll
        for (int a = 0; a < 8; a++) out[a] = (double)k[a] * (1.0 / 32.0);
    }
}

int link_grad_launch(rmhmc_ctx* ctx, int prec, const void* X, const void* Z, int nf, const double* w, double* G,
                     cudaStream_t st) {
    if (nf > kMaxPairs) return set_err(ctx, RMHMC_EINVAL, "at most %d field pairs", kMaxPairs);
    PairWeights pw{};
    for (int f = 0; f < nf; f++) pw.w[f] = w[f];
    const dim3 grid(lane_blocks(ctx), 4);
    if (prec == RMHMC_FP64)
        k_link_grad<double, 18><<<grid, kBlock, 0, st>>>(ctx->g, links64(ctx), (const double*)X, (const double*)Z,
                                                         field_elems(ctx), nf, pw, G);
    else
        k_link_grad<float, 18><<<grid, kBlock, 0, st>>>(ctx->g, links32(ctx), (const float*)X, (const float*)Z,
                                                        field_elems(ctx), nf, pw, G);
    ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}

// ------------------------------------------------------------------------------------------------
// Kinetic force straight from the Krylov basis.  With X_j = sum_k cx_jk r_k and Z_j = sum_k cz_jk r_k on the
// stored residuals r_k, the force on U = U_nu(y) is, in the adjoint representation R = Ad(U)
// (U T^b U^dag = sum_c R_cb T^c) and with the su(3) structure constants f,
//   G^a = (1/16) sum_cd f_acd (R C)_cd,   C = sum_mu sum_kl S_kl r_k,mu(y+nu) r_l,mu(y)^T,
//   S_kl = sum_j alpha_j (cx_jk cz_jl + cz_jk cx_jl),
// because coef_a(W Z - X W') = (1/2) f_acd [R (x' z^T + z' x^T)]_cd for W = U X' U^dag, W' = U Z' U^dag
// (x, z, x', z' the coefficient vectors of X(y), Z(y), X(y+nu), Z(y+nu)).  One pass over the n basis
// vectors replaces forming the 2 npole fields X_j, Z_j and the per-pole conjugations: per site about
// 8 n^2 + 256 n + 1400 FMA per link against 576 npole per link for the direct form.
// ------------------------------------------------------------------------------------------------

// G_a += sum_c f_acd rc_c for one column d (d a compile-time constant after unrolling)
template <typename T>
__device__ __forceinline__ void f_contract(int d, const T (&rc)[8], T (&G)[8]) {
    constexpr int tr[9][3] = {{0, 1, 2}, {0, 3, 6}, {0, 4, 5}, {1, 3, 5}, {1, 4, 6},
                              {2, 3, 4}, {2, 5, 6}, {3, 4, 7}, {5, 6, 7}};
    constexpr double fv[9] = {1.0, 0.5, -0.5, 0.5, 0.5, 0.5, -0.5, 0.86602540378443864676, 0.86602540378443864676};
#pragma unroll
    for (int t = 0; t < 9; t++) {
        const int i = tr[t][0], j = tr[t][1], k = tr[t][2];
        const T v = (T)fv[t];
        if (d == k) { G[i] = fma(v, rc[j], G[i]); G[j] = fma(-v, rc[i], G[j]); }
        else if (d == j) { G[k] = fma(v, rc[i], G[k]); G[i] = fma(-v, rc[k], G[i]); }
        else if (d == i) { G[j] = fma(v, rc[k], G[j]); G[k] = fma(-v, rc[j], G[k]); }
    }
}

// eight values from shared memory (plain loads: the read-only global path does not apply to shared memory)
__device__ __forceinline__ void lds8(const float* p, float* x) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}
__device__ __forceinline__ void lds8(const double* p, double* x) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const double2 v = reinterpret_cast<const double2*>(p)[i];
        x[2 * i] = v.x; x[2 * i + 1] = v.y;
    }
}

constexpr int kLgSites = 32;   // sites per block (4 lanes each)
constexpr int kLgKC = 4;       // basis vectors per chunk of W
constexpr int kLgPad = kLgKC * 32 + 4;

// S_kl (row stride ld) from the basis rows of X_j (rows j) and Z_j (rows ns + j), row stride ldr;
// n from flags[1] when flags is given
__global__ void __launch_bounds__(256) k_pair_matrix(const double* __restrict__ rows, int ldr, int ns, PairWeights w,
                                                     const int* __restrict__ flags, int n, double* __restrict__ S, int ld) {
    if (flags) n = flags[1];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x) {
        const int k = idx / n, l = idx % n;
        double s = 0.0;
        for (int j = 0; j < ns; j++) {
            const double* X = rows + (size_t)j * ldr;
            const double* Z = rows + (size_t)(ns + j) * ldr;
            s = fma(w.w[j], fma(X[k], Z[l], Z[k] * X[l]), s);
        }
        S[(size_t)k * ld + l] = s;
    }
}

// one block: kLgSites sites x 4 lanes.  Per chunk of kLgKC basis vectors: lane (y, mu) forms
// W_k,mu(y) = sum_l S_kl r_l,mu(y) into shared memory; then lane (y, nu) accumulates
// C += sum_mu r_k,mu(y+nu) W_k,mu(y)^T.  Finally lane (y, nu) conjugates the columns of C by U_nu(y) and
// contracts with f.  n from flags[1] when flags is given.
template <typename T, int LF>
__global__ void __launch_bounds__(kLgSites * 4, 4) k_link_grad_krylov(Geom g, typename LinksOf<T>::type U, const T* __restrict__ R,
                                                                   size_t fs, const int* __restrict__ flags, int n,
                                                                   const double* __restrict__ S, int ld, double* __restrict__ G) {
    __shared__ __align__(16) T Ws[kLgSites * kLgPad];
    __shared__ T Ss[kLgKC * kBasisCap];
    if (flags) n = flags[1];
    const int sl = threadIdx.x >> 2, q = threadIdx.x & 3;
    T* const wrow = Ws + sl * kLgPad;
    for (int base = blockIdx.x * kLgSites; base < g.V; base += gridDim.x * kLgSites) {
        const int y = base + sl;
        const bool live = y < g.V;
        int yn = 0;
        if (live) {
            int fwd[4], bwd[4];
            neighbours(g, y, fwd, bwd);
            yn = fwd[q];
        }
        T C[8][8];
#pragma unroll
        for (int b = 0; b < 8; b++)
#pragma unroll
            for (int d = 0; d < 8; d++) C[b][d] = T(0);
        for (int k0 = 0; k0 < n; k0 += kLgKC) {
            __syncthreads();
            for (int t = threadIdx.x; t < kLgKC * n; t += blockDim.x) {
                const int kk = t / n, l = t - kk * n;
                Ss[kk * kBasisCap + l] = k0 + kk < n ? (T)S[(size_t)(k0 + kk) * ld + l] : T(0);
            }
            __syncthreads();
            T w[kLgKC][8];
#pragma unroll
            for (int kk = 0; kk < kLgKC; kk++)
#pragma unroll
                for (int a = 0; a < 8; a++) w[kk][a] = T(0);
            if (live) {
                for (int l = 0; l < n; l++) {
                    T r[8];
                    load8_v8(R + (size_t)l * fs + (size_t)y * 32 + q * 8, r);
#pragma unroll
                    for (int kk = 0; kk < kLgKC; kk++) {
                        const T s = Ss[kk * kBasisCap + l];
#pragma unroll
                        for (int a = 0; a < 8; a++) w[kk][a] = fma(s, r[a], w[kk][a]);
                    }
                }
            }
#pragma unroll
            for (int kk = 0; kk < kLgKC; kk++) store8(wrow + kk * 32 + q * 8, w[kk]);
            __syncthreads();
            if (live) {
                const int kc = min(kLgKC, n - k0);
                for (int kk = 0; kk < kc; kk++) {
                    const T* rk = R + (size_t)(k0 + kk) * fs + (size_t)yn * 32;
#pragma unroll
                    for (int mu = 0; mu < 4; mu++) {
                        T rp[8], wv[8];
                        load8_v8(rk + mu * 8, rp);
                        lds8(wrow + kk * 32 + mu * 8, wv);
#pragma unroll
                        for (int b = 0; b < 8; b++)
#pragma unroll
                            for (int d = 0; d < 8; d++) C[b][d] = fma(rp[b], wv[d], C[b][d]);
                    }
                }
            }
        }
        if (live) {
            const mat3<T> u = LinkLoad<T, LF>::load(U, y, q);
            T Gk[8];
#pragma unroll
            for (int a = 0; a < 8; a++) Gk[a] = T(0);
#pragma unroll
            for (int d = 0; d < 8; d++) {
                T col[8], rc[8];
#pragma unroll
                for (int b = 0; b < 8; b++) col[b] = C[b][d];
                herm<T> E = h_zero<T>();
                acc_uxud_tl(E, u, coef_to_herm2(col));   // 2 sum_c (R C)_cd T^c
                herm2_to_coef_tl(E, rc);                  // (R C)_cd
                f_contract(d, rc, Gk);
            }
            double* out = G + (size_t)y * 32 + q * 8;
#pragma unroll
            for (int a = 0; a < 8; a++) out[a] = (double)Gk[a] * (1.0 / 16.0);
        }
    }
}

// The same contraction with the block's own basis rows staged once in shared memory (for n <= kLgStage):
// the kernel above reads r_l(y) for all l once per chunk of kLgKC basis vectors, i.e. n / kLgKC times from
// L2; here the 32 sites' n rows are copied in once (coalesced 16-byte loads, site records padded to 36
// floats so that a warp's 128-bit reads fall on distinct bank quads) and every chunk reads them from shared
// memory.  In the C phase the next neighbour row is loaded before the arithmetic of the current one.
// Longer runs (n > kLgStage, read on the device) take the global reads of the kernel above.
constexpr int kLgStage = 20;
constexpr int kLgRow = 36;   // floats per staged site row (32 + 4)

inline size_t lg_staged_smem() {
    return sizeof(float) * ((size_t)kLgStage * kLgSites * kLgRow + kLgSites * kLgPad + kLgKC * kBasisCap);
}

template <int LF>
__global__ void __launch_bounds__(kLgSites * 4, 2) k_link_grad_staged(Geom g, Links32 U, const float* __restrict__ R,
                                                                      size_t fs, const int* __restrict__ flags, int n,
                                                                      const double* __restrict__ S, int ld,
                                                                      double* __restrict__ G) {
    extern __shared__ __align__(16) float lgs[];
    float* Rs = lgs;                                          // [kLgStage][kLgSites][kLgRow]
    float* Ws = Rs + (size_t)kLgStage * kLgSites * kLgRow;    // [kLgSites][kLgPad]
    float* Ss = Ws + kLgSites * kLgPad;                       // [kLgKC][kBasisCap]
    if (flags) n = flags[1];
    const bool staged = n <= kLgStage;
    const int sl = threadIdx.x >> 2, q = threadIdx.x & 3;
    float* const wrow = Ws + sl * kLgPad;
    for (int base = blockIdx.x * kLgSites; base < g.V; base += gridDim.x * kLgSites) {
        const int y = base + sl;
        const bool live = y < g.V;
        const int yn = live ? step_site(g, y, q, 1) : 0;
        if (staged) {
            __syncthreads();   // the previous tile's reads of Rs are done
            const int nsite = min(kLgSites, g.V - base);
            for (int idx = threadIdx.x; idx < n * kLgSites * 8; idx += blockDim.x) {
                const int l = idx / (kLgSites * 8), rem = idx - l * (kLgSites * 8);
                const int ss = rem >> 3, c4 = rem & 7;
                if (ss < nsite) {
                    const float4 v = __ldg(reinterpret_cast<const float4*>(R + (size_t)l * fs + (size_t)(base + ss) * 32) + c4);
                    *reinterpret_cast<float4*>(Rs + ((size_t)l * kLgSites + ss) * kLgRow + c4 * 4) = v;
                }
            }
        }
        float C[8][8];
#pragma unroll
        for (int b = 0; b < 8; b++)
#pragma unroll
            for (int d = 0; d < 8; d++) C[b][d] = 0.f;
        for (int k0 = 0; k0 < n; k0 += kLgKC) {
            __syncthreads();
            for (int t = threadIdx.x; t < kLgKC * n; t += blockDim.x) {
                const int kk = t / n, l = t - kk * n;
                Ss[kk * kBasisCap + l] = k0 + kk < n ? (float)S[(size_t)(k0 + kk) * ld + l] : 0.f;
            }
            __syncthreads();
            float w[kLgKC][8];
#pragma unroll
            for (int kk = 0; kk < kLgKC; kk++)
#pragma unroll
                for (int a = 0; a < 8; a++) w[kk][a] = 0.f;
            if (live) {
                for (int l = 0; l < n; l++) {
                    float r[8];
                    if (staged) lds8(Rs + ((size_t)l * kLgSites + sl) * kLgRow + q * 8, r);
                    else load8_v8(R + (size_t)l * fs + (size_t)y * 32 + q * 8, r);
#pragma unroll
                    for (int kk = 0; kk < kLgKC; kk++) {
                        const float sv = Ss[kk * kBasisCap + l];
#pragma unroll
                        for (int a = 0; a < 8; a++) w[kk][a] = fmaf(sv, r[a], w[kk][a]);
                    }
                }
            }
#pragma unroll
            for (int kk = 0; kk < kLgKC; kk++) store8(wrow + kk * 32 + q * 8, w[kk]);
            __syncthreads();
            if (live) {
                const int kc = min(kLgKC, n - k0);
                // neighbour rows of the chunk, one (k, mu) ahead: iterations it = 4 kk + mu in pairs, the even
                // one in ra, the odd one in rb
                const float* rn = R + (size_t)k0 * fs + (size_t)yn * 32;   // (k0 + kk, mu) at rn + kk fs + 8 mu
                auto contract = [&](const float (&rv)[8], int it) {
                    float wv[8];
                    lds8(wrow + (it >> 2) * 32 + (it & 3) * 8, wv);
#pragma unroll
                    for (int b = 0; b < 8; b++)
#pragma unroll
                        for (int d = 0; d < 8; d++) C[b][d] = fmaf(rv[b], wv[d], C[b][d]);
                };
                float ra[8], rb[8];
                load8_v8(rn, ra);
                for (int it = 0; it < 4 * kc; it += 2) {
                    load8_v8(rn + (size_t)((it + 1) >> 2) * fs + ((it + 1) & 3) * 8, rb);   // it + 1 < 4 kc always
                    contract(ra, it);
                    if (it + 2 < 4 * kc) load8_v8(rn + (size_t)((it + 2) >> 2) * fs + ((it + 2) & 3) * 8, ra);
                    contract(rb, it + 1);
                }
            }
        }
        if (live) {
            const mat3<float> u = LinkLoad<float, LF>::load(U, y, q);
            float Gk[8];
#pragma unroll
            for (int a = 0; a < 8; a++) Gk[a] = 0.f;
#pragma unroll
            for (int d = 0; d < 8; d++) {
                float col[8], rc[8];
#pragma unroll
                for (int b = 0; b < 8; b++) col[b] = C[b][d];
                herm<float> E = h_zero<float>();
                acc_uxud_tl(E, u, coef_to_herm2(col));   // 2 sum_c (R C)_cd T^c
                herm2_to_coef_tl(E, rc);                  // (R C)_cd
                f_contract(d, rc, Gk);
            }
            double* out = G + (size_t)y * 32 + q * 8;
#pragma unroll
            for (int a = 0; a < 8; a++) out[a] = (double)Gk[a] * (1.0 / 16.0);
        }
    }
}

// The same contraction with eight lanes per link pair: the two halves of each (site, direction) split the rows b
// of C (C[b][d], b = 4 h + i), so that a lane holds 32 accumulators instead of 64 and chunks of 8 basis vectors
// (instead of 4) halve the passes over the site's own basis rows.  The half h is uniform per warp (threads
// 0..127: h = 0, 128..255: h = 1), so no branch on it diverges; the two halves' force contributions meet in
// shared memory in a fixed order.  The conjugation by the link uses the adjoint matrix (the lane's four
// columns of Ad(U_nu(y))).
constexpr int kLsSites = 32;             // sites per block: 4 directions x 2 halves = 8 lanes each
constexpr int kLsKC = 8;                 // basis vectors per chunk of W
constexpr int kLsPad = kLsKC * 32 + 4;   // W per site: [kk][mu][8] + 4

template <int LF>
__global__ void __launch_bounds__(kLsSites * 8, 2) k_link_grad_split(Geom g, Links32 U, const float* __restrict__ R,
                                                                     size_t fs, const int* __restrict__ flags, int n,
                                                                     const double* __restrict__ S, int ld,
                                                                     double* __restrict__ G) {
    __shared__ __align__(16) float Ws[kLsSites * kLsPad];
    __shared__ float Ss[kLsKC * kBasisCap];
    __shared__ float Gh[kLsSites * 4 * 8];   // the h = 1 halves' contributions
    if (flags) n = flags[1];
    const int h = threadIdx.x >> 7, sl = (threadIdx.x & 127) >> 2, nu = threadIdx.x & 3;
    float* const wrow = Ws + sl * kLsPad;
    for (int base = blockIdx.x * kLsSites; base < g.V; base += gridDim.x * kLsSites) {
        const int y = base + sl;
        const bool live = y < g.V;
        const int yn = live ? step_site(g, y, nu, 1) : 0;
        float C[4][8];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int d = 0; d < 8; d++) C[i][d] = 0.f;
        for (int k0 = 0; k0 < n; k0 += kLsKC) {
            __syncthreads();
            for (int t = threadIdx.x; t < kLsKC * n; t += blockDim.x) {
                const int kk = t / n, l = t - kk * n;
                Ss[kk * kBasisCap + l] = k0 + kk < n ? (float)S[(size_t)(k0 + kk) * ld + l] : 0.f;
            }
            __syncthreads();
            // W_k,mu(y) = sum_l S_kl r_l,mu(y) for this half's four k of the chunk (mu = nu)
            float w[4][8];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int a = 0; a < 8; a++) w[i][a] = 0.f;
            if (live) {
                for (int l = 0; l < n; l++) {
                    float r[8];
                    load8_v8(R + (size_t)l * fs + (size_t)y * 32 + nu * 8, r);
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const float sv = Ss[(4 * h + i) * kBasisCap + l];
#pragma unroll
                        for (int a = 0; a < 8; a++) w[i][a] = fmaf(sv, r[a], w[i][a]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 4; i++) store8(wrow + (4 * h + i) * 32 + nu * 8, w[i]);
            __syncthreads();
            // C[b][d] += r_k,mu(y+nu)[b] W_k,mu(y)[d] for the rows b = 4 h + i
            if (live) {
                const int kc = min(kLsKC, n - k0);
                for (int kk = 0; kk < kc; kk++) {
                    const float* rk = R + (size_t)(k0 + kk) * fs + (size_t)yn * 32 + 4 * h;
#pragma unroll
                    for (int mu = 0; mu < 4; mu++) {
                        const float4 rp = __ldg(reinterpret_cast<const float4*>(rk + mu * 8));
                        float wv[8];
                        lds8(wrow + kk * 32 + mu * 8, wv);
                        const float rb[4] = {rp.x, rp.y, rp.z, rp.w};
#pragma unroll
                        for (int i = 0; i < 4; i++)
#pragma unroll
                            for (int d = 0; d < 8; d++) C[i][d] = fmaf(rb[i], wv[d], C[i][d]);
                    }
                }
            }
        }
        // G^a = (1/16) sum_cd f_acd (Ad C)_cd; this half contributes the columns b = 4 h + i of Ad
        float Gk[8];
#pragma unroll
        for (int a = 0; a < 8; a++) Gk[a] = 0.f;
        if (live) {
            const mat3<float> u = LinkLoad<float, LF>::load(U, y, nu);
            float cols[4][8];
            adjoint_columns(u, [&](int bcol, const float (&col)[8]) {
                if ((bcol >> 2) == h)
#pragma unroll
                    for (int c = 0; c < 8; c++) cols[bcol & 3][c] = col[c];
            });
#pragma unroll
            for (int d = 0; d < 8; d++) {
                float rc[8];
#pragma unroll
                for (int c = 0; c < 8; c++) {
                    float v = 0.f;
#pragma unroll
                    for (int i = 0; i < 4; i++) v = fmaf(cols[i][c], C[i][d], v);
                    rc[c] = v;
                }
                f_contract(d, rc, Gk);
            }
        }
        if (h == 1) {
#pragma unroll
            for (int a = 0; a < 8; a++) Gh[(sl * 4 + nu) * 8 + a] = Gk[a];
        }
        __syncthreads();
        if (h == 0 && live) {
            double* out = G + (size_t)y * 32 + nu * 8;
#pragma unroll
            for (int a = 0; a < 8; a++) out[a] = (double)(Gk[a] + Gh[(sl * 4 + nu) * 8 + a]) * (1.0 / 16.0);
        }
        __syncthreads();   // Gh is rewritten by the next tile
    }
}

// The contraction of k_link_grad_krylov with the neighbour rows staged: in the C phase, lane (y, nu) needs
// the whole row r_k(y + nu) (128 bytes); read lane by lane, one load instruction of a warp touches 32
// different rows (one 32-byte sector each).  Here the 4 lanes of a site instead load the 4 chunks of each of
// its 4 neighbour rows (one instruction: 8 whole rows), store them to shared memory (rows padded to 36
// floats: a warp's 128-bit accesses fall on distinct bank quads), and after a warp barrier (the four lanes of a
// site are in one warp) every lane reads its own row there.
constexpr int kNbRow = 36;
template <int LF>
__global__ void __launch_bounds__(kLgSites * 4, 4) k_link_grad_nbs(Geom g, Links32 U, const float* __restrict__ R,
                                                                size_t fs, const int* __restrict__ flags, int n,
                                                                const double* __restrict__ S, int ld,
                                                                double* __restrict__ G) {
    __shared__ __align__(16) float Ws[kLgSites * kLgPad];
    __shared__ float Ss[kLgKC * kBasisCap];
    __shared__ __align__(16) float Nb[4 * kLgSites * kNbRow];   // [nu][site][kNbRow]
    if (flags) n = flags[1];
    const int sl = threadIdx.x >> 2, q = threadIdx.x & 3;
    float* const wrow = Ws + sl * kLgPad;
    for (int base = blockIdx.x * kLgSites; base < g.V; base += gridDim.x * kLgSites) {
        const int y = base + sl;
        const bool live = y < g.V;
        int fwd[4] = {0, 0, 0, 0}, bwd[4];
        if (live) neighbours(g, y, fwd, bwd);
        float C[8][8];
#pragma unroll
        for (int b = 0; b < 8; b++)
#pragma unroll
            for (int d = 0; d < 8; d++) C[b][d] = 0.f;
        // chunk q of the 4 neighbour rows of basis vector k: registers, then shared memory
        float t[4][8];
        auto gload = [&](int k) {
            const float* rk = R + (size_t)k * fs + q * 8;
#pragma unroll
            for (int nu = 0; nu < 4; nu++) load8_v8(rk + (size_t)fwd[nu] * 32, t[nu]);
        };
        auto sstore = [&]() {
#pragma unroll
            for (int nu = 0; nu < 4; nu++) {
                float4* d = reinterpret_cast<float4*>(Nb + (nu * kLgSites + sl) * kNbRow + q * 8);
                d[0] = make_float4(t[nu][0], t[nu][1], t[nu][2], t[nu][3]);
                d[1] = make_float4(t[nu][4], t[nu][5], t[nu][6], t[nu][7]);
            }
        };
        const float* const nrow = Nb + (q * kLgSites + sl) * kNbRow;
        for (int k0 = 0; k0 < n; k0 += kLgKC) {
            __syncthreads();
            for (int i = threadIdx.x; i < kLgKC * n; i += blockDim.x) {
                const int kk = i / n, l = i - kk * n;
                Ss[kk * kBasisCap + l] = k0 + kk < n ? (float)S[(size_t)(k0 + kk) * ld + l] : 0.f;
            }
            __syncthreads();
            float w[kLgKC][8];
#pragma unroll
            for (int kk = 0; kk < kLgKC; kk++)
#pragma unroll
                for (int a = 0; a < 8; a++) w[kk][a] = 0.f;
            if (live) {
                for (int l = 0; l < n; l++) {
                    float r[8];
                    load8_v8(R + (size_t)l * fs + (size_t)y * 32 + q * 8, r);
#pragma unroll
                    for (int kk = 0; kk < kLgKC; kk++) {
                        const float sv = Ss[kk * kBasisCap + l];
#pragma unroll
                        for (int a = 0; a < 8; a++) w[kk][a] = fmaf(sv, r[a], w[kk][a]);
                    }
                }
            }
#pragma unroll
            for (int kk = 0; kk < kLgKC; kk++) store8(wrow + kk * 32 + q * 8, w[kk]);
            const int kc = min(kLgKC, n - k0);   // uniform over the block
            for (int kk = 0; kk < kc; kk++) {
                if (live) {
                    gload(k0 + kk);
                    sstore();
                }
                __syncwarp();   // the rows of k (and, for kk = 0, the chunk's W) are in place: a site's
                                // rows and W are written and read by its own four lanes, within one warp
                if (live) {
#pragma unroll
                    for (int mu = 0; mu < 4; mu++) {
                        float rp[8], wv[8];
                        lds8(nrow + mu * 8, rp);
                        lds8(wrow + kk * 32 + mu * 8, wv);
#pragma unroll
                        for (int b = 0; b < 8; b++)
#pragma unroll
                            for (int d = 0; d < 8; d++) C[b][d] = fmaf(rp[b], wv[d], C[b][d]);
                    }
                }
                __syncwarp();   // the site's lanes have read the rows of k
            }
        }
        if (live) {
            const mat3<float> u = LinkLoad<float, LF>::load(U, y, q);
            float Gk[8];
#pragma unroll
            for (int a = 0; a < 8; a++) Gk[a] = 0.f;
#pragma unroll
            for (int d = 0; d < 8; d++) {
                float col[8], rc[8];
#pragma unroll
                for (int b = 0; b < 8; b++) col[b] = C[b][d];
                herm<float> E = h_zero<float>();
                acc_uxud_tl(E, u, coef_to_herm2(col));   // 2 sum_c (R C)_cd T^c
                herm2_to_coef_tl(E, rc);                  // (R C)_cd
                f_contract(d, rc, Gk);
            }
            double* out = G + (size_t)y * 32 + q * 8;
#pragma unroll
            for (int a = 0; a < 8; a++) out[a] = (double)Gk[a] * (1.0 / 16.0);
        }
    }
}

// F_K from the basis rows (X_j rows 0..ns-1, Z_j rows ns..2ns-1, row stride ldr, device float64) of the
// float32 basis R; n on the host, or read on the device from flags[1] when flags is given
int link_grad_krylov_launch(rmhmc_ctx* ctx, const float* R, const double* rows, int ldr, int ns, const double* alpha,
                            const int* flags, int n, double* F, cudaStream_t st) {
    if (ns > kMaxPairs) return set_err(ctx, RMHMC_EINVAL, "at most %d poles", kMaxPairs);
    int status = RMHMC_OK;
    double* S = (double*)workspace(ctx, "kf_pairs", sizeof(double) * kBasisCap * kBasisCap, &status);
    if (!S) return status;
    PairWeights pw{};
    for (int j = 0; j < ns; j++) pw.w[j] = alpha[j];
    k_pair_matrix<<<ctx->num_sms / 4 > 1 ? ctx->num_sms / 4 : 1, 256, 0, st>>>(rows, ldr, ns, pw, flags, n, S, kBasisCap);
    ++ctx->launches;
    if (ctx->lg_mode == 3) {
        const int grid = capped_grid(ctx, (size_t)ctx->g.V * 4, kLgSites * 4);
        k_link_grad_nbs<18><<<grid, kLgSites * 4, 0, st>>>(ctx->g, links32(ctx), R, field_elems(ctx), flags, n, S,
                                                           kBasisCap, F);
    } else if (ctx->lg_mode == 2) {
        const int ntile = (ctx->g.V + kLsSites - 1) / kLsSites;
        const int grid = std::max(1, std::min(ntile, (int)ctx->num_sms * 2));
        k_link_grad_split<18><<<grid, kLsSites * 8, 0, st>>>(ctx->g, links32(ctx), R, field_elems(ctx), flags, n, S,
                                                             kBasisCap, F);
    } else if (ctx->lg_mode == 1) {
        static bool configured[64] = {};
        if (ctx->device < 0 || ctx->device >= 64) return set_err(ctx, RMHMC_EINVAL, "device index too large");
        if (!configured[ctx->device]) {
            RM_CHECK(ctx, cudaFuncSetAttribute(k_link_grad_staged<18>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)lg_staged_smem()));
            configured[ctx->device] = true;
        }
        int per_sm = 0;
        RM_CHECK(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_link_grad_staged<18>, kLgSites * 4,
                                                                    lg_staged_smem()));
        const int ntile = (ctx->g.V + kLgSites - 1) / kLgSites;
        const int grid = std::max(1, std::min(ntile, (int)ctx->num_sms * std::max(per_sm, 1)));
        k_link_grad_staged<18><<<grid, kLgSites * 4, lg_staged_smem(), st>>>(ctx->g, links32(ctx), R, field_elems(ctx),
                                                                             flags, n, S, kBasisCap, F);
    } else {
        const int grid = capped_grid(ctx, (size_t)ctx->g.V * 4, kLgSites * 4);
        k_link_grad_krylov<float, 18><<<grid, kLgSites * 4, 0, st>>>(ctx->g, links32(ctx), R, field_elems(ctx), flags, n,
                                                                     S, kBasisCap, F);
    }
    ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    return RMHMC_OK;
}

// ------------------------------------------------------------------------------------------------
// kinetic pieces from a single Krylov run on P
// ------------------------------------------------------------------------------------------------
template <typename T>
static int kinetic_t(rmhmc_ctx* ctx, const MassTerm& m, const T* P, const double* P64, double tol, int maxiter, double* F,
                     double* Vel, double* Tkin, int* iters, cudaStream_t st) {
    const int ns = m.npole();
    const size_t fs = field_elems(ctx);
    int status = RMHMC_OK;
    if (ns == 0) {
        // M = c^{-2}: V = c^2 P, F_K = 0, T = c^2 |P|^2 / 2
        if (F) RM_CHECK(ctx, cudaMemsetAsync(F, 0, sizeof(double) * fs, st));
        if (Vel) RM_TRY(axpby64(ctx, m.c * m.c, P64, 0.0, nullptr, Vel, fs, st));
        if (Tkin) {
            double n2 = 0.0;
            RM_TRY(norm2_64(ctx, P64, fs, &n2, st));
            *Tkin = 0.5 * m.c * m.c * n2;
        }
        if (iters) *iters = 0;
        return RMHMC_OK;
    }
    const double s0 = *std::min_element(m.sigma.begin(), m.sigma.end());
    KrylovResult kr;
    RM_TRY(krylov_run<T>(ctx, P, s0, tol, maxiter, kr, st));
    if (kr.status == 2) return set_err(ctx, RMHMC_ENOCONV, "kinetic force: Krylov run hit its cap (%d)", kr.n);
    if (iters) *iters = kr.n;
    Tridiag tri;
    tri.build(kr);
    const int n = tri.n;
    // Galerkin coefficient vectors: y_j = (T+D_j)^{-1} e1|b|, g = R(T) e1|b|, z_j = (T+D_j)^{-1} g, v = R(T) g
    std::vector<double> e1(n, 0.0), g(n, 0.0), v(n, 0.0);
    if (n > 0) e1[0] = tri.bnorm;
    std::vector<std::vector<double>> ys(ns), zs(ns);
    for (int j = 0; j < ns; j++) tri.solve(m.sigma[j] - s0, e1, ys[j]);
    for (int k = 0; k < n; k++) {
        g[k] = m.c * e1[k];
        for (int j = 0; j < ns; j++) g[k] += m.alpha[j] * ys[j][k];
    }
    for (int j = 0; j < ns; j++) tri.solve(m.sigma[j] - s0, g, zs[j]);
    for (int k = 0; k < n; k++) {
        v[k] = m.c * g[k];
        for (int j = 0; j < ns; j++) v[k] += m.alpha[j] * zs[j][k];
    }
    if (Tkin) {
        // T = 1/2 |R P|^2 from the explicitly formed R P (float64 sum), not from |g|, which would
        // assume exactly orthonormal Lanczos vectors
        double* Y = (double*)workspace(ctx, "kf_y", sizeof(double) * fs, &status);
        if (!Y) return status;
        CombineSpec spec;
        spec.n = n;
        spec.M = 1;
        spec.coef.assign(n, 0.0);
        tri.to_basis(g, spec.coef.data());
        double* o[1] = {Y};
        RM_TRY((krylov_combine<T, double>(ctx, spec, o, st)));
        double y2 = 0.0;
        RM_TRY(norm2_64(ctx, Y, fs, &y2, st));
        *Tkin = 0.5 * y2;
    }
    if (Vel) {
        CombineSpec spec;
        spec.n = n;
        spec.M = 1;
        spec.coef.assign(n, 0.0);
        tri.to_basis(v, spec.coef.data());
        double* o[1] = {Vel};
        RM_TRY((krylov_combine<T, double>(ctx, spec, o, st)));
    }
    if (F && sizeof(T) == 4) {
        // float32 basis: the force straight from the basis (rows of X_j and Z_j on the stored residuals)
        double* rows = (double*)workspace(ctx, "kf_rows", sizeof(double) * (size_t)2 * ns * kBasisCap, &status);
        if (!rows) return status;
        std::vector<double> h((size_t)2 * ns * n, 0.0);
        for (int j = 0; j < ns; j++) {
            tri.to_basis(ys[j], h.data() + (size_t)j * n);
            tri.to_basis(zs[j], h.data() + (size_t)(ns + j) * n);
        }
        RM_TRY(upload(ctx, rows, h.data(), sizeof(double) * h.size(), st));
        RM_TRY(link_grad_krylov_launch(ctx, (const float*)krylov_basis<T>(ctx), rows, n, ns, m.alpha.data(), nullptr, n,
                                       F, st));
    } else if (F) {
        T* XZ = (T*)workspace(ctx, "kf_xz64", sizeof(T) * fs * 2 * ns, &status);
        if (!XZ) return status;
        CombineSpec spec;
        spec.n = n;
        spec.M = 2 * ns;
        spec.coef.assign((size_t)2 * ns * n, 0.0);
        std::vector<T*> outs(2 * ns);
        for (int j = 0; j < ns; j++) {
            tri.to_basis(ys[j], spec.coef.data() + (size_t)j * n);
            tri.to_basis(zs[j], spec.coef.data() + (size_t)(ns + j) * n);
            outs[j] = XZ + (size_t)j * fs;
            outs[ns + j] = XZ + (size_t)(ns + j) * fs;
        }
        RM_TRY((krylov_combine<T, T>(ctx, spec, outs.data(), st)));
        RM_TRY(link_grad_launch(ctx, sizeof(T) == 8 ? RMHMC_FP64 : RMHMC_FP32, XZ, XZ + (size_t)ns * fs, ns,
                                m.alpha.data(), F, st));
    }
    return RMHMC_OK;
}

int kinetic_from_krylov(rmhmc_ctx* ctx, const MassTerm& m, const double* P, double tol, int maxiter, int prec,
                        double* F, double* Vel, double* T, int* iters, cudaStream_t st) {
    if (prec == RMHMC_FP64) return kinetic_t<double>(ctx, m, P, P, tol, maxiter, F, Vel, T, iters, st);
    int status = RMHMC_OK;
    const size_t fs = field_elems(ctx);
    float* P32 = (float*)workspace(ctx, "kf_p32", sizeof(float) * fs, &status);
    if (!P32) return status;
    RM_TRY(to_float(ctx, P, P32, fs, st));
    return kinetic_t<float>(ctx, m, P32, P, tol, maxiter, F, Vel, T, iters, st);
}

}  // namespace rm

using namespace rm;

extern "C" int lap_link_grad(rmhmc_ctx* ctx, const double* U, const double* X, const double* Z, int nfield,
                             const double* w, int prec, double* G, cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (!X || !Z || !G || (nfield > 0 && !w)) return set_err(ctx, RMHMC_EINVAL, "lap_link_grad: null argument");
    if (nfield < 0 || nfield > kMaxPairs) return set_err(ctx, RMHMC_EINVAL, "lap_link_grad: nfield in [0, %d]", kMaxPairs);
    if (prec != RMHMC_FP64 && prec != RMHMC_FP32) return set_err(ctx, RMHMC_EINVAL, "lap_link_grad: bad prec");
    RM_TRY(ensure_links(ctx, U, stream));
    const size_t fs = field_elems(ctx);
    if (nfield == 0) {
        RM_CHECK(ctx, cudaMemsetAsync(G, 0, sizeof(double) * fs, stream));
        return RMHMC_OK;
    }
    if (prec == RMHMC_FP64) return link_grad_launch(ctx, prec, X, Z, nfield, w, G, stream);
    int status = RMHMC_OK;
    float* buf = (float*)workspace(ctx, "lg_xz32", sizeof(float) * fs * 2 * nfield, &status);
    if (!buf) return status;
    RM_TRY(to_float(ctx, X, buf, fs * nfield, stream));
    RM_TRY(to_float(ctx, Z, buf + fs * nfield, fs * nfield, stream));
    return link_grad_launch(ctx, prec, buf, buf + fs * nfield, nfield, w, G, stream);
}

extern "C" int kinetic_force(rmhmc_ctx* ctx, const double* U, const double* P, const rmhmc_mass* mass, double tol,
                             int prec, double* F, double* Vout, double* T, cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (!P) return set_err(ctx, RMHMC_EINVAL, "kinetic_force: null momenta");
    if (!(tol > 0.0)) return set_err(ctx, RMHMC_EINVAL, "kinetic_force: tol must be > 0");
    if (prec != RMHMC_FP64 && prec != RMHMC_MIXED) return set_err(ctx, RMHMC_EINVAL, "kinetic_force: bad prec");
    MassTerm m;
    RM_TRY(parse_mass(ctx, mass, m));
    RM_TRY(ensure_links(ctx, U, stream));
    return kinetic_from_krylov(ctx, m, P, tol, 1000, prec, F, Vout, T, nullptr, stream);
}

extern "C" int rmhmc_heatbath(rmhmc_ctx* ctx, const double* U, const double* xi, const rmhmc_mass* mass, double tol,
                              int prec, double* P, cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (!xi || !P) return set_err(ctx, RMHMC_EINVAL, "rmhmc_heatbath: null field");
    if (!(tol > 0.0)) return set_err(ctx, RMHMC_EINVAL, "rmhmc_heatbath: tol must be > 0");
    if (prec != RMHMC_FP64 && prec != RMHMC_MIXED) return set_err(ctx, RMHMC_EINVAL, "rmhmc_heatbath: bad prec");
    MassTerm m;
    RM_TRY(parse_mass(ctx, mass, m));
    RM_TRY(ensure_links(ctx, U, stream));
    return heatbath_apply(ctx, m, xi, tol, 1000, prec, P, stream);
}
