// Autotuner of the stencil launch shape: components per lane (NMU = 1, 2, 4, i.e. 4, 2 or 1 lanes per
// site, or the prefetching one-component variant) and threads per block (64, 128, 256).  On first use of a (precision, link format) in a context,
// every shape is timed with CUDA events on the context's own lattice (a plain A X application on scratch
// fields, three repetitions after a warm-up) and the fastest is kept for every stencil kernel of that
// precision and link format.
#pragma once
#include "common.cuh"

namespace rm {

// nmu: components per lane (1, 2, 4), or 0 for one component per lane with all neighbour values
// prefetched before the arithmetic, or 8 for the link-centric adjoint kernel (float32, 4D boxes swept in t)
struct StencilShape {
    int nmu = 1;
    int block = 128;
};
// minimum resident blocks of kBlockMax threads each stencil shape is compiled for (the register budget): the
// float32 one-component shape fits 64 registers (4 blocks, 32 warps per SM), the two-component and
// prefetching shapes 85 (3 blocks), the four-component shape 128 (2 blocks); float64 shapes are not bounded
template <typename T, int NMU> constexpr int stencil_min_blocks() {
    return sizeof(T) == 8 ? 1 : NMU == 1 ? 4 : NMU == 4 ? 2 : 3;
}

inline int lanes_per_site(int nmu) { return nmu == 0 ? 4 : nmu == 8 ? 4 : 4 / nmu; }

// shape for (sizeof(T), LF); tunes on first use
template <typename T, int LF>
int stencil_shape(rmhmc_ctx* ctx, cudaStream_t st, StencilShape& out);

inline int stencil_blocks(const rmhmc_ctx* ctx, const StencilShape& sh) {
    return capped_grid(ctx, (size_t)ctx->g.V * lanes_per_site(sh.nmu), sh.block);
}

}  // namespace rm
