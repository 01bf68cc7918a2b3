// Counter-based generator Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), host and device,
// and the Gaussian / uniform draws built on it: the momentum refresh and the Metropolis test of Sec. 3
// and the noise vectors of the trace in Eq. (4).
//   block: counter {c0, c1, c2, c3}, key {k0, k1}; ten rounds, key bumped by the Weyl constants
//   between rounds.  Uniforms take 53 bits from two 32-bit words and lie in (0, 1].
#pragma once
#include <stdint.h>
#include <math.h>

namespace rm {

struct u32x4 { uint32_t v[4]; };

__host__ __device__ __forceinline__ void mulhilo32(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

__host__ __device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c.v[0], hi0, lo0);
        mulhilo32(0xCD9E8D57u, c.v[2], hi1, lo1);
        u32x4 n;
        n.v[0] = hi1 ^ c.v[1] ^ k0;
        n.v[1] = lo1;
        n.v[2] = hi0 ^ c.v[3] ^ k1;
        n.v[3] = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__host__ __device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
    const uint64_t k = ((uint64_t)(hi >> 5) << 26) | (uint64_t)(lo >> 6);
    return ((double)k + 1.0) * 0x1p-53;
}

// Metropolis uniform: block {0, 0xFFFFFFFF, stream, tag}
__host__ __device__ __forceinline__ double philox_uniform(uint64_t seed, uint32_t stream, uint32_t tag) {
    u32x4 c{{0u, 0xFFFFFFFFu, stream, tag}};
    const u32x4 w = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return u53(w.v[0], w.v[1]);
}

}  // namespace rm
