// Counter-based start vectors of the FTLM chains (Section 2.2: normalised
// Gaussian random vectors; Rademacher +-1 for the batched configurations).
// Philox4x32-10 of Salmon, Moraes, Dror and Shaw (SC'11), written from its
// published definition: key (k0, k1), counter (c0, c1, c2, c3), ten rounds of
// the two multiplications with the key schedule bumped by the Weyl constants.
#pragma once

#include <math.h>
#include <stdint.h>

#include "ftlm.h"

namespace ftlm {

struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    }
    return c;
}

__device__ __forceinline__ double start_value(uint64_t row, uint32_t chain, uint32_t k0, uint32_t k1, int rng) {
    const U4 o = philox4x32_10(U4{(uint32_t)row, (uint32_t)(row >> 32), chain, 0u}, k0, k1);
    if (rng == FTLM_RADEMACHER) return (o.x & 1u) ? -1.0 : 1.0;
    const double u1 = ((double)(((uint64_t)(o.x >> 5) << 26) | (o.y >> 6)) + 0.5) * 0x1p-53;
    const double u2 = (double)(((uint64_t)(o.z >> 5) << 26) | (o.w >> 6)) * 0x1p-53;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

// The same draw for FP32 arithmetic (FP32 or FP16 vectors, which store it in
// FP32 or less): the same Philox words and uniforms, Box–Muller evaluated in
// FP32.  log(u1) is taken as log(u1) for u1 < 1/2 and as log1p(-(1 - u1))
// otherwise, so no uniform loses its accuracy; the result is within a few FP32
// ulps of the FP64 draw.  The uniforms are the exact dyadic numbers
// u1 = (2k + 1) 2^-54, 1 - u1 = (2^54 - 2k - 1) 2^-54 and u2 = m 2^-53, each
// rounded once to FP32 (integer-to-float conversion, then an exact power-of-two
// scale), with no FP64 arithmetic (1/70 of the FP32 rate on this GPU).
__device__ __forceinline__ float start_value_f32(uint64_t row, uint32_t chain, uint32_t k0, uint32_t k1, int rng) {
    const U4 o = philox4x32_10(U4{(uint32_t)row, (uint32_t)(row >> 32), chain, 0u}, k0, k1);
    if (rng == FTLM_RADEMACHER) return (o.x & 1u) ? -1.f : 1.f;
    const uint64_t k = ((uint64_t)(o.x >> 5) << 26) | (o.y >> 6);  // u1 = (k + 1/2) 2^-53
    const float lg = k < (1ull << 52) ? logf(__ull2float_rn(2 * k + 1) * 0x1p-54f)
                                      : log1pf(-(__ull2float_rn((1ull << 54) - 2 * k - 1) * 0x1p-54f));
    const float u2 = __ull2float_rn(((uint64_t)(o.z >> 5) << 26) | (o.w >> 6)) * 0x1p-53f;
    return sqrtf(-2.f * lg) * cospif(2.f * u2);
}

template <typename VT>
__device__ __forceinline__ VT start_value_t(uint64_t row, uint32_t chain, uint32_t k0, uint32_t k1, int rng) {
    if constexpr (sizeof(VT) == 4)
        return start_value_f32(row, chain, k0, k1, rng);
    else
        return start_value(row, chain, k0, k1, rng);
}

}  // namespace ftlm
