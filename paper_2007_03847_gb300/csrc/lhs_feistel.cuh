// The per-dimension stratum permutation of the Latin hypercube design
// (Section IV-B step 1): a keyed balanced Feistel network with cycle walking,
// stateless, so that any (sample, dimension) is computed on its own.
#pragma once

#include <stdint.h>

#include "fmc_common.cuh"

namespace fmc {

constexpr int kFeistelRounds = 6;

// Balanced Feistel network on 2h bits; round function = Philox word 0 of the
// counter (R, dim, 1 + round, 0) masked to h bits.
__device__ __forceinline__ uint32_t feistel(uint32_t x, uint32_t dim, int h, uint32_t mask, uint32_t k0,
                                            uint32_t k1)
{
    uint32_t L = (x >> h) & mask;
    uint32_t R = x & mask;
#pragma unroll
    for (int r = 0; r < kFeistelRounds; ++r) {
        U4 o = philox4x32_10(U4{R, dim, 1u + (uint32_t)r, 0u}, k0, k1);
        uint32_t nL = R;
        R = L ^ (o.x & mask);
        L = nL;
    }
    return (L << h) | R;
}

// pi_dim(k): cycle walking restricts the permutation of [0, 2^(2h)) to [0, N);
// it ends because the cycle through k < N returns to [0, N) within 2^(2h) - N + 1
// applications.
__device__ __forceinline__ uint32_t stratum(uint32_t k, uint32_t dim, uint32_t N, int h, uint32_t mask,
                                            uint32_t k0, uint32_t k1)
{
    uint32_t y = k;
    do {
        y = feistel(y, dim, h, mask, k0, k1);
    } while (y >= N);
    return y;
}

struct FeistelShape {
    int h;
    uint32_t mask;
};

inline FeistelShape feistel_shape(int64_t N)
{
    int b = 0;
    while ((int64_t(1) << b) < N) ++b;
    int h = (b + 1) / 2;
    if (h < 1) h = 1;
    FeistelShape f;
    f.h = h;
    f.mask = (h >= 32) ? 0xFFFFFFFFu : ((1u << h) - 1u);
    return f;
}

}  // namespace fmc
