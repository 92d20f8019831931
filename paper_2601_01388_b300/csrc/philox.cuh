// Counter-based random numbers for the device side: Philox4x64-10 written from its
// definition in Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as
// 1, 2, 3" (SC'11) -- ten rounds, each two 64x64 -> 128-bit products of counter words
// with the Philox multipliers, the round key advanced by the two Weyl increments
// between rounds.
#pragma once
#include <stdint.h>

namespace agis {

struct U128 { uint64_t lo, hi; };

__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                              uint64_t k0, uint64_t k1, uint64_t &o0, uint64_t &o1)
{
    const uint64_t kMulA = 0xD2E7470EE14C6C93ull, kMulB = 0xCA5A826395121157ull;
    const uint64_t kWeylA = 0x9E3779B97F4A7C15ull, kWeylB = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t hA = __umul64hi(kMulA, c0), lA = kMulA * c0;
        const uint64_t hB = __umul64hi(kMulB, c2), lB = kMulB * c2;
        const uint64_t n0 = hB ^ c1 ^ k0, n2 = hA ^ c3 ^ k1;
        c0 = n0; c1 = lB; c2 = n2; c3 = lA;
        k0 += kWeylA; k1 += kWeylB;
    }
    o0 = c0; o1 = c1;
}

// floor(U * W / 2^128) with U the first 128 bits (word 1 high, word 0 low) of the
// block at counter (a, b, stream, 0), key (seed, 0): an exact integer draw in [0, W).
__device__ __forceinline__ uint64_t draw_below(uint64_t W, uint64_t a, uint64_t b,
                                               uint64_t stream, uint64_t seed)
{
    uint64_t u0, u1;
    philox4x64_10(a, b, stream, 0, seed, 0, u0, u1);
    // U*W = u1*W*2^64 + u0*W; the result is the part above bit 128
    const uint64_t lo_hi = __umul64hi(u0, W);          // bits 64.. of u0*W
    const uint64_t mid_lo = u1 * W, mid_hi = __umul64hi(u1, W);
    const uint64_t s = mid_lo + lo_hi;
    return mid_hi + (s < mid_lo ? 1u : 0u);
}

}  // namespace agis
