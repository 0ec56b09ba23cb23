// Philox4x32-10 counter-based generator on the device.
//
// Written from the published definition (Salmon, Moraes, Dror, Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11): each of the ten rounds forms
// two 32x32->64-bit products of counter words with fixed multipliers, mixes
// the halves with the other counter words and the key, and the key advances
// by the Weyl constants between rounds.
#pragma once
#include <cstdint>

namespace relaybp {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k.x += W0; k.y += W1; }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t uint4_word(const uint4 &v, int t)
{
    return t == 0 ? v.x : (t == 1 ? v.y : (t == 2 ? v.z : v.w));
}

// Counter layout shared by the sampler (stream 0) and the memory-strength
// draws (stream 1): (block index, shot low word, shot high word, stream).
__device__ __forceinline__ uint4 philox_block(uint64_t seed, uint64_t shot, uint32_t stream, uint32_t block)
{
    return philox4x32_10(make_uint4(block, (uint32_t)shot, (uint32_t)(shot >> 32), stream),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

}  // namespace relaybp
