// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11), device side.
//
// Ten rounds; each round multiplies counter words 0 and 2 by the two Philox
// multipliers into 64-bit products, swaps the halves across the four words and
// mixes in the round key; the key advances by the two Weyl constants between
// rounds.  The round keys depend only on the simulation seed, so callers that
// draw many blocks with one key precompute them once (PhiloxKey).
#pragma once
#include <cstdint>

namespace cuba {

struct PhiloxKey {
    uint32_t k0[10];
    uint32_t k1[10];
};

__host__ __device__ __forceinline__ PhiloxKey philox_schedule(uint32_t key0, uint32_t key1)
{
    PhiloxKey s;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        s.k0[r] = key0 + (uint32_t)r * 0x9E3779B9u;
        s.k1[r] = key1 + (uint32_t)r * 0xBB67AE85u;
    }
    return s;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKey& k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ k.k0[r], lo1, hi0 ^ c.w ^ k.k1[r], lo0);
    }
    return c;
}

// Counter layout of the random streams used by the step (fourth word tags).
constexpr uint32_t kTagFine = 0x40000000u;   // low 24 bits of a pair's uniform
constexpr uint32_t kTagAngle = 0x80000000u;  // centre-of-mass direction
constexpr uint32_t kStepInit = 0xFFFFFFFFu;  // first word reserved for sampling

}  // namespace cuba
