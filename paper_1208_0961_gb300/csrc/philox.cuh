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

// Philox blocks of counters (a, b, c, d) that share a, b, c and differ in d
// only.  The first round's two products and its words X1, Y1, W1 do not depend
// on d, nor do the second round's M0 product and the third round's M1
// product; they are computed once per (a, b, c).  block(d) returns exactly
// philox4x32_10((a, b, c, d), key).
struct PhiloxRow {
    uint32_t A;   // round 0: Z1 = A ^ d
    uint32_t B;   // round 1: X2 = hi(M1 Z1) ^ B
    uint32_t F;   // round 2: X3 = lo(M1 Z1) ^ F
    uint32_t G;   // round 2: Z3 = hi(M0 X2) ^ G
    uint32_t Y3;  // round 2: Y3 (invariant)

    __device__ __forceinline__ void init(uint32_t a, uint32_t b, uint32_t c, const PhiloxKey& k)
    {
        const uint64_t p0 = (uint64_t)0xD2511F53u * a;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c;
        const uint32_t X1 = (uint32_t)(p1 >> 32) ^ b ^ k.k0[0];
        const uint32_t Y1 = (uint32_t)p1;
        const uint32_t W1 = (uint32_t)p0;
        A = (uint32_t)(p0 >> 32) ^ k.k1[0];
        const uint64_t q0 = (uint64_t)0xD2511F53u * X1;       // round 1, word X
        B = Y1 ^ k.k0[1];
        const uint32_t Z2 = (uint32_t)(q0 >> 32) ^ W1 ^ k.k1[1];
        const uint32_t W2 = (uint32_t)q0;
        const uint64_t r1 = (uint64_t)0xCD9E8D57u * Z2;       // round 2, word Z
        F = (uint32_t)(r1 >> 32) ^ k.k0[2];
        Y3 = (uint32_t)r1;
        G = W2 ^ k.k1[2];
    }

    __device__ __forceinline__ uint4 block(uint32_t d, const PhiloxKey& k) const { return block_z(A ^ d, k); }

    // the block whose first-round word Z1 = A ^ d is given (A depends on the
    // first counter word only)
    __device__ __forceinline__ uint4 block_z(uint32_t Z1, const PhiloxKey& k) const
    {
        const uint64_t q1 = (uint64_t)0xCD9E8D57u * Z1;       // round 1, word Z
        const uint32_t X2 = (uint32_t)(q1 >> 32) ^ B;
        const uint32_t Y2 = (uint32_t)q1;
        const uint64_t r0 = (uint64_t)0xD2511F53u * X2;       // round 2, word X
        uint4 c = make_uint4(Y2 ^ F, Y3, (uint32_t)(r0 >> 32) ^ G, (uint32_t)r0);
#pragma unroll
        for (int r = 3; r < 10; ++r) {
            const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
            const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
            c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.k1[r],
                           (uint32_t)p0);
        }
        return c;
    }
};

// Counter layout of the random streams used by the step (fourth word tags).
constexpr uint32_t kTagMid = 0x20000000u;    // bits 23..16 of a pair's uniform
constexpr uint32_t kTagFine = 0x40000000u;   // low 16 bits of a pair's uniform
constexpr uint32_t kTagAngle = 0x80000000u;  // centre-of-mass direction
constexpr uint32_t kTagSkip = 0xC0000000u;   // skip-ahead: k-th candidate draw of a row
constexpr uint32_t kTagMass = 0x40000000u;   // sampling (first word kStepInit): massive momentum, try k
constexpr uint32_t kStepInit = 0xFFFFFFFFu;  // first word reserved for sampling

}  // namespace cuba
