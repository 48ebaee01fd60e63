// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds, each
// two 32x32->64-bit products of counter words 0 and 2 with fixed
// multipliers, the high halves xor-ed with the other counter words and the
// round key, the key advanced by a Weyl increment after every round.
//
// The sweep kernels fold the rounds whose inputs do not change from one
// proposal to the next (the spin, quad and start words of the counter are
// fixed for a work item; only the sweep word moves) and call philox_rounds for
// the rest; every form computes the same words as philox4x32_10.
#pragma once
#include <stdint.h>

namespace spvar {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;  // round multipliers
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;  // key increments

// (hi, lo) of the 64-bit product of a round multiplier and a counter word.
__device__ __forceinline__ void philox_mulhilo(uint32_t m, uint32_t a, uint32_t &hi, uint32_t &lo)
{
    const uint64_t p = (uint64_t)m * a;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

// One round with that round's keys.
__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t rk0, uint32_t rk1)
{
    uint32_t h0, l0, h1, l1;
    philox_mulhilo(kPhiloxM0, c.x, h0, l0);
    philox_mulhilo(kPhiloxM1, c.z, h1, l1);
    return make_uint4(h1 ^ c.y ^ rk0, l1, h0 ^ c.w ^ rk1, l0);
}

// Keys of rounds R0 .. 9 of one seed (round r: k0 + r W0, k1 + r W1).
template <int R0>
struct PhiloxKeys {
    uint32_t k0[10 - R0], k1[10 - R0];
};

template <int R0>
__device__ __forceinline__ PhiloxKeys<R0> philox_keys(uint32_t k0, uint32_t k1)
{
    PhiloxKeys<R0> K;
#pragma unroll
    for (int r = R0; r < 10; ++r) {
        K.k0[r - R0] = k0 + (uint32_t)r * kPhiloxW0;
        K.k1[r - R0] = k1 + (uint32_t)r * kPhiloxW1;
    }
    return K;
}

// Rounds R0 .. 9 applied to the counter state after round R0 - 1, with keys
// starting at round KR0 <= R0.
template <int R0, int KR0>
__device__ __forceinline__ uint4 philox_rounds(uint4 c, const PhiloxKeys<KR0> &K)
{
    static_assert(KR0 <= R0 && R0 <= 10, "round range");
#pragma unroll
    for (int r = R0; r < 10; ++r) c = philox_round(c, K.k0[r - KR0], K.k1[r - KR0]);
    return c;
}

// The whole generator: counter c, key (k0, k1).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        c = philox_round(c, k0, k1);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

}  // namespace spvar
