// philox.cuh -- Philox4x32-10 counter-based generator for the sm_103a kernels.
//
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): each of the 10 rounds multiplies counter words 0 and 2 by two odd
// 32-bit constants; the high halves, xored with the other two words and the
// round key, and the low halves form the next counter; the two key words
// advance by Weyl increments between rounds.  The key of every stream here
// is the simulation seed, so the round keys are warp-uniform.
#pragma once

#include <cstdint>

namespace bitssa {

struct PhiloxKey {
  uint32_t lo, hi;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, PhiloxKey key) {
  uint32_t k0 = key.lo, k1 = key.hi;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const unsigned long long wide_a = (unsigned long long)x.x * 0xD2511F53ull;
    const unsigned long long wide_b = (unsigned long long)x.z * 0xCD9E8D57ull;
    const uint32_t hi_a = (uint32_t)(wide_a >> 32), lo_a = (uint32_t)wide_a;
    const uint32_t hi_b = (uint32_t)(wide_b >> 32), lo_b = (uint32_t)wide_b;
    x = make_uint4(hi_b ^ x.y ^ k0, lo_b, hi_a ^ x.w ^ k1, lo_a);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return x;
}

// Counter of call `call` of the (group, step, attempt, tag) stream:
// (group, step lo 32, step hi 16 | attempt << 16 | tag << 24, call).
__device__ __forceinline__ uint4 stream_counter(uint32_t group, unsigned long long step,
                                                uint32_t attempt, uint32_t tag, uint32_t call) {
  return make_uint4(group, (uint32_t)step,
                    ((uint32_t)(step >> 32) & 0xFFFFu) | (attempt << 16) | (tag << 24), call);
}

}  // namespace bitssa
