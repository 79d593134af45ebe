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

// Calls call0, call0 + stride, ... (NC of them) of one stream (counters that differ only in
// the last word), rounds outermost so that the NC independent chains are interleaved in
// program order.
template <int NC>
__device__ __forceinline__ void philox4x32_10_block(uint32_t (&w)[4 * NC], uint4 ctr, uint32_t call0,
                                                    PhiloxKey key, uint32_t stride = 1u) {
  uint32_t x0[NC], x1[NC], x2[NC], x3[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    x0[c] = ctr.x;
    x1[c] = ctr.y;
    x2[c] = ctr.z;
    x3[c] = call0 + stride * (uint32_t)c;
  }
  uint32_t k0 = key.lo, k1 = key.hi;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const unsigned long long wide_a = (unsigned long long)x0[c] * 0xD2511F53ull;
      const unsigned long long wide_b = (unsigned long long)x2[c] * 0xCD9E8D57ull;
      const uint32_t n0 = (uint32_t)(wide_b >> 32) ^ x1[c] ^ k0;
      const uint32_t n2 = (uint32_t)(wide_a >> 32) ^ x3[c] ^ k1;
      x1[c] = (uint32_t)wide_b;
      x3[c] = (uint32_t)wide_a;
      x0[c] = n0;
      x2[c] = n2;
    }
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    w[4 * c + 0] = x0[c];
    w[4 * c + 1] = x1[c];
    w[4 * c + 2] = x2[c];
    w[4 * c + 3] = x3[c];
  }
}

// Counter of call `call` of the (group, step, attempt, tag) stream:
// (group, step lo 32, step hi 16 | attempt << 16 | tag << 24, call).
__device__ __forceinline__ uint4 stream_counter(uint32_t group, unsigned long long step,
                                                uint32_t attempt, uint32_t tag, uint32_t call) {
  return make_uint4(group, (uint32_t)step,
                    ((uint32_t)(step >> 32) & 0xFFFFu) | (attempt << 16) | (tag << 24), call);
}

}  // namespace bitssa
