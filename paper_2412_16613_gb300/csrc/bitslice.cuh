// bitslice.cuh -- bit-sliced integer arithmetic on plane arrays (sm_103a).
//
// A bit-sliced integer of W planes is uint32_t x[W]; plane i holds bit i of
// 32 independent integers, one per lane (Sec. 4, Eqs. eq4 and eq6).  Every
// routine below works on all 32 lanes at once with word-wide logic; plane
// counts are compile-time so that loops unroll and the planes stay in
// registers.  The compiler maps each 2- or 3-input expression to one LOP3.
//
// Signed values are two's complement over their W planes; reading a signed
// operand beyond its width repeats its top plane (sign extension), reading an
// unsigned one beyond its width gives 0.
#pragma once

#include <cstdint>

namespace bitssa {
namespace bs {

// Full-adder carry (majority) and sum.  Sec. 4.1 prints the carry as
// (b2 & (b1 | c)) | (b1 & c) -- the majority -- and the partial sum must be the
// three-way xor (the printed "b1 & b2" cannot produce the paper's own Fig. 1).
__device__ __forceinline__ uint32_t maj(uint32_t a, uint32_t b, uint32_t c) {
  return (a & b) | (c & (a | b));
}
__device__ __forceinline__ uint32_t xor3(uint32_t a, uint32_t b, uint32_t c) { return a ^ b ^ c; }

// Plane i of an operand: SIGNED -> sign-extended, else zero-extended.
template <bool SIGNED, int W>
__device__ __forceinline__ uint32_t plane(const uint32_t (&x)[W], int i) {
  return i < W ? x[i] : (SIGNED ? x[W - 1] : 0u);
}

// Bit i of a compile-time integer constant, as a lane mask m or 0 (two's complement).
template <long long C>
__device__ __forceinline__ uint32_t cbit(int i, uint32_t m) {
  return ((unsigned long long)C >> (i < 63 ? i : 63)) & 1ull ? m : 0u;
}

// x += c, where lane l adds C1 if m1 has bit l, C2 if m2, C3 if m3 (masks disjoint),
// all in W-plane two's complement (Eq. equation-v: N -> N + [xi & nu_r]).
template <long long C1, long long C2, long long C3, int W>
__device__ __forceinline__ void add_select3(uint32_t (&x)[W], uint32_t m1, uint32_t m2, uint32_t m3) {
  uint32_t carry = 0u;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    const uint32_t a = cbit<C1>(i, m1) | cbit<C2>(i, m2) | cbit<C3>(i, m3);
    const uint32_t s = xor3(x[i], a, carry);
    if (i + 1 < W) carry = maj(x[i], a, carry);
    x[i] = s;
  }
}

// S (KW planes) += T (TW planes, signed) + cin, modulo 2^KW.
template <int KW, int TW>
__device__ __forceinline__ void add_signed(uint32_t (&S)[KW], const uint32_t (&T)[TW], uint32_t cin) {
  uint32_t carry = cin;
#pragma unroll
  for (int i = 0; i < KW; ++i) {
    const uint32_t t = plane<true>(T, i);
    const uint32_t s = xor3(S[i], t, carry);
    if (i + 1 < KW) carry = maj(S[i], t, carry);
    S[i] = s;
  }
}

// Lanes where n < S, both unsigned: the borrow out of n - S (Sec. 4 step c:
// the comparison word [m <= n] is the complement of [n < m]).
template <int KW>
__device__ __forceinline__ uint32_t less_than(const uint32_t (&n)[KW], const uint32_t (&S)[KW]) {
  uint32_t borrow = 0u;
#pragma unroll
  for (int i = 0; i < KW; ++i) borrow = maj(~n[i], S[i], borrow);
  return borrow;
}

// Lanes where n < C for an integer C shared by all lanes.
template <int KW>
__device__ __forceinline__ uint32_t less_than_const(const uint32_t (&n)[KW], uint32_t C) {
  uint32_t borrow = 0u;
#pragma unroll
  for (int i = 0; i < KW; ++i) {
    const uint32_t c = 0u - ((C >> i) & 1u);
    borrow = maj(~n[i], c, borrow);
  }
  return borrow;
}

// Lanes whose value is not zero.
template <int KW>
__device__ __forceinline__ uint32_t nonzero(const uint32_t (&x)[KW]) {
  uint32_t acc = 0u;
#pragma unroll
  for (int i = 0; i < KW; ++i) acc |= x[i];
  return acc;
}

// Lanes where x != y.
template <int KW>
__device__ __forceinline__ uint32_t differ(const uint32_t (&x)[KW], const uint32_t (&y)[KW]) {
  uint32_t acc = 0u;
#pragma unroll
  for (int i = 0; i < KW; ++i) acc |= x[i] ^ y[i];
  return acc;
}

// Schoolbook product of two unsigned bit-sliced integers, truncated to RW planes
// (the O(N_2^2) multiplication of Sec. 4.1; used once per group to build the
// initial propensities).
template <int RW, int XW, int YW>
__device__ __forceinline__ void multiply(uint32_t (&out)[RW], const uint32_t (&x)[XW],
                                         const uint32_t (&y)[YW]) {
#pragma unroll
  for (int i = 0; i < RW; ++i) out[i] = 0u;
#pragma unroll
  for (int j = 0; j < YW; ++j) {
    uint32_t carry = 0u;
#pragma unroll
    for (int i = 0; i < XW; ++i) {
      if (i + j < RW) {
        const uint32_t t = x[i] & y[j];
        const uint32_t s = xor3(out[i + j], t, carry);
        carry = maj(out[i + j], t, carry);
        out[i + j] = s;
      }
    }
    // the partial sum of rows 0..j fits in XW + j + 1 bits, so the carry lands in a zero plane
    if (XW + j < RW) out[XW + j] = carry;
  }
}

// acc += x * y (unsigned), modulo 2^RW: each row of the schoolbook product is rippled into acc.
template <int RW, int XW, int YW>
__device__ __forceinline__ void multiply_add(uint32_t (&acc)[RW], const uint32_t (&x)[XW],
                                             const uint32_t (&y)[YW]) {
#pragma unroll
  for (int j = 0; j < YW; ++j) {
    uint32_t carry = 0u;
#pragma unroll
    for (int i = j; i < RW; ++i) {
      const uint32_t t = (i - j < XW) ? (x[i - j] & y[j]) : 0u;
      const uint32_t s = xor3(acc[i], t, carry);
      carry = maj(acc[i], t, carry);
      acc[i] = s;
    }
  }
}

// Value of one lane, sign-extended from W planes when SIGNED.
template <bool SIGNED, int W>
__device__ __forceinline__ long long lane_value(const uint32_t (&x)[W], int lane) {
  long long v = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) v |= (long long)((x[i] >> lane) & 1u) << i;
  if (SIGNED && ((x[W - 1] >> lane) & 1u)) v -= (1ll << W);
  return v;
}

// Planes of one lane value set into x (other lanes untouched).
template <int W>
__device__ __forceinline__ void set_lane(uint32_t (&x)[W], int lane, long long v) {
  const uint32_t bit = 1u << lane;
#pragma unroll
  for (int i = 0; i < W; ++i) x[i] = ((v >> i) & 1) ? (x[i] | bit) : (x[i] & ~bit);
}

// All lanes equal to the constant v.
template <int W>
__device__ __forceinline__ void broadcast(uint32_t (&x)[W], long long v) {
#pragma unroll
  for (int i = 0; i < W; ++i) x[i] = ((v >> (i < 63 ? i : 63)) & 1) ? 0xFFFFFFFFu : 0u;
}

}  // namespace bs
}  // namespace bitssa
