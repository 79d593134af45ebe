// frank_kernel.cuh -- the bit-sliced Gillespie step loop for Frank's model on sm_103a.
//
// One thread owns one group of 32 runs (lane l of every plane is run 32 g + l)
// and keeps the whole group state in registers:
//   L                 the L count (B planes, Eq. eq4)
//   S1, S2, S3        cumulative integer propensities S_r = sum_{p<=r} h_p with
//                     h1 = A L, h2 = A D, h3 = L D (Eq. equation-as), K planes
//   P, U, R1, R3      signed linear forms of the counts; with Q = U + L and
//                     U3 = -U - 3 (one ripple each, per step) they are exactly
//                     the increments of S1..S3 for each reaction (App. A / B):
//                       dS1 = P | -L | R1,  dS2 = U | U | 2 U3,  dS3 = P | Q | R3
//                     for reactions 1 | 2 | 3, with P = A-L-1, Q = A-D-1,
//                     U = A-L-D-1, R1 = 2L-A-2, R3 = L+D-2A-3 in the counts
//                     before the reaction (the App. A right-hand sides).  The
//                     kept forms change by per-reaction constants, so each is
//                     updated with one masked constant add per step.
// D and A are read back from L and U (U = N - 2(L+D) - 1) when a snapshot or
// an output needs them.
//
// One group step (Sec. 3, steps 1-7, with the draw of step 5 done by Sec. 4's steps a-d):
//   1. Philox words of attempt 0: planes of the uniform integer n and the
//      group's waiting-time bits; lanes with n >= lambda_int redraw from the
//      next attempt.  With the state-following bound (template flag ADAPT) the
//      step's bound is 2^p, p the highest plane set in S3 over the live lanes,
//      and n keeps its low p planes: nothing is redrawn.
//   2. Clock: tau ~ Exp(Lambda) (Eq. equation-tau), Lambda = k_max 2^p under
//      ADAPT.  Snapshots whose time is passed record the state before the event;
//      passing t_end stops the group.  With per-run clocks (template flag LANE) every
//      run draws its own tau, keeps its own snapshots, and stops alone at t_end.
//   3. Comparators lt_r = [n < S_r] (borrow chains) and changer words
//      xi_r = lt_r & ~lt_{r-1} (Eq. equation-changer: the CDF walk of Fig. 2
//      done for all lanes at once); lanes with n >= S_3 fire a ghost reaction.
//   4. Non-unit rates: thinning against q-bit thresholds, most significant
//      bit first, stopping as soon as every lane is decided.
//   5. Masked updates of S1..S3 and of the linear forms (Eqs. equation-v,
//      equation-a-1..3).
//   6. Absorption: a lane whose reactions with k_r > 0 all have h_r = 0 stops.
#pragma once

#include <cstdint>

#include "bitslice.cuh"
#include "internal.h"
#include "philox.cuh"

namespace bitssa {


template <int K>
struct FrankShape {
  static constexpr int B = bit_length(frank_nmax(K));  // count planes
  static constexpr int WP = B + 1;                      // P, Q, U in [-N-1, N-1]
  static constexpr int WU3 = B + 2;                     // U3 in [-N-2, N-2]
  static constexpr int WR1 = B + 2;                     // R1 in [-N-2, 2N-2]
  static constexpr int WR3 = B + 3;                     // R3 in [-2N-3, N-3]
  static constexpr int NC0 = (K + 2 + 3) / 4;           // Philox calls for n and tau
  static constexpr int NCR = (K + 3) / 4;               // Philox calls for a redraw of n
};

constexpr double kLn2 = 0x1.62e42fefa39efp-1;  // ln 2 rounded to double


// Reads the (L, D, A) of one lane from the L and U planes: X = L + D = (N - 1 - U) / 2.
template <int B, int WP>
__device__ __forceinline__ void lane_counts(const uint32_t (&L)[B], const uint32_t (&U)[WP], int n_tot,
                                            int lane, int& l, int& d, int& a) {
  l = (int)bs::lane_value<false>(L, lane);
  const int u = (int)bs::lane_value<true>(U, lane);
  const int x = (n_tot - 1 - u) / 2;
  d = x - l;
  a = n_tot - x;
}

__device__ __forceinline__ int ee_bin(int l, int d) {
  if (l + d == 0) return 64;
  const int b = (64 * l) / (l + d);
  return b > 63 ? 63 : b;
}

// ---------------------------------------------------------------------------
// The group clock.  PROD (SSA_P64): exp(-Lambda t) = M 2^(E - 63) is kept as a
// 64-bit fixed-point mantissa M in [2^63, 2^64) and an integer exponent E; each
// step multiplies in the step's uniform u with integer instructions only (GB300's
// fp64 rate is 1/64 of its fp32 rate), so t = -(ln M + (E - 63) ln 2) / Lambda needs
// a logarithm only when a time is written out.  Otherwise: the fp64 sum of -log(u) / Lambda (SSA_P64_LOGSUM), or
// fp32 -logf(u) / Lambda summed with Kahan compensation (SSA_P32_KAHAN), into an
// fp64 accumulator (SSA_P32_D64ACC) or plainly in fp32 (SSA_P32_PLAIN).
// ---------------------------------------------------------------------------
template <bool PROD>
struct Clock;

template <>
struct Clock<true> {
  unsigned long long M;  // exp(-Lambda t) = M 2^(E - 63), M in [2^63, 2^64)
  long long E;
  long long th_E;                 // exponent of the next time point to cross
  const unsigned long long* th_M; // its mantissa, read only when the exponents tie
  __device__ __forceinline__ void reset() {
    M = 1ull << 63;
    E = 0;
  }
  __device__ __forceinline__ void aim(const Threshold& h) {
    th_E = h.E;
    th_M = &h.M;
  }
  __device__ __forceinline__ double time(const Ensemble& e, int) const {
    return -(log((double)M) + (double)(E - 63) * kLn2) / e.lambda;
  }
};

template <>
struct Clock<false> {
  double t;
  float t_f, c_f;
  double th_t;
  float th_f;
  __device__ __forceinline__ void reset() {
    t = 0.0;
    t_f = c_f = 0.0f;
  }
  __device__ __forceinline__ void aim(const Threshold& h) {
    th_t = h.t;
    th_f = h.t_f;
  }
  __device__ __forceinline__ double time(const Ensemble&, int precision) const {
    return (precision == kP32Kahan || precision == kP32Plain) ? (double)t_f : t;
  }
};

// Candidate clock after this step's event, from the step's waiting-time words w_K, w_{K+1}.
// Product clock: u = v 2^-53 with v = x + 1 in [1, 2^53]; the 117-bit product M v is
// renormalised to its top 64 bits in integer arithmetic (truncation: relative error below
// 2^-63 per step, far under the fp64 rounding of the summed time it stands for).
__device__ __forceinline__ bool clock_advance(const Clock<true>& c, Clock<true>& nx, uint32_t wk, uint32_t wk1,
                                              const Ensemble&, int) {
  const unsigned long long v = (((unsigned long long)wk1 << 21) | (wk >> 11)) + 1ull;
  const unsigned long long lo = c.M * v, hi = __umul64hi(c.M, v);
  nx = c;
  if (hi) {
    const int lz = __clzll((long long)hi);
    nx.M = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
    nx.E = c.E + 11 - lz;
  } else {  // v == 1: M v = M already has its top bit set
    nx.M = lo;
    nx.E = c.E - 53;
  }
  return nx.E < c.th_E || (nx.E == c.th_E && nx.M < *c.th_M);
}

// A step at the state-following bound's rate Lambda 2^-j (j = K - p) multiplies exp(-Lambda t)
// by u^(2^j): v is normalised to a 64-bit mantissa and squared j times, each square truncated
// to its top 64 bits (relative error below 2^-63 a square, doubling with each further square:
// 2^(j-62) in -ln of the factor, that is 2^-62 of the step's mean waiting time 2^j / Lambda).
__device__ __forceinline__ bool clock_advance(const Clock<true>& c, Clock<true>& nx, uint32_t wk, uint32_t wk1,
                                              const Ensemble& e, int precision, int j) {
  if (j == 0) return clock_advance(c, nx, wk, wk1, e, precision);
  const unsigned long long v = (((unsigned long long)wk1 << 21) | (wk >> 11)) + 1ull;
  const int lz0 = __clzll((long long)v);
  unsigned long long m = v << lz0;  // u = m 2^(f - 63)
  long long f = 10 - lz0;
  for (int k = 0; k < j; ++k) {
    const unsigned long long hi = __umul64hi(m, m), lo = m * m;
    if (hi >> 63) {
      m = hi;
      f = 2 * f + 1;
    } else {
      m = (hi << 1) | (lo >> 63);
      f = 2 * f;
    }
  }
  const unsigned long long hi = __umul64hi(c.M, m), lo = c.M * m;
  nx = c;
  if (hi >> 63) {
    nx.M = hi;
    nx.E = c.E + f + 1;
  } else {
    nx.M = (hi << 1) | (lo >> 63);
    nx.E = c.E + f;
  }
  return nx.E < c.th_E || (nx.E == c.th_E && nx.M < *c.th_M);
}

// The other clocks at rate Lambda 2^-j: the waiting time at rate Lambda times 2^j, which is
// exactly the waiting time at the lower rate (a power-of-two scaling rounds the same way).
__device__ __forceinline__ bool clock_advance(const Clock<false>& c, Clock<false>& nx, uint32_t wk, uint32_t wk1,
                                              const Ensemble& e, int precision, int j = 0) {
  nx = c;
  if (precision == kP64LogSum) {
    const unsigned long long x = ((unsigned long long)wk1 << 21) | (wk >> 11);
    const double u = (double)(x + 1ull) * 0x1p-53;
    nx.t = c.t + (-log(u) / e.lambda) * (double)(1ull << j);
    return nx.t > c.th_t;
  }
  const float u = (float)((wk1 >> 8) + 1u) * 0x1p-24f;  // the top 24 of the 53 bits
  const float tau = -logf(u) * e.inv_lambda_f * (float)(1u << j);
  if (precision == kP32Kahan) {
    const float y = tau - c.c_f;
    const float sum = c.t_f + y;
    nx.c_f = (sum - c.t_f) - y;
    nx.t_f = sum;
    return sum > c.th_f;
  }
  if (precision == kP32Plain) {
    nx.t_f = c.t_f + tau;
    return nx.t_f > c.th_f;
  }
  nx.t = c.t + (double)tau;
  return nx.t > c.th_t;
}

__device__ __forceinline__ bool clock_crosses(const Clock<true>& nx) {
  return nx.E < nx.th_E || (nx.E == nx.th_E && nx.M < *nx.th_M);
}
__device__ __forceinline__ bool clock_crosses(const Clock<false>& nx, int precision) {
  return (precision == kP32Kahan || precision == kP32Plain) ? nx.t_f > nx.th_f : nx.t > nx.th_t;
}

// Thinning (k_r < k_max, step (4) below): a drawn reaction is kept iff the q-bit uniform U is
// below T_r.  U is read most significant bit first, from words W0..W1-1 of the step's block
// (`word_at(k)`) and then from further calls of the same stream from call `next_call` on,
// stopping once every lane is decided.
template <int W0, int W1, typename WordAt>
__device__ __forceinline__ void thin_step(const Ensemble& e, WordAt word_at, uint32_t live, uint32_t sgroup,
                                          unsigned long long step, uint32_t next_call, PhiloxKey key,
                                          uint32_t& x1, uint32_t& x2, uint32_t& x3) {
  const uint32_t alw1 = (e.thin_always & 1u) ? ~0u : 0u;
  const uint32_t alw2 = (e.thin_always & 2u) ? ~0u : 0u;
  const uint32_t alw3 = (e.thin_always & 4u) ? ~0u : 0u;
  const uint32_t tested = (x1 & ~alw1) | (x2 & ~alw2) | (x3 & ~alw3);
  uint32_t und = tested & live;
  uint32_t rej = tested & ~live;
  const int q = e.thin_bits;
  auto bit = [&](int i, uint32_t word) {
    const int pos = q - 1 - i;
    const uint32_t b1 = 0u - (uint32_t)(((unsigned long long)e.thin_T[0] >> pos) & 1ull);
    const uint32_t b2 = 0u - (uint32_t)(((unsigned long long)e.thin_T[1] >> pos) & 1ull);
    const uint32_t b3 = 0u - (uint32_t)(((unsigned long long)e.thin_T[2] >> pos) & 1ull);
    const uint32_t tb = (x1 & b1) | (x2 & b2) | (x3 & b3);
    const uint32_t lower = und & ~word & tb;   // U < T decided
    const uint32_t higher = und & word & ~tb;  // U > T decided
    rej |= higher;
    und &= ~(lower | higher);
  };
#pragma unroll
  for (int k = W0; k < W1; ++k)
    if (k - W0 < q) bit(k - W0, word_at(k));
  int i = W1 - W0;
  for (uint32_t c = next_call; und != 0u && i < q; ++c) {
    const uint4 r = philox4x32_10(stream_counter(sgroup, step, 0u, 0u, c), key);
    const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (i < q) bit(i++, wv[j]);
  }
  rej |= und;  // U == T: not below
  x1 &= ~rej;
  x2 &= ~rej;
  x3 &= ~rej;
}

// The redraw of the lanes in `need` (those with n >= lambda_int).  A lane replaces its planes
// from p up, p the highest plane where n and lambda_int differ (every plane when they are
// equal), with the same planes of the next attempt; the planes below p are independent of the
// rejection and stay.  Planes are visited from the top: `above` collects the lanes that differ
// above the current plane.  Every call of an attempt is made: a warp takes this path whenever
// one of its runs is rejected, and the interleaved calls cost little more than one.  Returns
// false after 64 attempts.
template <int K>
__device__ __forceinline__ bool redraw_n(uint32_t (&n)[K], const Ensemble& e, uint32_t sgroup,
                                         unsigned long long step, uint32_t need, PhiloxKey key,
                                         unsigned int& redraws) {
  constexpr int NCR = FrankShape<K>::NCR;
  for (uint32_t attempt = 1u; need; ++attempt) {
    if (attempt >= 64u) return false;
    ++redraws;
    uint32_t above = 0u;
    if constexpr (K >= 25) {
      // wide n: the calls from the top, two at a time, while some lane replaces a lower plane
#pragma unroll
      for (int c = NCR - 1; c >= 0; c -= 2) {
        if (need & ~above) {
          constexpr int kPair = 2;
          const int lo = c > 0 ? c - 1 : 0;
          uint32_t wr[4 * kPair];
          philox4x32_10_block<kPair>(wr, stream_counter(sgroup, step, attempt, 0u, 0u), (uint32_t)lo, key);
#pragma unroll
          for (int j = 4 * kPair - 1; j >= 0; --j) {
            const int i = 4 * lo + j;
            if (i <= 4 * c + 3 && i < K) {
              const uint32_t m = need & ~above;
              above |= n[i] ^ (0u - ((e.lambda_int >> i) & 1u));
              n[i] = (n[i] & ~m) | (wr[j] & m);
            }
          }
        }
      }
    } else {
      uint32_t wr[4 * NCR];  // all calls of the attempt at once: their chains interleave
      philox4x32_10_block<NCR>(wr, stream_counter(sgroup, step, attempt, 0u, 0u), 0u, key);
#pragma unroll
      for (int i = K - 1; i >= 0; --i) {
        const uint32_t m = need & ~above;
        above |= n[i] ^ (0u - ((e.lambda_int >> i) & 1u));
        n[i] = (n[i] & ~m) | (wr[i] & m);
      }
    }
    need &= ~bs::less_than_const(n, e.lambda_int);
  }
  return true;
}

// Lanes (among `live`) whose n is at or above lambda_int.  n >= lambda_int needs every plane of
// lambda_int's leading run of ones set in n: that is tested first (a shallow AND tree), and the
// full comparison runs only when some lane passes.  A bound padded to 2^K rejects nothing.
template <int K>
__device__ __forceinline__ uint32_t rejected_lanes(const uint32_t (&n)[K], const Ensemble& e, uint32_t live) {
  if (!e.reject) return 0u;
  uint32_t a[K];
#pragma unroll
  for (int i = 0; i < K; ++i) a[i] = n[i] | e.top_mask[i];
#pragma unroll
  for (int width = K; width > 1; width = (width + 2) / 3) {
#pragma unroll
    for (int j = 0; j < (width + 2) / 3; ++j)
      a[j] = a[3 * j] & (3 * j + 1 < width ? a[3 * j + 1] : 0xFFFFFFFFu) &
             (3 * j + 2 < width ? a[3 * j + 2] : 0xFFFFFFFFu);
  }
  return (a[0] & live) ? ~bs::less_than_const(n, e.lambda_int) & live : 0u;
}

// Everything one thread keeps about its group between steps (all in registers).
template <int K, bool PROD>
struct GroupState {
  uint32_t S1[K], S2[K], S3[K];
  uint32_t L[FrankShape<K>::B], P[FrankShape<K>::WP], U[FrankShape<K>::WP];
  uint32_t R1[FrankShape<K>::WR1], R3[FrankShape<K>::WR3];
  uint32_t live;     // lanes that can still react
  uint32_t stopped;  // per-run clock: lanes stopped at t_end (they cannot react any more either)
  uint32_t sgroup;   // stream group index
  int nvalid;        // lanes holding a run (the last group may be partial)
  int ens;           // ensemble index
  int snap;          // next snapshot
  unsigned long long step;
  Clock<PROD> clk;
  unsigned long long reactions, lane_steps;
  unsigned int redraws;
  bool done;
};

// Output row of lane 0 of the group.
template <int K, bool PROD>
__device__ __forceinline__ long long group_row0(const GroupState<K, PROD>& s, const Ensemble& e) {
  return e.run_offset + ((long long)s.sgroup - e.group_base) * 32;
}

template <int K, bool PROD>
__device__ __forceinline__ uint32_t live_lanes(const GroupState<K, PROD>& s, const Ensemble& e) {
  if (e.active == 7u) return bs::nonzero(s.S3);
  uint32_t m = 0u;
  if (e.active & 1u) m |= bs::nonzero(s.S1);
  if (e.active & 2u) m |= bs::differ(s.S2, s.S1);
  if (e.active & 4u) m |= bs::differ(s.S3, s.S2);
  return m;
}

// Dynamic shared memory of the one-thread kernel: the histogram of a single ensemble, then the
// per-thread staging rows of the snapshot dump.
extern __shared__ unsigned int frank_dyn_smem[];

// The current state of every valid lane into snapshot `snap`: histogram and per-run counts.
// With the dump on, a full group's 32 rows of 3 counts (384 contiguous bytes of the output) are
// staged in this thread's shared-memory rows and written with 24 16-byte stores; a partial group,
// or an output not 16-byte aligned, is written count by count.
template <int K, bool PROD>
__device__ __forceinline__ void capture(const FrankLaunch& p, const GroupState<K, PROD>& s, const Ensemble& e,
                                        int snap, unsigned int* s_hist) {
  using Sh = FrankShape<K>;
  int* const rows = p.snap_counts ? p.snap_counts + ((long long)snap * p.n_runs_total + group_row0(s, e)) * 3 : nullptr;
  const bool staged = rows && p.stage_offset >= 0 && s.nvalid == 32 && p.n_species == 3 &&
                      (reinterpret_cast<uintptr_t>(rows) & 15u) == 0u;
  unsigned int* const buf = frank_dyn_smem + p.stage_offset + threadIdx.x * kStageStride;
  for (int l = 0; l < s.nvalid; ++l) {
    int cl, cd, ca;
    lane_counts<Sh::B, Sh::WP>(s.L, s.U, e.n_tot, l, cl, cd, ca);
    if (s_hist) atomicAdd(&s_hist[snap * kHistBins + ee_bin(cl, cd)], 1u);
    else atomicAdd(&p.hist[((long long)s.ens * p.n_snap + snap) * kHistBins + ee_bin(cl, cd)], 1ull);
    if (staged) {
      buf[3 * l + p.perm[0]] = (unsigned int)cl;
      buf[3 * l + p.perm[1]] = (unsigned int)cd;
      buf[3 * l + p.perm[2]] = (unsigned int)ca;
    } else if (rows) {
      int* o = rows + l * p.n_species;
      o[p.perm[0]] = cl;
      o[p.perm[1]] = cd;
      o[p.perm[2]] = ca;
    }
  }
  if (staged) {
    const uint4* src = reinterpret_cast<const uint4*>(buf);
    uint4* dst = reinterpret_cast<uint4*>(rows);
#pragma unroll 4
    for (int k = 0; k < 24; ++k) dst[k] = src[k];
  }
}

// ---------------------------------------------------------------------------
// Per-run clocks (SSA_CLOCK_LANE).  Each run of a group has its own clock, kept in dynamic shared
// memory from word p.lane_offset: a 16-byte record per run laid out [lane][thread] (a warp reads
// 32 consecutive records), holding the product clock's mantissa and exponent, or the fp64 time and
// the fp32 time with its compensation; then a byte per run, [lane][thread], with the index of its
// next time point (snapshot, or t_end).  Run j's waiting time at step s comes from words 0 and 1
// of its own Philox stream, counter (j lo 32, s lo 32, s hi 16 | (j >> 32) << 16 | 1 << 24, 0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4* lane_record(const FrankLaunch& p, int lane) {
  return reinterpret_cast<uint4*>(frank_dyn_smem + p.lane_offset) + lane * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ unsigned char* lane_next(const FrankLaunch& p, int lane) {
  return reinterpret_cast<unsigned char*>(frank_dyn_smem + p.lane_offset + 4 * 32 * blockDim.x) +
         lane * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ uint4 pack_clock(const Clock<true>& c) {
  return make_uint4((uint32_t)c.M, (uint32_t)(c.M >> 32), (uint32_t)c.E, (uint32_t)((unsigned long long)c.E >> 32));
}
__device__ __forceinline__ void unpack_clock(Clock<true>& c, uint4 r) {
  c.M = ((unsigned long long)r.y << 32) | r.x;
  c.E = (long long)(((unsigned long long)r.w << 32) | r.z);
}
__device__ __forceinline__ uint4 pack_clock(const Clock<false>& c) {
  const unsigned long long t = (unsigned long long)__double_as_longlong(c.t);
  return make_uint4((uint32_t)t, (uint32_t)(t >> 32), __float_as_uint(c.t_f), __float_as_uint(c.c_f));
}
__device__ __forceinline__ void unpack_clock(Clock<false>& c, uint4 r) {
  c.t = __longlong_as_double((long long)(((unsigned long long)r.y << 32) | r.x));
  c.t_f = __uint_as_float(r.z);
  c.c_f = __uint_as_float(r.w);
}
__device__ __forceinline__ uint4 lane_clock_counter(unsigned long long run, unsigned long long step) {
  return make_uint4((uint32_t)run, (uint32_t)step,
                    ((uint32_t)(step >> 32) & 0xFFFFu) | (((uint32_t)(run >> 32) & 0xFFu) << 16) | (1u << 24), 0u);
}

// The current state of lane l into snapshot `snap` (histogram and per-run counts).
template <int K, bool PROD>
__device__ __forceinline__ void capture_lane(const FrankLaunch& p, const GroupState<K, PROD>& s, const Ensemble& e,
                                             int snap, unsigned int* s_hist, int l) {
  using Sh = FrankShape<K>;
  int cl, cd, ca;
  lane_counts<Sh::B, Sh::WP>(s.L, s.U, e.n_tot, l, cl, cd, ca);
  if (s_hist) atomicAdd(&s_hist[snap * kHistBins + ee_bin(cl, cd)], 1u);
  else atomicAdd(&p.hist[((long long)s.ens * p.n_snap + snap) * kHistBins + ee_bin(cl, cd)], 1ull);
  if (p.snap_counts) {
    int* o = p.snap_counts + ((long long)snap * p.n_runs_total + group_row0(s, e) + l) * p.n_species;
    o[p.perm[0]] = cl;
    o[p.perm[1]] = cd;
    o[p.perm[2]] = ca;
  }
}

// Set up group `group_local` of ensemble `e`: initial planes, cumulative propensities by
// bit-sliced products, the linear forms, the runs that start absorbed.
template <int K, bool PROD, bool LANE = false>
__device__ __forceinline__ void group_init(const FrankLaunch& p, GroupState<K, PROD>& s, const Ensemble& e,
                                           const Threshold* thr, long long group_local, int ens_index,
                                           unsigned int* s_hist) {
  using Sh = FrankShape<K>;
  constexpr int B = Sh::B, WP = Sh::WP, WR1 = Sh::WR1, WR3 = Sh::WR3;
  const long long run0 = group_local * 32;
  const long long left = e.n_runs - run0;
  s.nvalid = left >= 32 ? 32 : (int)left;
  const uint32_t valid = s.nvalid >= 32 ? 0xFFFFFFFFu : ((1u << s.nvalid) - 1u);
  s.sgroup = (uint32_t)(e.group_base + group_local);
  const long long row0 = e.run_offset + run0;
  s.ens = ens_index;
  const int n_tot = e.n_tot;

  // initial planes (padding lanes hold (0, 0, N): absorbed, never counted)
  uint32_t Lp[B], Dp[B], Ap[B];
  if (p.init_counts) {
    bs::broadcast(Lp, 0);
    bs::broadcast(Dp, 0);
    bs::broadcast(Ap, n_tot);
    for (int l = 0; l < s.nvalid; ++l) {
      const int* c = p.init_counts + (row0 + l) * 3;
      bs::set_lane(Lp, l, c[0]);
      bs::set_lane(Dp, l, c[1]);
      bs::set_lane(Ap, l, c[2]);
    }
  } else {
    bs::broadcast(Lp, e.init[0]);
    bs::broadcast(Dp, e.init[1]);
    bs::broadcast(Ap, e.init[2]);
#pragma unroll
    for (int i = 0; i < B; ++i) {
      Lp[i] &= valid;
      Dp[i] &= valid;
      Ap[i] = (Ap[i] & valid) | (((n_tot >> i) & 1) ? ~valid : 0u);
    }
  }
  // cumulative propensities (Eq. equation-as) by bit-sliced products
  bs::multiply(s.S1, Ap, Lp);
  bs::multiply(s.S2, Ap, Dp);
  bs::multiply_add(s.S2, Ap, Lp);  // A D + A L
#pragma unroll
  for (int i = 0; i < K; ++i) s.S3[i] = s.S2[i];
  bs::multiply_add(s.S3, Lp, Dp);  // + L D
  // the linear forms, by ripple adds of (shifted, complemented) count planes
#pragma unroll
  for (int i = 0; i < B; ++i) s.L[i] = Lp[i];
  uint32_t c = 0u;  // P = A + ~L = A - L - 1
#pragma unroll
  for (int i = 0; i < WP; ++i) {
    const uint32_t a = bs::plane<false>(Ap, i), b = ~bs::plane<false>(Lp, i);
    s.P[i] = bs::xor3(a, b, c);
    c = bs::maj(a, b, c);
  }
  c = 0xFFFFFFFFu;  // U = P + ~D + 1 = A - L - D - 1
#pragma unroll
  for (int i = 0; i < WP; ++i) {
    const uint32_t a = s.P[i], b = ~bs::plane<false>(Dp, i);
    s.U[i] = bs::xor3(a, b, c);
    c = bs::maj(a, b, c);
  }
  c = 0u;  // R1 = (L << 1) + ~A - 1 = 2L - A - 2
#pragma unroll
  for (int i = 0; i < WR1; ++i) {
    const uint32_t a = i == 0 ? 0u : bs::plane<false>(Lp, i - 1), b = ~bs::plane<false>(Ap, i);
    s.R1[i] = bs::xor3(a, b, c);
    c = bs::maj(a, b, c);
  }
  bs::add_select3<-1, -1, -1>(s.R1, 0xFFFFFFFFu, 0u, 0u);
  c = 0u;  // R3 = L + D + (~A << 1) - 1 = L + D - 2A - 3
#pragma unroll
  for (int i = 0; i < WR3; ++i) {
    const uint32_t a = bs::plane<false>(Lp, i), b = bs::plane<false>(Dp, i);
    s.R3[i] = bs::xor3(a, b, c);
    c = bs::maj(a, b, c);
  }
  c = 0u;
#pragma unroll
  for (int i = 0; i < WR3; ++i) {
    const uint32_t a = s.R3[i], b = i == 0 ? 0u : ~bs::plane<false>(Ap, i - 1);
    s.R3[i] = bs::xor3(a, b, c);
    c = bs::maj(a, b, c);
  }
  bs::add_select3<-1, -1, -1>(s.R3, 0xFFFFFFFFu, 0u, 0u);

  s.live = live_lanes(s, e) & valid;
  uint32_t at0 = valid & ~s.live;  // runs that start absorbed are absorbed at t = 0
  while (at0) {
    const int l = __ffs(at0) - 1;
    at0 &= at0 - 1;
    p.t_abs[row0 + l] = 0.0;
  }
  s.step = 0;
  s.clk.reset();
  s.snap = 0;
  s.clk.aim(thr[0]);
  s.reactions = s.lane_steps = 0;
  s.redraws = 0;
  s.stopped = 0u;
  s.done = s.live == 0u;
  if constexpr (LANE) {  // every run's clock at t = 0, aimed at the first time point
    Clock<PROD> c;
    c.reset();
    for (int l = 0; l < 32; ++l) {
      *lane_record(p, l) = pack_clock(c);
      *lane_next(p, l) = 0;
    }
  } else if (s.done) {
    for (; s.snap < p.n_snap; ++s.snap) capture<K, PROD>(p, s, e, s.snap, s_hist);
  }
}

// One group step (see the file header).  Never leaves the caller's loop: a group that
// stops sets s.done.
template <int K, bool PROD, bool ADAPT, bool LANE = false>
__device__ __forceinline__ void group_step(const FrankLaunch& p, GroupState<K, PROD>& s, const Ensemble& e,
                                           const Threshold* thr, unsigned int* s_hist, unsigned int& errors) {
  using Sh = FrankShape<K>;
  constexpr int WP = Sh::WP, WU3 = Sh::WU3, WR1 = Sh::WR1, WR3 = Sh::WR3;
  constexpr int NC0 = Sh::NC0;
  const PhiloxKey key{(uint32_t)e.seed, (uint32_t)(e.seed >> 32)};
  const int precision = p.precision;

  if (p.step_budget > 0 && (long long)s.step >= p.step_budget) {
    errors |= kErrTimeout;
    s.done = true;
    return;
  }
  // (1) the random words of attempt 0
  uint32_t w[4 * NC0];
  philox4x32_10_block<NC0>(w, stream_counter(s.sgroup, s.step, 0u, 0u, 0u), 0u, key);
  uint32_t n[K];
#pragma unroll
  for (int i = 0; i < K; ++i) n[i] = w[i];
  // the state-following bound: 2^p, p the bit length of the largest S_3 over the live lanes,
  // and n its low p planes
  int j = 0;
  if constexpr (ADAPT) {
    int bits = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) bits = (s.S3[i] & s.live) ? i + 1 : bits;
#pragma unroll
    for (int i = 0; i < K; ++i) n[i] = i < bits ? n[i] : 0u;
    j = K - bits;
  }
  // the rejection test and the three comparators are independent borrow chains: run them
  // together, and redo the comparators only in the rare step where a lane redraws
  const uint32_t need = rejected_lanes<K>(n, e, s.live);
  uint32_t lt1 = bs::less_than(n, s.S1);
  uint32_t lt2 = bs::less_than(n, s.S2);
  uint32_t lt3 = bs::less_than(n, s.S3);
  if (need) {
    if (!redraw_n<K>(n, e, s.sgroup, s.step, need, key, s.redraws)) {
      errors |= kErrRedraw;
      s.done = true;
      return;
    }
    lt1 = bs::less_than(n, s.S1);
    lt2 = bs::less_than(n, s.S2);
    lt3 = bs::less_than(n, s.S3);
  }

  // (2) the clock: the candidate time of this step's event, snapshots, t_end
  if constexpr (LANE) {
    // every live run advances its own clock; a run whose event lies beyond t_end stops
    uint32_t stop = 0u;
    const unsigned long long run0 = (unsigned long long)s.sgroup * 32u;
    for (uint32_t m = s.live; m; m &= m - 1u) {
      const int l = __ffs((int)m) - 1;
      const uint4 r = philox4x32_10(lane_clock_counter(run0 + (unsigned)l, s.step), key);
      uint4* rec = lane_record(p, l);
      unsigned char* nxt = lane_next(p, l);
      int k = *nxt;
      Clock<PROD> c, nc;
      unpack_clock(c, *rec);
      c.aim(thr[k]);
      bool crossed = clock_advance(c, nc, r.x, r.y, e, precision);
      while (crossed) {
        if (k >= p.n_snap) {  // t_end passed: the run's event is not applied
          stop |= 1u << l;
          break;
        }
        capture_lane<K, PROD>(p, s, e, k, s_hist, l);
        ++k;
        nc.aim(thr[k]);
        if constexpr (PROD) crossed = clock_crosses(nc);
        else crossed = clock_crosses(nc, precision);
      }
      *nxt = (unsigned char)k;
      if (!((stop >> l) & 1u)) *rec = pack_clock(nc);
    }
    if (stop) {
      s.lane_steps += (unsigned long long)__popc(stop) * s.step;
      s.live &= ~stop;
      s.stopped |= stop;
      if (!s.live) {
        s.done = true;
        return;
      }
    }
  } else {
    Clock<PROD> nx;
    bool crossed;
    if constexpr (ADAPT) crossed = clock_advance(s.clk, nx, w[K], w[K + 1], e, precision, j);
    else crossed = clock_advance(s.clk, nx, w[K], w[K + 1], e, precision);
    while (crossed) {
      if (s.snap >= p.n_snap) {  // t_end passed: the event is not applied
        s.done = true;
        return;
      }
      capture<K, PROD>(p, s, e, s.snap, s_hist);
      ++s.snap;
      nx.aim(thr[s.snap]);
      if constexpr (PROD) crossed = clock_crosses(nx);
      else crossed = clock_crosses(nx, precision);
    }
    s.clk = nx;
  }

  // (3) changer words: xi_r = [S_{r-1} <= n < S_r].  A lane that cannot react has S_r = 0
  // for every reaction with k_r > 0, so only reactions that thinning rejects can be picked
  // (with per-run clocks, a run stopped at t_end is masked out).
  uint32_t x1 = lt1, x2 = lt2 & ~lt1, x3 = lt3 & ~lt2;
  if constexpr (LANE) {
    x1 &= s.live;
    x2 &= s.live;
    x3 &= s.live;
  }

  // (4) thinning for k_r < k_max
  if (e.thin)
    thin_step<K + 2, 4 * NC0>(e, [&](int k) { return w[k]; }, s.live, s.sgroup, s.step, NC0, key, x1, x2, x3);

  // (5) updates from the counts before the reaction (App. B).  A step in which no lane
  // fires (frequent once most lanes of a group have absorbed) changes nothing.
  const uint32_t x12 = x1 | x2;
  const uint32_t fired = x12 | x3;
  ++s.step;
  if (!fired) return;
  {
    uint32_t T[WR1];
#pragma unroll
    for (int i = 0; i < WR1; ++i)
      T[i] = (x1 & bs::plane<true>(s.P, i)) | (x2 & ~bs::plane<false>(s.L, i)) | (x3 & s.R1[i]);
    bs::add_signed(s.S1, T, x2);  // -L = ~L + 1
  }
  {
    uint32_t U3[WU3];  // -U - 3 = ~U - 2
#pragma unroll
    for (int i = 0; i < WU3; ++i) U3[i] = ~bs::plane<true>(s.U, i);
    bs::add_select3<-2, -2, -2>(U3, 0xFFFFFFFFu, 0u, 0u);
    uint32_t T[WU3 + 1];
#pragma unroll
    for (int i = 0; i < WU3 + 1; ++i)
      T[i] = (x12 & bs::plane<true>(s.U, i)) | (x3 & (i == 0 ? 0u : U3[i - 1]));
    bs::add_signed(s.S2, T, 0u);
  }
  {
    uint32_t Q[WP];  // A - D - 1 = U + L
    uint32_t c = 0u;
#pragma unroll
    for (int i = 0; i < WP; ++i) {
      const uint32_t a = s.U[i], b = bs::plane<false>(s.L, i);
      Q[i] = bs::xor3(a, b, c);
      c = bs::maj(a, b, c);
    }
    uint32_t T[WR3];
#pragma unroll
    for (int i = 0; i < WR3; ++i)
      T[i] = (x1 & bs::plane<true>(s.P, i)) | (x2 & bs::plane<true>(Q, i)) | (x3 & s.R3[i]);
    bs::add_signed(s.S3, T, 0u);
  }
  bs::add_select3<1, 0, -1>(s.L, x1, x2, x3);
  bs::add_select3<-2, -1, 3>(s.P, x1, x2, x3);
  bs::add_select3<-2, -2, 4>(s.U, x1, x2, x3);
  bs::add_select3<3, 1, -4>(s.R1, x1, x2, x3);
  bs::add_select3<3, 3, -6>(s.R3, x1, x2, x3);
  s.reactions += (unsigned)__popc(fired);

  // (6) absorption
  const uint32_t now_live = live_lanes(s, e) & s.live;
  uint32_t newly = s.live & ~now_live;
  if (newly) {
    s.lane_steps += (unsigned long long)__popc(newly) * s.step;
    if constexpr (LANE) {  // each run's own clock gives its absorption time
      while (newly) {
        const int l = __ffs(newly) - 1;
        newly &= newly - 1;
        Clock<PROD> c;
        unpack_clock(c, *lane_record(p, l));
        p.t_abs[group_row0(s, e) + l] = c.time(e, precision);
      }
    } else {
      const double tn = s.clk.time(e, precision);
      while (newly) {
        const int l = __ffs(newly) - 1;
        newly &= newly - 1;
        p.t_abs[group_row0(s, e) + l] = tn;
      }
    }
    s.live = now_live;
    if (!s.live) {
      s.done = true;
      if constexpr (!LANE)  // (per-run clocks: each absorbed run fills its own, at the end)
        for (; s.snap < p.n_snap; ++s.snap) capture<K, PROD>(p, s, e, s.snap, s_hist);
    }
  }
}

// Outputs of a finished group: final counts, outcomes, per-ensemble tallies, counters.
template <int K, bool PROD, bool LANE = false>
__device__ __forceinline__ void group_finish(const FrankLaunch& p, GroupState<K, PROD>& s, const Ensemble& e,
                                             unsigned int* s_hist = nullptr) {
  using Sh = FrankShape<K>;
  unsigned long long outc[4] = {0, 0, 0, 0};
  uint32_t unabsorbed = s.live;
  if constexpr (LANE) {
    unabsorbed |= s.stopped;
    // an absorbed run keeps its state for ever: it fills the snapshots its clock had not reached
    const uint32_t valid = s.nvalid >= 32 ? 0xFFFFFFFFu : ((1u << s.nvalid) - 1u);
    for (uint32_t m = valid & ~unabsorbed; m; m &= m - 1u) {
      const int l = __ffs((int)m) - 1;
      for (int k = *lane_next(p, l); k < p.n_snap; ++k) capture_lane<K, PROD>(p, s, e, k, s_hist, l);
    }
  }
  for (int l = 0; l < s.nvalid; ++l) {
    int cl, cd, ca;
    lane_counts<Sh::B, Sh::WP>(s.L, s.U, e.n_tot, l, cl, cd, ca);
    int* o = p.final_counts + (group_row0(s, e) + l) * p.n_species;
    o[p.perm[0]] = cl;
    o[p.perm[1]] = cd;
    o[p.perm[2]] = ca;
    signed char oc = -1;
    if (!((unabsorbed >> l) & 1u)) {
      const int nz = (cl != 0) + (cd != 0) + (ca != 0);
      oc = nz == 1 ? (signed char)(cl ? p.perm[0] : (cd ? p.perm[1] : p.perm[2])) : (signed char)-2;
      outc[nz == 1 ? (int)oc : 3] += 1;  // [3] also counts absorbed-with-several
    } else {
      p.t_abs[group_row0(s, e) + l] = __longlong_as_double(0x7FF0000000000000ll);
      outc[3] += 1;
    }
    p.outcome[group_row0(s, e) + l] = oc;
  }
  if (p.ens_absorbed) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (outc[k]) atomicAdd(&p.ens_absorbed[(long long)s.ens * 4 + k], outc[k]);
  }
  const uint32_t valid = s.nvalid >= 32 ? 0xFFFFFFFFu : ((1u << s.nvalid) - 1u);
  s.lane_steps += (unsigned long long)__popc(s.live) * s.step;  // lanes that never absorbed
  atomicAdd(&p.counters[kGroupSteps], s.step);
  atomicAdd(&p.counters[kLaneSteps], s.lane_steps);
  atomicAdd(&p.counters[kReactions], s.reactions);
  atomicAdd(&p.counters[kNullLaneSteps], s.lane_steps - s.reactions);
  if (s.redraws) atomicAdd(&p.counters[kRedrawRounds], (unsigned long long)s.redraws);
  atomicAdd(&p.counters[kAbsorbed], (unsigned long long)__popc(valid & ~unabsorbed));
  atomicAdd(&p.counters[kGroupsDone], 1ull);
  atomicMax(&p.counters[kMaxGroupSteps], s.step);
}

template <bool PROD>
struct TailGroups;
template <int K, bool BATCH, bool PROD>
__device__ __forceinline__ TailGroups<PROD> tail_take(const FrankLaunch& p, const GroupState<K, PROD>& s, bool active,
                                                      int& ns);
template <int K, bool BATCH, bool PROD, bool ADAPT>
__device__ __noinline__ unsigned int tail_run(const FrankLaunch& p, TailGroups<PROD> g, int ns, unsigned int* s_hist,
                                              uint32_t* wbuf);
template <int K>
struct TailShape;
constexpr int kTailWarps = 8;  // warps of the largest block (256 threads)

// The persistent kernel.  Every thread owns one group at a time and takes the next
// work item from a queue when its group finishes.  The loop is warp-synchronous: all
// 32 threads stay in it until the whole warp has run out of work, and the warp
// reconverges after every group step, so the rare divergent paths (redraws,
// snapshots, absorptions, a new group) cost one pass each instead of leaving the warp
// split for the rest of the run.  Single-ensemble launches read the ensemble from the
// kernel parameters (warp-uniform); batches from a table.  Once the queue is drained, a warp
// whose running groups are few enough hands them to tail_run (frank_tail.cuh), which finishes
// them with one run per thread.
template <int K, bool BATCH, bool PROD, bool ADAPT, bool LANE = false>
__global__ void __launch_bounds__(256) frank_kernel(const __grid_constant__ FrankLaunch p) {
  __shared__ __align__(16) uint32_t tail_words[kTailWarps][TailShape<K>::kWarpWords];
  unsigned int* const s_hist_mem = frank_dyn_smem;
  const bool smem_hist = !BATCH && p.n_snap > 0;
  unsigned int* s_hist = smem_hist ? s_hist_mem : nullptr;
  if (smem_hist) {
    for (int i = threadIdx.x; i < p.n_snap * kHistBins; i += blockDim.x) s_hist_mem[i] = 0u;
    __syncthreads();
  }
  unsigned int errors = 0u;
  GroupState<K, PROD> s;
  s.done = true;
  bool active = false, exhausted = false;
  const Threshold* thr = p.thr;
  for (;;) {
    if (!active && !exhausted) {
      const long long item = (long long)atomicAdd(p.queue, 1ull) + p.item_begin;
      if (item >= p.item_end) {
        exhausted = true;
      } else if (!BATCH) {
        group_init<K, PROD, LANE>(p, s, p.ens, thr, item, 0, s_hist);
        active = true;
      } else {
        const int ei = p.item_ens[item];
        thr = p.thr + (long long)ei * (p.n_snap + 1);
        group_init<K, PROD>(p, s, p.ens_table[ei], thr, p.item_group[item], ei, nullptr);
        active = true;
      }
    }
    if (__all_sync(0xFFFFFFFFu, exhausted && !active)) break;
    if (!LANE && p.tail_groups > 0) {
      const bool running = active && !s.done;  // (a group can be done at its start: absorbed)
      const uint32_t alive = __ballot_sync(0xFFFFFFFFu, running);
      if (__popc(alive) <= min(p.tail_groups, kTailSlots) && __any_sync(0xFFFFFFFFu, exhausted) &&
          !__any_sync(0xFFFFFFFFu, running && (BATCH ? p.ens_table[s.ens].thin : p.ens.thin))) {
        if (active && s.done) group_finish<K, PROD>(p, s, BATCH ? p.ens_table[s.ens] : p.ens);
        int ns = 0;
        const TailGroups<PROD> g = tail_take<K, BATCH, PROD>(p, s, running, ns);
        errors |= tail_run<K, BATCH, PROD, ADAPT>(p, g, ns, s_hist, tail_words[threadIdx.x >> 5]);
        break;  // the queue is drained and every group of the warp has finished
      }
    }
    if (active) {
      const Ensemble& e = BATCH ? p.ens_table[s.ens] : p.ens;
      if (!s.done) group_step<K, PROD, ADAPT, LANE>(p, s, e, thr, s_hist, errors);
      if (s.done) {
        group_finish<K, PROD, LANE>(p, s, e, s_hist);
        active = false;
      }
    }
    __syncwarp();
  }
  const unsigned int err = __reduce_or_sync(0xFFFFFFFFu, errors);
  if ((threadIdx.x & 31) == 0 && err) atomicOr(p.status, err);
  if (smem_hist) {
    __syncthreads();
    for (int i = threadIdx.x; i < p.n_snap * kHistBins; i += blockDim.x)
      if (s_hist_mem[i]) atomicAdd(&p.hist[i], (unsigned long long)s_hist_mem[i]);
  }
}

}  // namespace bitssa
