// frank_trio.cuh -- the bit-sliced step of Frank's model with the three reactions on
// three warps.
//
// A block of 96 threads serves 32 groups at a time ("slots"; lane l of every warp is
// slot l).  Warp r keeps the cumulative propensity S_{r+1} of each slot's group (K
// planes) and the signed linear forms that are the increments of S_{r+1} for reactions
// 1 | 2 | 3 in the counts before the reaction (App. A / B):
//   warp 0: dS1 = P | -L | R1     forms P = A-L-1, L, R1 = 2L-A-2
//   warp 1: dS2 = U | U  | V      forms U = A-L-D-1, V = -2U-6
//   warp 2: dS3 = P | Q  | R3     forms P, Q = A-D-1, R3 = L+D-2A-3
// Each form changes by a per-reaction constant, so all of them are kept up to date with
// one masked constant add per step.  The CDF walk of Sec. 4 (steps a-d) becomes parallel
// over r: warp r forms lt_r = [n < S_r] and the three comparator words meet in shared
// memory, so that every warp forms the same changer words xi_r.
//
// Everything that does not depend on the counts is done a step or two ahead, off the
// path from one comparison to the next: the Philox words of step s + 2 (warps 0 and 1),
// the rejection test and redraw of n for step s + 1 (the warp that finds the live lanes,
// on the next step's words in shared memory), and the clock of step s + 1 with the
// snapshots and t_end it passes (warp 1).  A step is then
//   (1) snapshots due before this event (warp 0), lt_r = [n < S_r]            -- barrier
//   (2) changer words, thinning, masked updates, the live lanes; the work ahead -- barrier
//   (3) absorption times (warp 1), outputs of finished groups (warp 0), new groups.
// A new group is set up in (3) and takes its first step two iterations later, once its
// words and its first look-ahead are in place.  The counts are read back from warp 0's
// forms: L, A = P + L + 1, D = N - L - A.  The stream, the rule and every output are
// those of the one-thread-per-group kernel.
#pragma once

#include <cstdint>

#include "bitslice.cuh"
#include "frank_kernel.cuh"
#include "internal.h"
#include "philox.cuh"

namespace bitssa {

template <int K>
struct TrioShape {
  static constexpr int B = FrankShape<K>::B;
  static constexpr int NC0 = FrankShape<K>::NC0;
  static constexpr int NCR = FrankShape<K>::NCR;
  static constexpr int NJ = (NC0 + 1) / 2;  // Philox calls per step of warps 0 and 1
  static constexpr int W1 = B + 1;          // P, U, Q in [-N-1, N-1]
  static constexpr int W2 = B + 2;          // R1 in [-N-2, 2N-2]
  static constexpr int W3 = B + 3;          // V in [-2N-4, 2N-4], R3 in [-2N-3, N-3]
};

constexpr int kTrioRow = 4 * ((kMaxK + 2 + 3) / 4);  // 36 words = 144 bytes: conflict-free 128-bit rows

// Shared memory of one block.  words[t % 3][slot] holds the attempt-0 words of step t, its
// n planes replaced by the redraw where a lane was rejected.  The clock, the look-ahead
// flags and the run counters belong to one warp each and live here rather than in
// registers, which every warp of the block would pay for.
template <bool PROD>
struct TrioShared {
  uint32_t words[3][32][kTrioRow];
  uint32_t lt[3][32];                 // comparator word of each warp
  uint32_t live[32];                  // lanes still live after the step
  uint32_t ahead_clock[32];           // next step: snapshots it passes | t_end passed << 16
  uint32_t ahead_fail[32];            // next step: 64 draws of n rejected in a row
  long long item[32];                 // work item for a free slot (-1: none left)
  Clock<PROD> clk[32];                // the clock after the last applied event
  Clock<PROD> clk_next[32];           // ... after the next step's event
  unsigned long long reactions[32], lane_steps[32];
  unsigned int redraws[32];
};

// What one thread keeps about its slot's group.  F1 | F2 | F3 are (P, L, R1) on warp 0,
// (U, V, -) on warp 1 and (P, Q, R3) on warp 2.
template <int K>
struct TrioState {
  uint32_t S[K];
  uint32_t F1[TrioShape<K>::W1], F2[TrioShape<K>::W3], F3[TrioShape<K>::W3];
  uint32_t live;
  uint32_t sgroup;
  int nvalid, ens, snap;
  int buf;  // step % 3
  unsigned long long step;
};

enum TrioSlot : int { kSlotPending = 0, kSlotActive = 1, kSlotExhausted = 2 };

template <int K>
__device__ __forceinline__ long long trio_row0(const TrioState<K>& s, const Ensemble& e) {
  return e.run_offset + ((long long)s.sgroup - e.group_base) * 32;
}

// The first W planes of a wider plane array.
template <int W, int WF>
__device__ __forceinline__ auto first_planes(const uint32_t (&x)[WF]) -> const uint32_t (&)[W] {
  static_assert(W <= WF, "view wider than the array");
  return reinterpret_cast<const uint32_t(&)[W]>(x);
}
template <int W, int WF>
__device__ __forceinline__ auto first_planes(uint32_t (&x)[WF]) -> uint32_t (&)[W] {
  static_assert(W <= WF, "view wider than the array");
  return reinterpret_cast<uint32_t(&)[W]>(x);
}

// Counts of one lane from warp 0's forms: L, A = P + L + 1, D = N - L - A.
template <int K>
__device__ __forceinline__ void trio_lane_counts(const TrioState<K>& s, int n_tot, int lane, int& l, int& d,
                                                 int& a) {
  l = (int)bs::lane_value<false>(first_planes<TrioShape<K>::B>(s.F2), lane);
  a = (int)bs::lane_value<true>(s.F1, lane) + l + 1;
  d = n_tot - l - a;
}

template <int K>
__device__ __forceinline__ void trio_capture(const FrankLaunch& p, const TrioState<K>& s, const Ensemble& e,
                                             int snap, unsigned int* s_hist) {
  const long long row0 = trio_row0(s, e);
  for (int l = 0; l < s.nvalid; ++l) {
    int cl, cd, ca;
    trio_lane_counts(s, e.n_tot, l, cl, cd, ca);
    if (s_hist) atomicAdd(&s_hist[snap * kHistBins + ee_bin(cl, cd)], 1u);
    else atomicAdd(&p.hist[((long long)s.ens * p.n_snap + snap) * kHistBins + ee_bin(cl, cd)], 1ull);
    if (p.snap_counts) {
      int* o = p.snap_counts + ((long long)snap * p.n_runs_total + row0 + l) * p.n_species;
      o[p.perm[0]] = cl;
      o[p.perm[1]] = cd;
      o[p.perm[2]] = ca;
    }
  }
}

// out = a + b + cin over W planes, the operands given plane by plane.
template <int W, typename FA, typename FB>
__device__ __forceinline__ void ripple(uint32_t (&out)[W], FA a, FB b, uint32_t cin) {
  uint32_t c = cin;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    const uint32_t x = a(i), y = b(i);
    out[i] = bs::xor3(x, y, c);
    c = bs::maj(x, y, c);
  }
}

// Set-up of one group on warp `role`: count planes, S_r by bit-sliced products, the
// warp's forms.  Returns the lanes that can react (the same on every warp).
template <int K>
__device__ __forceinline__ uint32_t trio_init(const FrankLaunch& p, TrioState<K>& s, const Ensemble& e,
                                              long long group_local, int ens_index, int role) {
  using Sh = TrioShape<K>;
  constexpr int B = Sh::B, W1 = Sh::W1, W2 = Sh::W2, W3 = Sh::W3;
  const long long run0 = group_local * 32;
  const long long left = e.n_runs - run0;
  s.nvalid = left >= 32 ? 32 : (int)left;
  const uint32_t valid = s.nvalid >= 32 ? 0xFFFFFFFFu : ((1u << s.nvalid) - 1u);
  s.sgroup = (uint32_t)(e.group_base + group_local);
  s.ens = ens_index;
  const long long row0 = e.run_offset + run0;
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
  const auto Lz = [&](int i) { return bs::plane<false>(Lp, i); };
  const auto Dz = [&](int i) { return bs::plane<false>(Dp, i); };
  const auto Az = [&](int i) { return bs::plane<false>(Ap, i); };
  // lanes that can react: some reaction with k_r > 0 has both reactants present
  const uint32_t nzL = bs::nonzero(Lp), nzD = bs::nonzero(Dp), nzA = bs::nonzero(Ap);
  const uint32_t live = (((e.active & 1u) ? (nzA & nzL) : 0u) | ((e.active & 2u) ? (nzA & nzD) : 0u) |
                         ((e.active & 4u) ? (nzL & nzD) : 0u)) & valid;
  if (role == 0) {
    bs::multiply(s.S, Ap, Lp);                                       // S1 = A L
    ripple(s.F1, Az, [&](int i) { return ~Lz(i); }, 0u);             // P = A - L - 1
#pragma unroll
    for (int i = 0; i < W3; ++i) s.F2[i] = Lz(i);                    // L
    uint32_t(&R1)[W2] = first_planes<W2>(s.F3);
    ripple(R1, [&](int i) { return i == 0 ? 0u : Lz(i - 1); }, [&](int i) { return ~Az(i); }, 0u);
    bs::add_select3<-1, -1, -1>(R1, 0xFFFFFFFFu, 0u, 0u);            // R1 = 2L - A - 2
  } else if (role == 1) {
    bs::multiply(s.S, Ap, Dp);
    bs::multiply_add(s.S, Ap, Lp);                                   // S2 = A D + A L
    uint32_t P[W1];
    ripple(P, Az, [&](int i) { return ~Lz(i); }, 0u);
    ripple(s.F1, [&](int i) { return P[i]; }, [&](int i) { return ~Dz(i); }, 0xFFFFFFFFu);  // U
#pragma unroll
    for (int i = 0; i < W3; ++i) s.F2[i] = i == 0 ? 0u : ~bs::plane<true>(s.F1, i - 1);
    bs::add_select3<-4, -4, -4>(s.F2, 0xFFFFFFFFu, 0u, 0u);          // V = 2 ~U - 4 = -2U - 6
  } else {
    bs::multiply(s.S, Ap, Dp);
    bs::multiply_add(s.S, Ap, Lp);
    bs::multiply_add(s.S, Lp, Dp);                                   // S3 = S2 + L D
    ripple(s.F1, Az, [&](int i) { return ~Lz(i); }, 0u);             // P
    uint32_t(&Q)[W1] = first_planes<W1>(s.F2);
    ripple(Q, Az, [&](int i) { return ~Dz(i); }, 0u);                // Q = A - D - 1
    uint32_t X[W3];
    ripple(X, Lz, Dz, 0u);
    ripple(s.F3, [&](int i) { return X[i]; }, [&](int i) { return i == 0 ? 0u : ~Az(i - 1); }, 0u);
    bs::add_select3<-1, -1, -1>(s.F3, 0xFFFFFFFFu, 0u, 0u);          // R3 = L + D - 2A - 3
  }
  s.step = 0;
  s.snap = 0;
  return live;
}

// Masked updates of warp `role`'s S and forms for the changer words x1, x2, x3 (App. B).
template <int K>
__device__ __forceinline__ void trio_update(TrioState<K>& s, int role, uint32_t x1, uint32_t x2, uint32_t x3) {
  using Sh = TrioShape<K>;
  constexpr int B = Sh::B, W1 = Sh::W1, W2 = Sh::W2, W3 = Sh::W3;
  if (role == 0) {
    uint32_t(&L)[B] = first_planes<B>(s.F2);
    uint32_t(&R1)[W2] = first_planes<W2>(s.F3);
    uint32_t T[W2];
#pragma unroll
    for (int i = 0; i < W2; ++i)
      T[i] = (x1 & bs::plane<true>(s.F1, i)) | (x2 & ~bs::plane<false>(L, i)) | (x3 & R1[i]);
    bs::add_signed(s.S, T, x2);  // -L = ~L + 1
    bs::add_select3<-2, -1, 3>(s.F1, x1, x2, x3);
    bs::add_select3<1, 0, -1>(L, x1, x2, x3);
    bs::add_select3<3, 1, -4>(R1, x1, x2, x3);
  } else if (role == 1) {
    const uint32_t x12 = x1 | x2;
    uint32_t T[W3];
#pragma unroll
    for (int i = 0; i < W3; ++i) T[i] = (x12 & bs::plane<true>(s.F1, i)) | (x3 & s.F2[i]);
    bs::add_signed(s.S, T, 0u);
    bs::add_select3<-2, -2, 4>(s.F1, x1, x2, x3);
    bs::add_select3<4, 4, -8>(s.F2, x1, x2, x3);
  } else {
    uint32_t(&Q)[W1] = first_planes<W1>(s.F2);
    uint32_t T[W3];
#pragma unroll
    for (int i = 0; i < W3; ++i)
      T[i] = (x1 & bs::plane<true>(s.F1, i)) | (x2 & bs::plane<true>(Q, i)) | (x3 & s.F3[i]);
    bs::add_signed(s.S, T, 0u);
    bs::add_select3<-2, -1, 3>(s.F1, x1, x2, x3);
    bs::add_select3<-1, -2, 3>(Q, x1, x2, x3);
    bs::add_select3<3, 3, -6>(s.F3, x1, x2, x3);
  }
}

// Lanes that can still react, from warp 0's forms (needed when some k_r = 0).
template <int K>
__device__ __forceinline__ uint32_t trio_live_from_forms(const TrioState<K>& s, const Ensemble& e) {
  using Sh = TrioShape<K>;
  constexpr int B = Sh::B, W1 = Sh::W1;
  const uint32_t(&L)[B] = first_planes<B>(s.F2);
  const auto Lz = [&](int i) { return bs::plane<false>(L, i); };
  uint32_t A[W1], X[W1], D[W1];
  ripple(A, [&](int i) { return s.F1[i]; }, Lz, 0xFFFFFFFFu);  // A = P + L + 1
  ripple(X, [&](int i) { return A[i]; }, Lz, 0u);              // L + A
  ripple(D, [&](int i) { return ((e.n_tot >> i) & 1) ? 0xFFFFFFFFu : 0u; }, [&](int i) { return ~X[i]; },
         0xFFFFFFFFu);                                         // D = N - (L + A)
  const uint32_t nzL = bs::nonzero(L), nzA = bs::nonzero(A), nzD = bs::nonzero(D);
  return ((e.active & 1u) ? (nzA & nzL) : 0u) | ((e.active & 2u) ? (nzA & nzD) : 0u) |
         ((e.active & 4u) ? (nzL & nzD) : 0u);
}

// Lanes where n < C (C shared by all lanes), n's planes read from shared memory.
template <int K>
__device__ __forceinline__ uint32_t trio_less_than_const(const uint32_t* n, uint32_t C) {
  uint32_t borrow = 0u;
#pragma unroll
  for (int i = 0; i < K; ++i) borrow = bs::maj(~n[i], 0u - ((C >> i) & 1u), borrow);
  return borrow;
}

// Lanes where n < S, n's planes read from shared memory (the borrow out of n - S).
template <int K>
__device__ __forceinline__ uint32_t trio_less_than(const uint32_t* n, const uint32_t (&S)[K]) {
  uint32_t q[4 * ((K + 3) / 4)];
#pragma unroll
  for (int c = 0; c < (K + 3) / 4; ++c) {
    const uint4 v = reinterpret_cast<const uint4*>(n)[c];
    q[4 * c] = v.x;
    q[4 * c + 1] = v.y;
    q[4 * c + 2] = v.z;
    q[4 * c + 3] = v.w;
  }
  uint32_t borrow = 0u;
#pragma unroll
  for (int i = 0; i < K; ++i) borrow = bs::maj(~q[i], S[i], borrow);
  return borrow;
}

__device__ __forceinline__ long long trio_take(const FrankLaunch& p) {
  const long long item = (long long)atomicAdd(p.queue, 1ull) + p.item_begin;
  return item < p.item_end ? item : -1;
}

// Attempt-0 words of `step` into one slot's row: warp `role` (0 or 1) makes calls role,
// role + 2, ...
template <int K>
__device__ __forceinline__ void trio_words(uint32_t* row, uint32_t sgroup, unsigned long long step, int role,
                                           PhiloxKey key) {
  constexpr int NC0 = TrioShape<K>::NC0, NJ = TrioShape<K>::NJ;
  uint32_t w[4 * NJ];
  philox4x32_10_block<NJ>(w, stream_counter(sgroup, step, 0u, 0u, 0u), (uint32_t)role, key, 2u);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int c = 2 * j + role;
    if (c < NC0) *reinterpret_cast<uint4*>(row + 4 * c) = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
  }
}

// The rejection test of one step's n (planes in `row`) for the lanes in `live`, and the
// redraw of rejected lanes in place: a rejected lane replaces its planes from the highest
// one where n and lambda_int differ (all of them when equal) with the same planes of the
// next attempt.  Returns false after 64 rejections in a row.
template <int K>
__device__ __forceinline__ bool trio_redraw(uint32_t* row, const Ensemble& e, uint32_t sgroup,
                                            unsigned long long step, uint32_t live, PhiloxKey key,
                                            unsigned int& rounds) {
  constexpr int NCR = TrioShape<K>::NCR;
  if (!e.reject) return true;  // a bound padded to 2^K accepts every draw
  uint32_t pass = 0xFFFFFFFFu;  // n >= lambda_int needs every plane of its leading run of ones set
#pragma unroll
  for (int i = 0; i < K; ++i) pass &= row[i] | e.top_mask[i];
  if (!(pass & live)) return true;
  uint32_t need = ~trio_less_than_const<K>(row, e.lambda_int) & live;
  for (uint32_t attempt = 1u; need; ++attempt) {
    if (attempt >= 64u) return false;
    ++rounds;
    uint32_t above = 0u;
    if constexpr (K >= 25) {
      // wide n: the calls from the top, two at a time, until no lane replaces a lower plane
      // (near N_tot = 46 400, where half of all draws are rejected, three of eight calls suffice)
#pragma unroll
      for (int c = NCR - 1; c >= 0; c -= 2) {
        if (need & ~above) {
          const int lo = c > 0 ? c - 1 : 0;
          uint32_t wr[8];
          philox4x32_10_block<2>(wr, stream_counter(sgroup, step, attempt, 0u, 0u), (uint32_t)lo, key);
#pragma unroll
          for (int j = 7; j >= 0; --j) {
            const int i = 4 * lo + j;
            if (i <= 4 * c + 3 && i < K) {
              const uint32_t m = need & ~above;
              const uint32_t ni = row[i];
              above |= ni ^ (0u - ((e.lambda_int >> i) & 1u));
              row[i] = (ni & ~m) | (wr[j] & m);
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
        const uint32_t ni = row[i];
        above |= ni ^ (0u - ((e.lambda_int >> i) & 1u));
        row[i] = (ni & ~m) | (wr[i] & m);
      }
    }
    need &= ~trio_less_than_const<K>(row, e.lambda_int);
  }
  return true;
}

// Resident blocks per SM the register allocation is sized for: 128 registers a thread up to
// K = 24, more for the wider states above.
constexpr int trio_min_blocks(int K) { return K <= 24 ? 5 : (K <= 28 ? 4 : 2); }

template <int K, bool BATCH, bool PROD>
__global__ void __launch_bounds__(kTrioBlock, trio_min_blocks(K))
    frank_trio_kernel(const __grid_constant__ FrankLaunch p) {
  using Sh = TrioShape<K>;
  constexpr int NC0 = Sh::NC0;
  static_assert(4 * NC0 <= kTrioRow, "word row too small");
  extern __shared__ unsigned int s_hist_mem[];
  __shared__ __align__(16) TrioShared<PROD> sh;
  const int role = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool smem_hist = !BATCH && p.n_snap > 0;
  unsigned int* s_hist = smem_hist ? s_hist_mem : nullptr;
  if (smem_hist)
    for (int i = threadIdx.x; i < p.n_snap * kHistBins; i += blockDim.x) s_hist_mem[i] = 0u;
  if (role == 0) sh.item[lane] = trio_take(p);
  __syncthreads();

  TrioState<K> s;
  s.ens = 0;
  s.live = 0u;
  s.step = 0ull;
  s.buf = 0;
  int slot = kSlotPending;
  bool fresh = false;  // set up in the last iteration: no step before its look-ahead is done
  unsigned int errors = 0u;
  const int precision = p.precision;

  // a pending slot reads its work item (taken by warp 0 at least one barrier earlier)
  auto start_group = [&]() {
    const long long item = sh.item[lane];
    if (item < 0) {
      slot = kSlotExhausted;
      return;
    }
    const int ei = BATCH ? p.item_ens[item] : 0;
    const Ensemble& e = BATCH ? p.ens_table[ei] : p.ens;
    const uint32_t live0 = trio_init<K>(p, s, e, BATCH ? (long long)p.item_group[item] : item, ei, role);
    if (role == 0) {
      const uint32_t valid = s.nvalid >= 32 ? 0xFFFFFFFFu : ((1u << s.nvalid) - 1u);
      uint32_t at0 = valid & ~live0;  // runs that start absorbed are absorbed at t = 0
      const long long row0 = trio_row0(s, e);
      while (at0) {
        const int l = __ffs(at0) - 1;
        at0 &= at0 - 1;
        p.t_abs[row0 + l] = 0.0;
      }
      sh.reactions[lane] = sh.lane_steps[lane] = 0ull;
      sh.redraws[lane] = 0u;
    }
    if (role == 1) {
      Clock<PROD> clk;
      clk.reset();
      clk.aim(p.thr[(long long)ei * (p.n_snap + 1)]);
      sh.clk[lane] = clk;
    }
    if (role < 2) {  // the words of steps 0 and 1
      const PhiloxKey key{(uint32_t)e.seed, (uint32_t)(e.seed >> 32)};
      trio_words<K>(sh.words[0][lane], s.sgroup, 0ull, role, key);
      trio_words<K>(sh.words[1][lane], s.sgroup, 1ull, role, key);
    }
    s.live = live0;
    s.buf = 0;
    slot = kSlotActive;
    fresh = true;
  };
  start_group();

  for (;;) {
    if (__all_sync(0xFFFFFFFFu, slot == kSlotExhausted)) break;  // the same on every warp
    const Ensemble& e = BATCH ? p.ens_table[s.ens] : p.ens;
    const Threshold* thr = p.thr + (BATCH ? (long long)s.ens * (p.n_snap + 1) : 0ll);
    const PhiloxKey key{(uint32_t)e.seed, (uint32_t)(e.seed >> 32)};
    const bool act = slot == kSlotActive;
    bool stepping = act && !fresh && s.live != 0u;
    bool stopped = false;
    if (stepping && p.step_budget > 0 && (long long)s.step >= p.step_budget) {
      errors |= kErrTimeout;
      stepping = false;
      stopped = true;
    }
    const uint32_t* row = sh.words[s.buf][lane];

    // ---- (1) what the look-ahead found for this step; snapshots; the warp's comparator
    uint32_t lt = 0u;
    if (stepping) {
      if (sh.ahead_fail[lane]) {
        errors |= kErrRedraw;
        stopped = true;
      } else {
        const uint32_t ac = sh.ahead_clock[lane];
        if (role == 0)
          for (uint32_t k = ac & 0xFFFFu; k > 0u; --k) {  // the state before this step's event
            trio_capture<K>(p, s, e, s.snap, s_hist);
            ++s.snap;
          }
        stopped = (ac >> 16) != 0u;  // t_end passed: the event is not applied
      }
      if (!stopped) lt = trio_less_than<K>(row, s.S);
    }
    sh.lt[role][lane] = lt;
    __syncthreads();

    // ---- (2) changer words, thinning, updates, live lanes; the work ahead
    const bool go = stepping && !stopped;
    const bool live_writer = (e.active == 7u) ? role == 2 : role == 0;
    uint32_t now_live = s.live;
    if (go) {
      const uint32_t lt1 = sh.lt[0][lane], lt2 = sh.lt[1][lane], lt3 = sh.lt[2][lane];
      uint32_t x1 = lt1, x2 = lt2 & ~lt1, x3 = lt3 & ~lt2;
      if (e.thin)
        thin_step<K + 2, 4 * NC0>(e, [&](int k) { return row[k]; }, s.live, s.sgroup, s.step, NC0, key, x1, x2, x3);
      const uint32_t fired = x1 | x2 | x3;
      ++s.step;
      s.buf = s.buf == 2 ? 0 : s.buf + 1;
      if (fired) {
        trio_update<K>(s, role, x1, x2, x3);
        if (role == 0) sh.reactions[lane] += (unsigned)__popc(fired);
        if (live_writer)
          now_live = (e.active == 7u ? bs::nonzero(s.S) : trio_live_from_forms<K>(s, e)) & s.live;
      }
      if (role == 1) sh.clk[lane] = sh.clk_next[lane];  // the event is applied
    }
    if (go || (act && fresh)) {  // ahead: step s.step (the next one)
      uint32_t* row_next = sh.words[s.buf][lane];
      if (role == 1) {
        const Clock<PROD> clk = sh.clk[lane];
        Clock<PROD> nx;
        bool crossed = clock_advance(clk, nx, row_next[K], row_next[K + 1], e, precision);
        uint32_t passed = 0u, stop = 0u;
        while (crossed) {
          if (s.snap >= p.n_snap) {
            stop = 1u;
            break;
          }
          ++passed;
          ++s.snap;
          nx.aim(thr[s.snap]);
          if constexpr (PROD) crossed = clock_crosses(nx);
          else crossed = clock_crosses(nx, precision);
        }
        sh.clk_next[lane] = nx;
        sh.ahead_clock[lane] = passed | (stop << 16);
      }
      if (live_writer) {
        uint32_t fail = 0u;
        // the paper's shared draw (Sec. 4, step a): lane 0's n, redrawn whether or not lane 0 is
        // live, then copied to every lane
        if (now_live && !(p.step_budget > 0 && (long long)s.step >= p.step_budget))
          fail = trio_redraw<K>(row_next, e, s.sgroup, s.step, e.shared_n ? 1u : now_live, key, sh.redraws[lane])
                     ? 0u : 1u;
        if (e.shared_n)
          for (int i = 0; i < K; ++i) row_next[i] = 0u - (row_next[i] & 1u);
        sh.ahead_fail[lane] = fail;
      }
      if (go && role < 2) trio_words<K>(sh.words[s.buf == 2 ? 0 : s.buf + 1][lane], s.sgroup, s.step + 1ull, role, key);
    }
    if (live_writer) sh.live[lane] = now_live;
    __syncthreads();

    // ---- (3) absorption times (warp 1), finished groups (warp 0), new groups
    if (act && fresh) {
      fresh = false;
    } else if (act) {
      const uint32_t nl = sh.live[lane];
      uint32_t newly = s.live & ~nl;
      if (newly) {
        const long long row0 = trio_row0(s, e);
        if (role == 0) sh.lane_steps[lane] += (unsigned long long)__popc(newly) * s.step;
        if (role == 1) {
          const double tn = sh.clk[lane].time(e, precision);
          while (newly) {
            const int l = __ffs(newly) - 1;
            newly &= newly - 1;
            p.t_abs[row0 + l] = tn;
          }
        }
      }
      s.live = nl;
      if (!s.live || stopped) {
        if (role == 0) {
          if (!s.live)
            for (; s.snap < p.n_snap; ++s.snap) trio_capture<K>(p, s, e, s.snap, s_hist);
          const long long row0 = trio_row0(s, e);
          unsigned long long outc[4] = {0, 0, 0, 0};
          for (int l = 0; l < s.nvalid; ++l) {
            int cl, cd, ca;
            trio_lane_counts(s, e.n_tot, l, cl, cd, ca);
            int* o = p.final_counts + (row0 + l) * p.n_species;
            o[p.perm[0]] = cl;
            o[p.perm[1]] = cd;
            o[p.perm[2]] = ca;
            signed char oc = -1;
            if (!((s.live >> l) & 1u)) {
              const int nz = (cl != 0) + (cd != 0) + (ca != 0);
              oc = nz == 1 ? (signed char)(cl ? p.perm[0] : (cd ? p.perm[1] : p.perm[2])) : (signed char)-2;
              outc[nz == 1 ? (int)oc : 3] += 1;  // [3] also counts absorbed-with-several
            } else {
              p.t_abs[row0 + l] = __longlong_as_double(0x7FF0000000000000ll);
              outc[3] += 1;
            }
            p.outcome[row0 + l] = oc;
          }
          if (p.ens_absorbed) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (outc[k]) atomicAdd(&p.ens_absorbed[(long long)s.ens * 4 + k], outc[k]);
          }
          const uint32_t valid = s.nvalid >= 32 ? 0xFFFFFFFFu : ((1u << s.nvalid) - 1u);
          const unsigned long long lane_steps =
              sh.lane_steps[lane] + (unsigned long long)__popc(s.live) * s.step;  // + lanes never absorbed
          const unsigned long long reactions = sh.reactions[lane];
          atomicAdd(&p.counters[kGroupSteps], s.step);
          atomicAdd(&p.counters[kLaneSteps], lane_steps);
          atomicAdd(&p.counters[kReactions], reactions);
          atomicAdd(&p.counters[kNullLaneSteps], lane_steps - reactions);
          if (sh.redraws[lane]) atomicAdd(&p.counters[kRedrawRounds], (unsigned long long)sh.redraws[lane]);
          atomicAdd(&p.counters[kAbsorbed], (unsigned long long)__popc(valid & ~s.live));
          atomicAdd(&p.counters[kGroupsDone], 1ull);
          atomicMax(&p.counters[kMaxGroupSteps], s.step);
          sh.item[lane] = trio_take(p);
        }
        slot = kSlotPending;
      }
    } else if (slot == kSlotPending) {
      start_group();
    }
  }
  const unsigned int err = __reduce_or_sync(0xFFFFFFFFu, errors);
  if (lane == 0 && err) atomicOr(p.status, err);
  if (smem_hist) {
    __syncthreads();
    for (int i = threadIdx.x; i < p.n_snap * kHistBins; i += blockDim.x)
      if (s_hist_mem[i]) atomicAdd(&p.hist[i], (unsigned long long)s_hist_mem[i]);
  }
}

}  // namespace bitssa
