// general_kernel.cuh -- the bit-sliced Gillespie step loop for any conserved mass-action
// network of order 1 or 2 (Sec. 2) on sm_103a.
//
// One thread owns one group of 32 runs (lane l of every plane is run 32 g + l).  The
// Frank kernel keeps cumulative propensities and their linear increments; this one
// recomputes every propensity at every step from the count planes, with the bit-sliced
// schoolbook product of Sec. 4.1:
//   h_r = x_a x_b            (A + B -> ...)
//   h_r = x_a (x_a - 1) / 2  (2A -> ...)
//   h_r = x_a                (A -> ...)
// The count planes live in shared memory (each warp's region laid out [word][lane], plane i of
// species s at word s PL + i), so that a reaction's reactants are found by index at run time and
// one kernel serves every network of up to 8 species and 8 reactions; the per-step values (n,
// the running sum S, one product) stay in registers.
//
// Incremental mode (the default) keeps every h_r in shared memory as well and, after each
// event, adds its change, which for mass action is linear in the counts before the event
// (App. A generalised): with d_s in [-2, 2] the change of species s in a lane,
//   d(x_a x_b)            = d_b x_a + d_a x_b + d_a d_b
//   d(x_a (x_a - 1) / 2)  = d_a x_a + d_a (d_a - 1) / 2
//   d(x_a)                = d_a
// Each term is a masked, shifted, conditionally negated copy of a count: no product per step.
//
// One group step (Sec. 3, steps 1-7, the draw done by Sec. 4's steps a-d), in the order of
// the Frank kernel and the oracle:
//   1. Philox words of attempt 0: the K planes of n (rejection and partial redraw above
//      lambda_int unless the bound is padded to 2^K) and the clock's two words.
//   2. Clock, snapshots (state before the event), t_end.
//   3. For r = 0..R-1: xi_r = [S_{r-1} <= n < S_r] (Eq. equation-changer), taken as the borrow
//      of n - h_0 - ... - h_r out of the r-th subtraction; a lane with n >= S_R fires nothing (a
//      ghost or null event).
//   4. Thinning of reactions with k_r < k_max.
//   5. x_i += sum_r xi_r nu_ri for every species (Eq. equation-v), two's complement.
//   6. Absorption: a lane none of whose reactions with k_r > 0 has a nonzero propensity.
#pragma once

#include <cstdint>

#include "bitslice.cuh"
#include "frank_kernel.cuh"
#include "internal.h"
#include "philox.cuh"

namespace bitssa {

// Count planes a general network may need at K propensity planes when it has a reaction of
// order 2: lambda_int >= N (N - 1) / 2, so N is at most Frank's largest N for K planes.
template <int K>
struct GeneralShape {
  static constexpr int BM = FrankShape<K>::B;     // count planes read by the products
  static constexpr int NC0 = (K + 2 + 3) / 4;     // Philox calls for n and tau
  static constexpr int B1 = K < kMaxCountPlanes ? K : kMaxCountPlanes;  // first-order reads
};

// The state one thread keeps in registers; the counts are in shared memory.
template <bool PROD>
struct GeneralState {
  uint32_t live;     // lanes that can still react
  uint32_t valid;    // lanes holding a run
  uint32_t sgroup;   // stream group index
  int nvalid;
  int ens;
  int snap;
  unsigned long long step;
  Clock<PROD> clk;
  unsigned long long reactions, lane_steps;
  unsigned int redraws;
  bool done;
};

// Shared-memory view of one thread's words.  Each warp has its own region, laid out
// [word][lane] with a stride of 32, so that a plane's offset is a compile-time immediate and
// the 32 lanes of a warp touch 32 banks: plane i of species s at [(s PL + i) 32], the scratch
// words (per species: the lanes with a nonzero count, with at least two, and the three planes
// of its change in this step), and in incremental mode plane i of h_r.
struct CountPlanes {
  static constexpr int kStride = 32;
  uint32_t* base;     // this thread's word of plane 0 of species 0
  uint32_t* scratch;  // this thread's word of scratch 0
  uint32_t* hp;       // incremental mode: this thread's word of plane 0 of h_0
  int PL;             // planes stored per species
  int K;              // planes of each h_r
  __device__ __forceinline__ uint32_t& at(int s, int i) const { return base[(s * PL + i) * kStride]; }
  __device__ __forceinline__ uint32_t& nonzero(int s) const { return scratch[s * kStride]; }
  __device__ __forceinline__ uint32_t& two(int s) const { return scratch[(kMaxSpecies + s) * kStride]; }
  // the change of species s in this step, plane b of three (two's complement)
  __device__ __forceinline__ uint32_t& change(int s, int b) const {
    return scratch[(2 * kMaxSpecies + 3 * s + b) * kStride];
  }
  __device__ __forceinline__ uint32_t& h(int r, int i) const { return hp[(r * K + i) * kStride]; }
};


template <int W>
__device__ __forceinline__ void load_planes(uint32_t (&x)[W], const CountPlanes& c, int s) {
#pragma unroll
  for (int i = 0; i < W; ++i) x[i] = c.at(s, i);
}

// Count planes of an ensemble: the bit length of its N_tot.
__device__ __forceinline__ int count_planes(const Ensemble& e) { return 32 - __clz(e.n_tot); }

// Lanes where some reaction with k_r > 0 has h_r > 0: h = x_a x_b > 0 iff both are nonzero,
// x_a (x_a - 1) / 2 > 0 iff x_a >= 2, x_a > 0 iff it is nonzero.  The planes at and above the
// ensemble's B are zero, so the first BM planes are read unrolled and only counts wider than
// that (first-order networks) take the loop.
template <int K>
__device__ __forceinline__ uint32_t general_live(const Network& net, const Ensemble& e, const CountPlanes& c) {
  constexpr int BM = GeneralShape<K>::BM;
  const int B = count_planes(e);
  for (int s = 0; s < net.S; ++s) {
    uint32_t x[BM];
    load_planes(x, c, s);
    uint32_t two = 0u;
#pragma unroll
    for (int i = 1; i < BM; ++i) two |= x[i];
    for (int i = BM; i < B; ++i) two |= c.at(s, i);
    c.nonzero(s) = x[0] | two;
    c.two(s) = two;
  }
  uint32_t m = 0u;
  for (int r = 0; r < net.R; ++r) {
    if (!((e.active >> r) & 1u)) continue;
    const int a = net.a[r], b = net.b[r];
    m |= net.order[r] == 1 ? c.nonzero(a) : (b == a ? c.two(a) : (c.nonzero(a) & c.nonzero(b)));
  }
  return m;
}

// h (K planes) = x (x - 1) / 2 for the W planes of x: the product is even and below 2^(K+1);
// its plane 0 is dropped.
template <int K, int W>
__device__ __forceinline__ void half_square(uint32_t (&h)[K], const uint32_t (&x)[W]) {
  uint32_t xm[W];
  uint32_t borrow = 0xFFFFFFFFu;  // x - 1
#pragma unroll
  for (int i = 0; i < W; ++i) {
    xm[i] = x[i] ^ borrow;
    borrow &= ~x[i];
  }
  uint32_t p[K + 1];
  bs::multiply(p, x, xm);
#pragma unroll
  for (int i = 0; i < K; ++i) h[i] = p[i + 1];
}

// h (K planes) = the propensity of reaction r in every lane, from the count planes.
template <int K>
__device__ __forceinline__ void general_propensity(uint32_t (&h)[K], const Network& net, int r,
                                                   const CountPlanes& c, int B) {
  using Sh = GeneralShape<K>;
  constexpr int BM = Sh::BM;
  const int a = net.a[r];
  if (net.order[r] == 1) {  // h = x_a, zero-extended
#pragma unroll
    for (int i = 0; i < K; ++i) h[i] = (i < Sh::B1 && i < B) ? c.at(a, i) : 0u;
    return;
  }
  uint32_t xa[BM];
  load_planes(xa, c, a);
  if (net.b[r] != a) {  // h = x_a x_b
    uint32_t xb[BM];
    load_planes(xb, c, net.b[r]);
    bs::multiply(h, xa, xb);
    return;
  }
  half_square(h, xa);
}

// h (K planes) += d x for a lane-wise d in [-2, 2] (three two's-complement planes) and an
// unsigned x (W planes): the lanes with |d| = 1 add x, with |d| = 2 add 2x (x one plane up),
// negated where d < 0 (complemented, plus one at the carry-in).  A plane of the addend is
// (nz & (two ? x_{i-1} : x_i)) ^ neg: two three-input operations.
template <int K, int W>
__device__ __forceinline__ void add_scaled(uint32_t (&h)[K], const uint32_t (&x)[W], const uint32_t (&d)[3]) {
  const uint32_t nz = d[0] | d[1], two = d[1] & ~d[0], neg = d[2];
  uint32_t carry = neg;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const uint32_t xi = i < W ? x[i] : 0u, xm = (i >= 1 && i - 1 < W) ? x[i - 1] : 0u;
    const uint32_t t = (nz & ((two & xm) | (~two & xi))) ^ neg;
    const uint32_t s = bs::xor3(h[i], t, carry);
    carry = bs::maj(h[i], t, carry);
    h[i] = s;
  }
}

// h (K planes) += a small signed lane-wise constant given by its low planes c[0..2] and its
// sign plane c[3] (two's complement, sign-extended).
template <int K>
__device__ __forceinline__ void add_small(uint32_t (&h)[K], const uint32_t (&c)[4]) {
  uint32_t carry = 0u;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const uint32_t t = c[i < 3 ? i : 3];
    const uint32_t s = bs::xor3(h[i], t, carry);
    carry = bs::maj(h[i], t, carry);
    h[i] = s;
  }
}

// The constant term of a homodimer's change, d_a (d_a - 1) / 2: 3, 1, 0, 0, 1 for d_a = -2..2,
// as the low planes and the sign plane add_small takes.
__device__ __forceinline__ void same_constant(const uint32_t (&da)[3], uint32_t (&cst)[4]) {
  const uint32_t m2 = da[1] & ~da[0];  // |d| = 2
  cst[0] = da[1] & (da[2] | ~da[0]);   // d = -2, -1 or 2
  cst[1] = m2 & da[2];                 // d = -2
  cst[2] = 0u;
  cst[3] = 0u;
}

// The constant term of a pair's change, d_a d_b: magnitude 1, 2 or 4, negative when exactly one
// of them is; two's complement of -m: m1 -> ...1111, m2 -> ...1110, m4 -> ...1100.
__device__ __forceinline__ void pair_constant(const uint32_t (&da)[3], const uint32_t (&db)[3], uint32_t (&cst)[4]) {
  const uint32_t a1 = da[0], a2 = da[1] & ~da[0], b1 = db[0], b2 = db[1] & ~db[0];
  const uint32_t m1 = a1 & b1, m2 = (a1 & b2) | (a2 & b1), m4 = a2 & b2;
  const uint32_t neg = (da[2] ^ db[2]) & (m1 | m2 | m4);
  cst[0] = m1;
  cst[1] = (m2 & ~neg) | (neg & (m1 | m2));
  cst[2] = (m4 & ~neg) | (neg & (m1 | m2 | m4));
  cst[3] = neg;
}

// h_r += its change in this step (see the file header), from the counts before the event and
// the change planes of every species.
// m -= h over K planes, modulo 2^K; returns the lanes that borrow out of the top plane.  Taking
// h_0, h_1, ... off n in turn, the subtraction of h_r is the first to borrow exactly where
// S_{r-1} <= n < S_r (the running value n - S_r stays above -2^K, so it borrows at most once
// while S_R < 2^K): the changer word of reaction r (Eq. equation-changer) at one subtraction per
// reaction instead of a sum and a comparison.
template <int K>
__device__ __forceinline__ uint32_t sub_borrow(uint32_t (&m)[K], const uint32_t (&h)[K]) {
  uint32_t borrow = 0u;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const uint32_t mi = m[i];
    m[i] = bs::xor3(mi, h[i], borrow);
    borrow = bs::maj(~mi, h[i], borrow);
  }
  return borrow;
}

template <int K>
__device__ __forceinline__ void general_increment(const Network& net, int r, const CountPlanes& c) {
  using Sh = GeneralShape<K>;
  constexpr int BM = Sh::BM;
  const int a = net.a[r], b = net.b[r];
  const bool moves = ((net.changes >> a) & 1u) || (b >= 0 && ((net.changes >> b) & 1u));
  if (!moves) return;
  const uint32_t da[3] = {c.change(a, 0), c.change(a, 1), c.change(a, 2)};
  uint32_t h[K];
#pragma unroll
  for (int i = 0; i < K; ++i) h[i] = c.h(r, i);
  if (net.order[r] == 1) {  // + d_a
    const uint32_t cst[4] = {da[0], da[1], da[2], da[2]};
    add_small(h, cst);
  } else if (b == a) {  // + d_a x_a + d_a (d_a - 1) / 2, the last in {3, 1, 0, 0, 1} for d_a = -2..2
    uint32_t xa[BM];
    load_planes(xa, c, a);
    add_scaled(h, xa, da);
    uint32_t cst[4];
    same_constant(da, cst);
    add_small(h, cst);
  } else {  // + d_b x_a + d_a x_b + d_a d_b
    const uint32_t db[3] = {c.change(b, 0), c.change(b, 1), c.change(b, 2)};
    uint32_t xa[BM], xb[BM];
    load_planes(xa, c, a);
    load_planes(xb, c, b);
    add_scaled(h, xa, db);
    add_scaled(h, xb, da);
    uint32_t cst[4];
    pair_constant(da, db, cst);
    add_small(h, cst);
  }
#pragma unroll
  for (int i = 0; i < K; ++i) c.h(r, i) = h[i];
}

// Set up a group: counts into shared memory (padding lanes hold zero counts and never react),
// the live lanes, the clock.
template <int K, bool PROD>
__device__ __forceinline__ void general_init(const FrankLaunch& p, GeneralState<PROD>& s, const Ensemble& e,
                                             const Threshold* thr, long long group_local, int ens_index,
                                             const CountPlanes& c, unsigned int* s_hist);

template <int K, bool PROD>
__device__ __forceinline__ void general_capture(const FrankLaunch& p, const GeneralState<PROD>& s,
                                                const Ensemble& e, int snap, const CountPlanes& c,
                                                unsigned int* s_hist);

// Counts of lane l: species s from its planes.
__device__ __forceinline__ int lane_count(const CountPlanes& c, int s, int B, int l) {
  int v = 0;
  for (int i = 0; i < B; ++i) v |= (int)((c.at(s, i) >> l) & 1u) << i;
  return v;
}

__device__ __forceinline__ long long general_row0(uint32_t sgroup, const Ensemble& e) {
  return e.run_offset + ((long long)sgroup - e.group_base) * 32;
}

// One snapshot of a group: the ee histogram and, if kept, every run's counts; count(s, l) reads
// species s of lane l.
template <bool PROD, class Count>
__device__ __forceinline__ void capture_counts(const FrankLaunch& p, const GeneralState<PROD>& s,
                                               const Ensemble& e, int snap, unsigned int* s_hist, Count&& count) {
  const Network& net = p.net;
  for (int l = 0; l < s.nvalid; ++l) {
    const int cx = net.hist_x >= 0 ? count(net.hist_x, l) : 0;
    const int cy = net.hist_y >= 0 ? count(net.hist_y, l) : 0;
    const int bin = ee_bin(cx, cy);
    if (s_hist) atomicAdd(&s_hist[snap * kHistBins + bin], 1u);
    else atomicAdd(&p.hist[((long long)s.ens * p.n_snap + snap) * kHistBins + bin], 1ull);
    if (p.snap_counts) {
      int* o = p.snap_counts + ((long long)snap * p.n_runs_total + general_row0(s.sgroup, e) + l) * net.S;
      for (int sp = 0; sp < net.S; ++sp) o[sp] = count(sp, l);
    }
  }
}

template <int K, bool PROD>
__device__ __forceinline__ void general_capture(const FrankLaunch& p, const GeneralState<PROD>& s,
                                                const Ensemble& e, int snap, const CountPlanes& c,
                                                unsigned int* s_hist) {
  const int B = count_planes(e);
  capture_counts(p, s, e, snap, s_hist, [&](int sp, int l) { return lane_count(c, sp, B, l); });
}

template <int K, bool PROD>
__device__ __forceinline__ void general_init(const FrankLaunch& p, GeneralState<PROD>& s, const Ensemble& e,
                                             const Threshold* thr, long long group_local, int ens_index,
                                             const CountPlanes& c, unsigned int* s_hist) {
  const Network& net = p.net;
  const long long run0 = group_local * 32;
  const long long left = e.n_runs - run0;
  s.nvalid = left >= 32 ? 32 : (int)left;
  s.valid = s.nvalid >= 32 ? 0xFFFFFFFFu : ((1u << s.nvalid) - 1u);
  s.sgroup = (uint32_t)(e.group_base + group_local);
  s.ens = ens_index;
  const long long row0 = e.run_offset + run0;
  for (int sp = 0; sp < net.S; ++sp) {
    for (int i = 0; i < c.PL; ++i) {
      uint32_t w = 0u;
      if (p.init_counts) {
        for (int l = 0; l < s.nvalid; ++l) w |= (uint32_t)((p.init_counts[(row0 + l) * net.S + sp] >> i) & 1) << l;
      } else if ((e.init[sp] >> i) & 1) {
        w = s.valid;
      }
      c.at(sp, i) = w;
    }
  }
  if (net.incremental) {
    const int B = count_planes(e);
    for (int r = 0; r < net.R; ++r) {
      uint32_t h[K];
      general_propensity<K>(h, net, r, c, B);
#pragma unroll
      for (int i = 0; i < K; ++i) c.h(r, i) = h[i];
    }
  }
  s.live = general_live<K>(net, e, c) & s.valid;
  uint32_t at0 = s.valid & ~s.live;  // runs that start absorbed are absorbed at t = 0
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
  s.done = s.live == 0u;
  if (s.done)
    for (; s.snap < p.n_snap; ++s.snap) general_capture<K, PROD>(p, s, e, s.snap, c, s_hist);
}

// Steps (1) and (2) of a group step: the Philox words of attempt 0 (w) and n, redrawn where it is
// at or above lambda_int, then the clock, with capture(snap) called for every snapshot the event
// passes.  False when the group stops at this step (t_end passed, the step budget, a failed
// redraw); the event is then not applied.
template <int K, bool PROD, class Capture>
__device__ __forceinline__ bool general_draw(const FrankLaunch& p, GeneralState<PROD>& s, const Ensemble& e,
                                             const Threshold* thr, uint32_t (&n)[K],
                                             uint32_t (&w)[4 * GeneralShape<K>::NC0], unsigned int& errors,
                                             Capture&& capture) {
  constexpr int NC0 = GeneralShape<K>::NC0;
  const PhiloxKey key{(uint32_t)e.seed, (uint32_t)(e.seed >> 32)};
  const int precision = p.precision;
  if (p.step_budget > 0 && (long long)s.step >= p.step_budget) {
    errors |= kErrTimeout;
    s.done = true;
    return false;
  }
  // (1) the random words of attempt 0; n, redrawn where it is at or above lambda_int
  philox4x32_10_block<NC0>(w, stream_counter(s.sgroup, s.step, 0u, 0u, 0u), 0u, key);
#pragma unroll
  for (int i = 0; i < K; ++i) n[i] = w[i];
  // the paper's shared draw (Sec. 4, step a): lane 0's n, redrawn whether or not it is live
  const uint32_t need = rejected_lanes<K>(n, e, e.shared_n ? 1u : s.live);
  if (need && !redraw_n<K>(n, e, s.sgroup, s.step, need, key, s.redraws)) {
    errors |= kErrRedraw;
    s.done = true;
    return false;
  }
  if (e.shared_n) {
#pragma unroll
    for (int i = 0; i < K; ++i) n[i] = 0u - (n[i] & 1u);
  }

  // (2) the clock: the candidate time of this step's event, snapshots, t_end
  Clock<PROD> nx;
  bool crossed = clock_advance(s.clk, nx, w[K], w[K + 1], e, precision);
  while (crossed) {
    if (s.snap >= p.n_snap) {  // t_end passed: the event is not applied
      s.done = true;
      return false;
    }
    capture(s.snap);
    ++s.snap;
    nx.aim(thr[s.snap]);
    if constexpr (PROD) crossed = clock_crosses(nx);
    else crossed = clock_crosses(nx, precision);
  }
  s.clk = nx;
  return true;
}

// Step (4) of a group step: thinning of the reactions with k_r < k_max, for the first RN reactions
// (xi beyond the network's R are zero): U (q bits, most significant first, from word K+2 of w
// on, then further Philox calls of the step) < T_r keeps the event.
template <int K, int RN, bool PROD>
__device__ __forceinline__ void general_thin(uint32_t (&xi)[RN], const uint32_t (&w)[4 * GeneralShape<K>::NC0],
                                             const Ensemble& e, const GeneralState<PROD>& s) {
  if (!e.thin) return;
  constexpr int NC0 = GeneralShape<K>::NC0;
  const PhiloxKey key{(uint32_t)e.seed, (uint32_t)(e.seed >> 32)};
  uint32_t tested = 0u;
#pragma unroll
  for (int r = 0; r < RN; ++r)
    if (!((e.thin_always >> r) & 1u)) tested |= xi[r];
  uint32_t und = tested & s.live, rej = tested & ~s.live;
  const int q = e.thin_bits;
  auto bit = [&](int i, uint32_t word) {
    const int pos = q - 1 - i;
    uint32_t tb = 0u;
#pragma unroll
    for (int r = 0; r < RN; ++r)
      if ((((unsigned long long)e.thin_T[r] >> pos) & 1ull) != 0ull) tb |= xi[r];
    const uint32_t lower = und & ~word & tb;
    const uint32_t higher = und & word & ~tb;
    rej |= higher;
    und &= ~(lower | higher);
  };
  int i = 0;
#pragma unroll
  for (int k = K + 2; k < 4 * NC0; ++k)
    if (k - (K + 2) < q) bit(i++, w[k]);
  for (uint32_t call = NC0; und != 0u && i < q; ++call) {
    const uint4 rw = philox4x32_10(stream_counter(s.sgroup, s.step, 0u, 0u, call), key);
    const uint32_t wv[4] = {rw.x, rw.y, rw.z, rw.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (i < q) bit(i++, wv[j]);
  }
  rej |= und;  // U == T: not below
#pragma unroll
  for (int r = 0; r < RN; ++r) xi[r] &= ~rej;
}

// One group step (see the file header).
template <int K, bool PROD>
__device__ __forceinline__ void general_step(const FrankLaunch& p, GeneralState<PROD>& s, const Ensemble& e,
                                             const Threshold* thr, const CountPlanes& c, unsigned int* s_hist,
                                             unsigned int& errors) {
  using Sh = GeneralShape<K>;
  const Network& net = p.net;
  const int B = count_planes(e);
  uint32_t n[K], w[4 * Sh::NC0];
  if (!general_draw<K, PROD>(p, s, e, thr, n, w, errors,
                             [&](int snap) { general_capture<K, PROD>(p, s, e, snap, c, s_hist); }))
    return;

  // (3) the CDF walk over the reactions in order: xi_r = [S_{r-1} <= n < S_r], S_r = sum_{p<=r} h_p,
  // as the borrow of n - S_{r-1} - h_r
  uint32_t xi[kMaxReactions];
  {
#pragma unroll 1
    for (int r = 0; r < net.R; ++r) {
      uint32_t h[K];
      if (net.incremental) {
#pragma unroll
        for (int i = 0; i < K; ++i) h[i] = c.h(r, i);
      } else {
        general_propensity<K>(h, net, r, c, B);
      }
      const uint32_t x = sub_borrow(n, h);
      // (a run-time r cannot index a register array: place x by an unrolled compare)
#pragma unroll
      for (int q = 0; q < kMaxReactions; ++q)
        if (q == r) xi[q] = x;
    }
#pragma unroll
    for (int q = 0; q < kMaxReactions; ++q)
      if (q >= net.R) xi[q] = 0u;
  }

  // (4) thinning for k_r < k_max
  general_thin<K>(xi, w, e, s);

  // (5) the counts: x_s += sum_r xi_r nu_rs (nu in [-2, 2]: three two's-complement planes)
  uint32_t fired = 0u;
#pragma unroll
  for (int r = 0; r < kMaxReactions; ++r) fired |= xi[r];
  ++s.step;
  if (!fired) return;
  // the change of every species in every lane
  for (int sp = 0; sp < net.S; ++sp) {
    uint32_t d[3] = {0u, 0u, 0u};
    if ((net.changes >> sp) & 1u) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const unsigned int sel = net.nu_bits[sp][b];
#pragma unroll
        for (int r = 0; r < kMaxReactions; ++r)
          if ((sel >> r) & 1u) d[b] |= xi[r];
      }
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) c.change(sp, b) = d[b];
  }
  // incremental mode: h_r += its change, from the counts before the event
  if (net.incremental)
    for (int r = 0; r < net.R; ++r) general_increment<K>(net, r, c);
  // the counts: x_s += d_s
  for (int sp = 0; sp < net.S; ++sp) {
    const uint32_t d[3] = {c.change(sp, 0), c.change(sp, 1), c.change(sp, 2)};
    if (!(d[0] | d[1] | d[2])) continue;
    constexpr int BM = Sh::BM;
    uint32_t x[BM];
    load_planes(x, c, sp);
    uint32_t carry = 0u;
#pragma unroll
    for (int i = 0; i < BM; ++i) {
      const uint32_t di = d[i < 2 ? i : 2];
      c.at(sp, i) = bs::xor3(x[i], di, carry);
      carry = bs::maj(x[i], di, carry);
    }
    for (int i = BM; i < B; ++i) {  // counts wider than the products read (first-order networks)
      const uint32_t xv = c.at(sp, i);
      c.at(sp, i) = bs::xor3(xv, d[2], carry);
      carry = bs::maj(xv, d[2], carry);
    }
  }
  s.reactions += (unsigned)__popc(fired);

  // (6) absorption
  const uint32_t now_live = general_live<K>(net, e, c) & s.live;
  uint32_t newly = s.live & ~now_live;
  if (newly) {
    const double tn = s.clk.time(e, p.precision);
    s.lane_steps += (unsigned long long)__popc(newly) * s.step;
    const long long row0 = general_row0(s.sgroup, e);
    while (newly) {
      const int l = __ffs(newly) - 1;
      newly &= newly - 1;
      p.t_abs[row0 + l] = tn;
    }
    s.live = now_live;
    if (!s.live) {
      s.done = true;
      for (; s.snap < p.n_snap; ++s.snap) general_capture<K, PROD>(p, s, e, s.snap, c, s_hist);
    }
  }
}

// Outputs of a finished group: final counts, outcomes, per-ensemble tallies, counters.
// count(s, l) reads species s of lane l.
template <bool PROD, class Count>
__device__ __forceinline__ void finish_counts(const FrankLaunch& p, GeneralState<PROD>& s, const Ensemble& e,
                                              Count&& count) {
  const Network& net = p.net;
  unsigned long long outc[4] = {0, 0, 0, 0};
  const long long row0 = general_row0(s.sgroup, e);
  for (int l = 0; l < s.nvalid; ++l) {
    int* o = p.final_counts + (row0 + l) * net.S;
    int nz = 0, who = -1;
    for (int sp = 0; sp < net.S; ++sp) {
      const int v = count(sp, l);
      o[sp] = v;
      if (v) {
        ++nz;
        who = sp;
      }
    }
    signed char oc = -1;
    if (!((s.live >> l) & 1u)) {
      oc = nz == 1 ? (signed char)who : (signed char)-2;
      outc[(nz == 1 && who < 3) ? who : 3] += 1;  // [3]: another species, or several left
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
  s.lane_steps += (unsigned long long)__popc(s.live) * s.step;  // lanes that never absorbed
  atomicAdd(&p.counters[kGroupSteps], s.step);
  atomicAdd(&p.counters[kLaneSteps], s.lane_steps);
  atomicAdd(&p.counters[kReactions], s.reactions);
  atomicAdd(&p.counters[kNullLaneSteps], s.lane_steps - s.reactions);
  if (s.redraws) atomicAdd(&p.counters[kRedrawRounds], (unsigned long long)s.redraws);
  atomicAdd(&p.counters[kAbsorbed], (unsigned long long)__popc(s.valid & ~s.live));
  atomicAdd(&p.counters[kGroupsDone], 1ull);
  atomicMax(&p.counters[kMaxGroupSteps], s.step);
}

template <int K, bool PROD>
__device__ __forceinline__ void general_finish(const FrankLaunch& p, GeneralState<PROD>& s, const Ensemble& e,
                                               const CountPlanes& c) {
  const int B = count_planes(e);
  finish_counts(p, s, e, [&](int sp, int l) { return lane_count(c, sp, B, l); });
}

// Planes stored per species: enough for the products' reads and for the counts themselves.
__host__ __device__ constexpr int general_planes(int BM, int B) { return BM > B ? BM : B; }

// The persistent loop of the general kernels: the queue, warp-synchronous loop and histogram
// handling of the Frank kernel.  init(s, e, thr, group, ens, s_hist) sets up a group,
// step(s, e, thr, s_hist, errors) runs one step, finish(s, e) writes a finished group's outputs.
// The histogram (single ensemble) is the first n_snap * 65 words of the dynamic shared memory.
template <bool BATCH, bool PROD, class Init, class Step, class Finish>
__device__ __forceinline__ void general_queue(const FrankLaunch& p, unsigned int* s_mem, Init&& init, Step&& step,
                                              Finish&& finish) {
  const bool smem_hist = !BATCH && p.n_snap > 0;
  unsigned int* s_hist = smem_hist ? s_mem : nullptr;
  const int hist_words = smem_hist ? p.n_snap * kHistBins : 0;
  if (smem_hist) {
    for (int i = threadIdx.x; i < hist_words; i += blockDim.x) s_mem[i] = 0u;
    __syncthreads();
  }
  unsigned int errors = 0u;
  GeneralState<PROD> s;
  s.done = true;
  bool active = false, exhausted = false;
  const Threshold* thr = p.thr;
  for (;;) {
    if (!active && !exhausted) {
      const long long item = (long long)atomicAdd(p.queue, 1ull) + p.item_begin;
      if (item >= p.item_end) {
        exhausted = true;
      } else if (!BATCH) {
        init(s, p.ens, thr, item, 0, s_hist);
        active = true;
      } else {
        const int ei = p.item_ens[item];
        thr = p.thr + (long long)ei * (p.n_snap + 1);
        init(s, p.ens_table[ei], thr, (long long)p.item_group[item], ei, (unsigned int*)nullptr);
        active = true;
      }
    }
    if (__all_sync(0xFFFFFFFFu, exhausted && !active)) break;
    if (active) {
      const Ensemble& e = BATCH ? p.ens_table[s.ens] : p.ens;
      if (!s.done) step(s, e, thr, s_hist, errors);
      if (s.done) {
        finish(s, e);
        active = false;
      }
    }
    __syncwarp();
  }
  const unsigned int err = __reduce_or_sync(0xFFFFFFFFu, errors);
  if ((threadIdx.x & 31) == 0 && err) atomicOr(p.status, err);
  if (smem_hist) {
    __syncthreads();
    for (int i = threadIdx.x; i < hist_words; i += blockDim.x)
      if (s_mem[i]) atomicAdd(&p.hist[i], (unsigned long long)s_mem[i]);
  }
}

// The general kernel with its planes in shared memory.  Dynamic shared memory: the histogram
// (single ensemble), the count planes of every thread of the block, the scratch words of every
// thread, and in incremental mode the K planes of every h_r of every thread.
template <int K, bool BATCH, bool PROD>
__global__ void __launch_bounds__(256) general_kernel(const __grid_constant__ FrankLaunch p) {
  extern __shared__ unsigned int s_mem[];
  const int hist_words = (!BATCH && p.n_snap > 0) ? p.n_snap * kHistBins : 0;
  const int planes = general_planes(GeneralShape<K>::BM, p.net.B);
  const int count_words = p.net.S * planes, h_words = p.net.incremental ? p.net.R * K : 0;
  uint32_t* const warp_base = s_mem + hist_words + (threadIdx.x >> 5) * 32 * (count_words + kGeneralScratch + h_words) +
                              (threadIdx.x & 31);
  const CountPlanes c{warp_base, warp_base + 32 * count_words, warp_base + 32 * (count_words + kGeneralScratch),
                      planes, K};
  general_queue<BATCH, PROD>(
      p, s_mem,
      [&](GeneralState<PROD>& s, const Ensemble& e, const Threshold* thr, long long group, int ens,
          unsigned int* s_hist) { general_init<K, PROD>(p, s, e, thr, group, ens, c, s_hist); },
      [&](GeneralState<PROD>& s, const Ensemble& e, const Threshold* thr, unsigned int* s_hist,
          unsigned int& errors) { general_step<K, PROD>(p, s, e, thr, c, s_hist, errors); },
      [&](GeneralState<PROD>& s, const Ensemble& e) { general_finish<K, PROD>(p, s, e, c); });
}

}  // namespace bitssa
