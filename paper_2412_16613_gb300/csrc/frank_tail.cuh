// frank_tail.cuh -- the last groups of a warp, one run per thread.
//
// Late in a launch the work queue is empty and a warp of the one-thread kernel holds only a
// few groups that are still running; each of its steps then costs the latency of the whole
// bit-sliced step (about 1500-3000 cycles) however few lanes are live.  Such a warp hands its
// groups (at most kTailSlots) to this routine, which lays them out by run instead of by
// plane: thread l holds run l of every group as plain integers (L, D, with A = N - L - D),
// and thread i also keeps the scalars of group i (its stream index, step, clock, next
// snapshot).  One step of every group then takes:
//   - the Philox calls of all groups, spread over the warp, into shared memory;
//   - per group, a 32 x 32 bit transpose of its words (five shuffle stages), after which
//     thread l holds its own n = sum_i bit_l(w_i) 2^i; the redraw, when a lane is rejected,
//     replaces the bits from the highest one where n and lambda_int differ (Sec. 3, step 5(i)
//     with the partial redraw of the bit-sliced kernel);
//   - the clocks of all groups at once, each on its own thread (the same integer product or
//     floating-point clock as the bit-sliced kernel);
//   - per run, h_1 = A L, h_2 = A D, h_3 = L D (Eq. equation-as), the CDF walk n < S_r
//     (Sec. 3, step 5) and the count update of the fired reaction (Eq. equation-v).
// The words, the integer rule and the clock are those of the bit-sliced step, so the runs,
// snapshots and absorption times are the same bit for bit.  Groups whose ensemble thins
// reactions (k_r < k_max) stay on the bit-sliced path.
#pragma once

#include <cstdint>

#include "frank_kernel.cuh"

namespace bitssa {

constexpr int kTailSlots = 8;

// A 32 x 32 bit transpose across the warp: thread r holds row r (bit c = entry (r, c)); on
// return thread `lane` holds column `lane` (bit r = entry (r, lane)).  Each stage swaps the
// off-diagonal j x j blocks of every 2j x 2j block.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
#pragma unroll
  for (int j = 16; j >= 1; j >>= 1) {
    const uint32_t m = j == 16 ? 0x0000FFFFu : j == 8 ? 0x00FF00FFu : j == 4 ? 0x0F0F0F0Fu
                     : j == 2 ? 0x33333333u : 0x55555555u;
    const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, j);
    const bool up = (lane & j) != 0;
    const uint32_t moved = up ? (y >> j) : (y << j);
    const uint32_t keep = up ? ~m : m;
    x = (x & keep) | (moved & ~keep);
  }
  return x;
}

// Position of the k-th set bit of `mask` (k = 0 the lowest); mask must have more than k bits set.
__device__ __forceinline__ int nth_set_bit(uint32_t mask, int k) {
  for (int j = 0; j < k; ++j) mask &= mask - 1u;
  return __ffs((int)mask) - 1;
}

// arr[i] for a run-time i, without indexing a register array at run time.
template <typename T, int N>
__device__ __forceinline__ T pick(const T (&arr)[N], int i) {
  T v = arr[0];
#pragma unroll
  for (int k = 1; k < N; ++k) v = i == k ? arr[k] : v;
  return v;
}
template <typename T, int N>
__device__ __forceinline__ void put(T (&arr)[N], int i, T v) {
#pragma unroll
  for (int k = 0; k < N; ++k) arr[k] = i == k ? v : arr[k];
}

// Warp sum of a 64-bit value (all 32 threads).
__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
  const unsigned long long lo = __reduce_add_sync(0xFFFFFFFFu, (unsigned int)(v & 0xFFFFFFFFull));
  const unsigned long long mid = __reduce_add_sync(0xFFFFFFFFu, (unsigned int)((v >> 32) & 0xFFFFull));
  const unsigned long long hi = __reduce_add_sync(0xFFFFFFFFu, (unsigned int)(v >> 48));
  return lo + (mid << 32) + (hi << 48);
}

__device__ __forceinline__ unsigned long long shfl64(unsigned long long v, int src) {
  const uint32_t lo = __shfl_sync(0xFFFFFFFFu, (uint32_t)v, src);
  const uint32_t hi = __shfl_sync(0xFFFFFFFFu, (uint32_t)(v >> 32), src);
  return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ double shfl_double(double v, int src) {
  return __longlong_as_double((long long)shfl64((unsigned long long)__double_as_longlong(v), src));
}

// Group i's clock moved to thread i (owner) from the thread that ran the group (src).
__device__ __forceinline__ void shfl_clock(Clock<true>& dst, const Clock<true>& c, int src) {
  dst.M = shfl64(c.M, src);
  dst.E = (long long)shfl64((unsigned long long)c.E, src);
}
__device__ __forceinline__ void shfl_clock(Clock<false>& dst, const Clock<false>& c, int src) {
  dst.t = shfl_double(c.t, src);
  dst.t_f = __shfl_sync(0xFFFFFFFFu, c.t_f, src);
  dst.c_f = __shfl_sync(0xFFFFFFFFu, c.c_f, src);
}

// Words of shared memory a warp needs: the attempt's calls of every group.
template <int K>
struct TailShape {
  static constexpr int NC0 = FrankShape<K>::NC0;
  static constexpr int NCR = FrankShape<K>::NCR;
  static constexpr int W = 4 * NC0;                  // words per group
  static constexpr int kWarpWords = kTailSlots * W;  // words per warp
};

// Runs the warp's live groups (the threads with `active` set, at most kTailSlots of them) to
// the end, writing every output a finished group writes.  Called by all 32 threads of the warp
// together; returns when every one of those groups has finished.
template <int K, bool BATCH, bool PROD, bool ADAPT>
__device__ __forceinline__ void tail_run(const FrankLaunch& p, const GroupState<K, PROD>& s, bool active,
                                      unsigned int* s_hist, uint32_t* wbuf, unsigned int& errors) {
  using Sh = FrankShape<K>;
  constexpr int B = Sh::B, WP = Sh::WP;
  constexpr int NW = TailShape<K>::W, NC0 = TailShape<K>::NC0, NCR = TailShape<K>::NCR;
  constexpr uint32_t FULL = 0xFFFFFFFFu;
  constexpr uint32_t kMaskK = K >= 32 ? 0xFFFFFFFFu : ((1u << K) - 1u);
  const int lane = threadIdx.x & 31;
  const int precision = p.precision;

  const uint32_t alive = __ballot_sync(FULL, active);
  const int nslots = __popc(alive);
  if (lane == 0) atomicOr(&p.counters[kLayoutUsed], (unsigned long long)kLayoutTail);

  // the group's counters so far; the rest is counted run by run below
  if (active) {
    atomicAdd(&p.counters[kReactions], s.reactions);
    atomicAdd(&p.counters[kLaneSteps], s.lane_steps);
    atomicAdd(&p.counters[kNullLaneSteps], s.lane_steps - s.reactions);  // modular: the tail adds the rest
    if (s.redraws) atomicAdd(&p.counters[kRedrawRounds], (unsigned long long)s.redraws);
  }

  // ---- owner scalars: thread i < nslots keeps group i (the i-th live thread's group)
  const int src = lane < nslots ? nth_set_bit(alive, lane) : 0;
  // (threads without a group take zeros: the source thread may hold no group at all)
  const bool owner = lane < nslots;
  uint32_t o_sgroup = __shfl_sync(FULL, s.sgroup, src);
  int o_ens = __shfl_sync(FULL, s.ens, src);
  int o_snap = __shfl_sync(FULL, s.snap, src);
  unsigned long long o_step = shfl64(s.step, src);
  Clock<PROD> o_clk;
  shfl_clock(o_clk, s.clk, src);
  if (!owner) {
    o_sgroup = 0u;
    o_ens = o_snap = 0;
    o_step = 0ull;
    o_clk.reset();
  }
  const Threshold* o_thr = BATCH ? p.thr + (long long)o_ens * (p.n_snap + 1) : p.thr;
  o_clk.aim(o_thr[o_snap]);
  int o_j = 0;         // the state-following bound: K - p of the step
  bool o_fail = false; // the group gave up redrawing n

  // ---- lane data: thread l keeps run l of every group (plain integers)
  int tl[kTailSlots], td[kTailSlots];
  uint32_t tlive = 0u, tvalid = 0u;
#pragma unroll
  for (int i = 0; i < kTailSlots; ++i) {
    tl[i] = td[i] = 0;
    if (i < nslots) {  // warp-uniform
      const int g = nth_set_bit(alive, i);
      uint32_t l = 0u, u = 0u;
#pragma unroll
      for (int k = 0; k < B; ++k) l |= ((__shfl_sync(FULL, s.L[k], g) >> lane) & 1u) << k;
#pragma unroll
      for (int k = 0; k < WP; ++k) u |= ((__shfl_sync(FULL, s.U[k], g) >> lane) & 1u) << k;
      const int uv = (int)(u << (32 - WP)) >> (32 - WP);  // sign-extended U = N - 2 (L + D) - 1
      const uint32_t lv = __shfl_sync(FULL, s.live, g);
      const int nv = __shfl_sync(FULL, s.nvalid, g);
      const int ens = __shfl_sync(FULL, s.ens, g);
      const int n_tot = BATCH ? p.ens_table[ens].n_tot : p.ens.n_tot;
      const int x = (n_tot - 1 - uv) / 2;
      tl[i] = (int)l;
      td[i] = x - (int)l;
      if ((lv >> lane) & 1u) tlive |= 1u << i;
      if (lane < nv) tvalid |= 1u << i;
    }
  }

  uint32_t* const W = wbuf;  // [kTailSlots][NW] words of this warp
  uint32_t done = nslots >= 32 ? 0u : (FULL << nslots);  // slots finished (bit i), warp-uniform
  unsigned long long t_react = 0, t_lsteps = 0, t_redraws = 0;

  // the outputs of a finished group (every thread: its own run)
  auto finish = [&](int i, const Ensemble& e) {
    const unsigned long long step = shfl64(o_step, i);
    const int ens = __shfl_sync(FULL, o_ens, i);
    const uint32_t sg = __shfl_sync(FULL, o_sgroup, i);
    const long long row = e.run_offset + ((long long)sg - e.group_base) * 32 + lane;
    const bool valid = (tvalid >> i) & 1u, live = (tlive >> i) & 1u;
    int cls = 3;
    if (valid) {
      const int l = pick(tl, i), d = pick(td, i), a = e.n_tot - l - d;
      int* o = p.final_counts + row * p.n_species;
      o[p.perm[0]] = l;
      o[p.perm[1]] = d;
      o[p.perm[2]] = a;
      signed char oc = -1;
      if (!live) {
        const int nz = (l != 0) + (d != 0) + (a != 0);
        oc = nz == 1 ? (signed char)(l ? p.perm[0] : (d ? p.perm[1] : p.perm[2])) : (signed char)-2;
        cls = nz == 1 ? (int)oc : 3;
      } else {
        p.t_abs[row] = __longlong_as_double(0x7FF0000000000000ll);
        t_lsteps += step;  // runs that never absorbed
      }
      p.outcome[row] = oc;
    }
    if (p.ens_absorbed) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const unsigned int c = __reduce_add_sync(FULL, (valid && cls == k) ? 1u : 0u);
        if (lane == 0 && c) atomicAdd(&p.ens_absorbed[(long long)ens * 4 + k], (unsigned long long)c);
      }
    }
    const unsigned int absorbed = __popc(__ballot_sync(FULL, valid && !live));
    if (lane == 0) {
      atomicAdd(&p.counters[kGroupSteps], step);
      atomicAdd(&p.counters[kAbsorbed], (unsigned long long)absorbed);
      atomicAdd(&p.counters[kGroupsDone], 1ull);
      atomicMax(&p.counters[kMaxGroupSteps], step);
    }
  };
  // the current state of every run of group i into snapshot `snap`
  auto capture_slot = [&](int i, const Ensemble& e, int snap) {
    const int ens = __shfl_sync(FULL, o_ens, i);
    const uint32_t sg = __shfl_sync(FULL, o_sgroup, i);
    if ((tvalid >> i) & 1u) {
      const int l = pick(tl, i), d = pick(td, i), a = e.n_tot - l - d;
      if (s_hist) atomicAdd(&s_hist[snap * kHistBins + ee_bin(l, d)], 1u);
      else atomicAdd(&p.hist[((long long)ens * p.n_snap + snap) * kHistBins + ee_bin(l, d)], 1ull);
      if (p.snap_counts) {
        const long long row = e.run_offset + ((long long)sg - e.group_base) * 32 + lane;
        int* o = p.snap_counts + ((long long)snap * p.n_runs_total + row) * p.n_species;
        o[p.perm[0]] = l;
        o[p.perm[1]] = d;
        o[p.perm[2]] = a;
      }
    }
  };
  auto ens_of = [&](int i) -> const Ensemble& {
    if constexpr (BATCH) return p.ens_table[__shfl_sync(FULL, o_ens, i)];
    else return p.ens;
  };

  while (done != FULL) {
    const uint32_t lslots = ~done;  // live slots, warp-uniform
    // (0) step budget
    if (p.step_budget > 0) {
      const uint32_t over = __ballot_sync(FULL, ((lslots >> lane) & 1u) && (long long)o_step >= p.step_budget);
      if (over) {
        errors |= kErrTimeout;
#pragma unroll 1
        for (int i = 0; i < kTailSlots; ++i)
          if ((over >> i) & 1u) finish(i, ens_of(i));
        done |= over;
        continue;
      }
    }
    // (1) the words of attempt 0 of every live group, spread over the warp
    const int nlive = __popc(lslots);
    for (int base = 0; base < nlive * NC0; base += 32) {
      const int q = base + lane;
      const bool mine = q < nlive * NC0;
      const int k = mine ? q / NC0 : 0;
      const int c = mine ? q - k * NC0 : 0;
      const int slot = nth_set_bit(lslots, k);
      const uint32_t sg = __shfl_sync(FULL, o_sgroup, slot & 31);
      const unsigned long long st = shfl64(o_step, slot & 31);
      unsigned long long seed;
      if constexpr (BATCH) seed = p.ens_table[__shfl_sync(FULL, o_ens, slot & 31)].seed;
      else seed = p.ens.seed;
      const PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
      const uint4 r = philox4x32_10(stream_counter(sg, st, 0u, 0u, (uint32_t)c), key);
      if (mine) *reinterpret_cast<uint4*>(&W[slot * NW + 4 * c]) = r;
    }
    __syncwarp();

    // (2) per group: n of every run (transpose), the state-following bound, redraws
    uint32_t tn[kTailSlots];
    uint32_t redo = 0u;  // groups with a run to redraw, warp-uniform
#pragma unroll
    for (int i = 0; i < kTailSlots; ++i) {
      tn[i] = 0u;
      if (!((lslots >> i) & 1u)) continue;
      const Ensemble& e = ens_of(i);
      uint32_t x = lane < NW ? W[i * NW + lane] : 0u;
      x = warp_transpose32(x, lane);
      uint32_t n = x & kMaskK;
      const bool live = (tlive >> i) & 1u;
      const int l = tl[i], d = td[i], a = e.n_tot - l - d;
      const uint32_t S3 = (uint32_t)(a * l) + (uint32_t)(a * d) + (uint32_t)(l * d);
      if constexpr (ADAPT) {
        const uint32_t top = __reduce_max_sync(FULL, live ? S3 : 0u);
        const int bits = 32 - __clz((int)top);
        n &= bits >= 32 ? 0xFFFFFFFFu : ((1u << bits) - 1u);
        if (lane == i) o_j = K - bits;
      }
      tn[i] = n;
      if (e.reject && __any_sync(FULL, live && n >= e.lambda_int)) redo |= 1u << i;
    }
    // groups where a run drew n >= lambda_int: redraws (the bits from the highest one where n
    // and lambda_int differ, from the next attempt of the same stream)
#pragma unroll 1
    for (int i = 0; i < kTailSlots; ++i) {
      if (!((redo >> i) & 1u)) continue;
      const Ensemble& e = ens_of(i);
      const uint32_t lam = e.lambda_int;
      uint32_t n = pick(tn, i);
      bool need = ((tlive >> i) & 1u) && n >= lam;
      const unsigned long long st = shfl64(o_step, i);
      const uint32_t sg = __shfl_sync(FULL, o_sgroup, i);
      const PhiloxKey key{(uint32_t)e.seed, (uint32_t)(e.seed >> 32)};
      for (uint32_t attempt = 1u; __any_sync(FULL, need); ++attempt) {
        if (attempt >= 64u) {  // as the bit-sliced kernel: stop the group with an error
          errors |= kErrRedraw;
          need = false;
          if (lane == i) o_fail = true;
          break;
        }
        ++t_redraws;
        // the calls of this attempt, one per thread, then the same transpose
        uint4 r = make_uint4(0u, 0u, 0u, 0u);
        if (lane < NCR) r = philox4x32_10(stream_counter(sg, st, attempt, 0u, (uint32_t)lane), key);
        const int wsrc = lane >> 2;
        const uint32_t a0 = __shfl_sync(FULL, r.x, wsrc), a1 = __shfl_sync(FULL, r.y, wsrc);
        const uint32_t a2 = __shfl_sync(FULL, r.z, wsrc), a3 = __shfl_sync(FULL, r.w, wsrc);
        const int comp = lane & 3;
        uint32_t xr = comp == 0 ? a0 : comp == 1 ? a1 : comp == 2 ? a2 : a3;
        xr = lane < K ? xr : 0u;
        xr = warp_transpose32(xr, lane) & kMaskK;
        if (need) {
          const int from = n == lam ? 0 : 31 - __clz((int)(n ^ lam));
          const uint32_t low = (1u << from) - 1u;
          n = (n & low) | (xr & ~low);
          need = n >= lam;
        }
      }
      put(tn, i, n);
    }
    // a group that gave up redrawing stops with the error flag set
    {
      const uint32_t bad = __ballot_sync(FULL, ((lslots >> lane) & 1u) && o_fail);
      if (bad) {
#pragma unroll 1
        for (int i = 0; i < kTailSlots; ++i)
          if ((bad >> i) & 1u) finish(i, ens_of(i));
        done |= bad;
      }
    }
    const uint32_t stepping = ~done;

    // (3) the clocks of all groups at once (thread i: group i), snapshots, t_end
    Clock<PROD> nx = o_clk;
    bool crossed = false;
    const bool own = (stepping >> lane) & 1u;
    {
      const Ensemble& eo = BATCH ? p.ens_table[own ? o_ens : 0] : p.ens;
      if (own) {
        const uint32_t wk = W[lane * NW + K], wk1 = W[lane * NW + K + 1];
        if constexpr (ADAPT) crossed = clock_advance(o_clk, nx, wk, wk1, eo, precision, o_j);
        else crossed = clock_advance(o_clk, nx, wk, wk1, eo, precision);
      }
    }
    uint32_t ended = 0u;  // groups whose next event lies beyond t_end
    for (uint32_t cross = __ballot_sync(FULL, own && crossed); cross;) {
#pragma unroll 1
      for (int i = 0; i < kTailSlots; ++i) {
        if (!((cross >> i) & 1u)) continue;
        const int snap = __shfl_sync(FULL, o_snap, i);
        if (snap >= p.n_snap) {
          ended |= 1u << i;
        } else {
          capture_slot(i, ens_of(i), snap);
        }
      }
      // owners move on to the next time point
      bool again = false;
      if (own && ((cross >> lane) & 1u) && !((ended >> lane) & 1u)) {
        ++o_snap;
        const Threshold* thr = BATCH ? p.thr + (long long)o_ens * (p.n_snap + 1) : p.thr;
        nx.aim(thr[o_snap]);
        if constexpr (PROD) again = clock_crosses(nx);
        else again = clock_crosses(nx, precision);
      }
      cross = __ballot_sync(FULL, again);
    }
    if (own && !((ended >> lane) & 1u)) o_clk = nx;
    if (ended) {
#pragma unroll 1
      for (int i = 0; i < kTailSlots; ++i)
        if ((ended >> i) & 1u) finish(i, ens_of(i));
      done |= ended;
    }

    // (4) per group: the CDF walk, the update, absorption
    const uint32_t firing = stepping & ~ended;
    if (own && !((ended >> lane) & 1u)) ++o_step;
    uint32_t absorbed_all = 0u;
#pragma unroll
    for (int i = 0; i < kTailSlots; ++i) {
      if (!((firing >> i) & 1u)) continue;
      const Ensemble& e = ens_of(i);
      const bool live = (tlive >> i) & 1u;
      int l = tl[i], d = td[i];
      const int a = e.n_tot - l - d;
      const uint32_t h1 = (uint32_t)(a * l), h2 = (uint32_t)(a * d), h3 = (uint32_t)(l * d);
      const uint32_t n = tn[i];
      const uint32_t S1 = h1, S2 = h1 + h2, S3 = S2 + h3;
      const int r = n < S1 ? 0 : (n < S2 ? 1 : (n < S3 ? 2 : -1));
      bool now_live = live;
      if (r >= 0) {  // only live runs have S3 > 0
        l += r == 0 ? 1 : (r == 2 ? -1 : 0);
        d += r == 1 ? 1 : (r == 2 ? -1 : 0);
        tl[i] = l;
        td[i] = d;
        ++t_react;
        const int a2 = e.n_tot - l - d;
        now_live = (a2 * l + a2 * d + l * d) != 0;
      }
      const uint32_t newly_mask = __ballot_sync(FULL, live && !now_live);
      if (newly_mask) {
        const unsigned long long step = shfl64(o_step, i);
        double tn_abs = 0.0;
        if (lane == i) tn_abs = o_clk.time(e, precision);  // the owner's clock: the event's time
        tn_abs = shfl_double(tn_abs, i);
        if (live && !now_live) {
          t_lsteps += step;
          tlive &= ~(1u << i);
        }
        const uint32_t sg = __shfl_sync(FULL, o_sgroup, i);
        if ((newly_mask >> lane) & 1u) p.t_abs[e.run_offset + ((long long)sg - e.group_base) * 32 + lane] = tn_abs;
        if (!__any_sync(FULL, (tlive >> i) & 1u)) absorbed_all |= 1u << i;
      }
    }
    if (absorbed_all) {
      // every run of the group has absorbed: the remaining snapshots hold the final state
#pragma unroll 1
      for (int i = 0; i < kTailSlots; ++i) {
        if (!((absorbed_all >> i) & 1u)) continue;
        const Ensemble& e = ens_of(i);
        for (int snap = __shfl_sync(FULL, o_snap, i); snap < p.n_snap; ++snap) capture_slot(i, e, snap);
        finish(i, e);
      }
      done |= absorbed_all;
    }
    __syncwarp();
  }

  // the counters of the runs stepped here
  const unsigned long long react = warp_sum64(t_react);
  const unsigned long long lsteps = warp_sum64(t_lsteps);
  if (lane == 0) {
    atomicAdd(&p.counters[kReactions], react);
    atomicAdd(&p.counters[kLaneSteps], lsteps);
    atomicAdd(&p.counters[kNullLaneSteps], lsteps - react);
    if (t_redraws) atomicAdd(&p.counters[kRedrawRounds], t_redraws);
  }
}

}  // namespace bitssa
