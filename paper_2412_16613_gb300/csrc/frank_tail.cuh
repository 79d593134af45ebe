// frank_tail.cuh -- the last groups of a warp, one run per thread.
//
// Late in a launch the work queue is empty and a warp of the one-thread kernel holds only a
// few groups that are still running; each of its steps then costs the latency of the whole
// bit-sliced step (about 2500 cycles on GB300) however few lanes are live.  Such a warp hands
// its groups (at most kTailSlots) to tail_run, which lays them out by run instead of by plane:
// every thread keeps the scalars of every group (stream index, step, clock, next snapshot), so
// that every decision on them is warp-uniform, and thread l keeps run l of each group as plain
// integers (L, D, with A = N - L - D).
//
// A group's random words do not depend on its state, so tail_lockstep draws them kTailDepth
// steps ahead: the Philox calls of those steps for every group, spread over the warp, into
// shared memory, then per step a 32 x 32 bit transpose of the step's words (five shuffle
// stages, the transposes of a group's steps side by side), after which thread l holds its own
// n = sum_i bit_l(w_i) 2^i.  Then, step by step and group by group:
//   - under the state-following bound, n keeps the low p bits, p from the largest S_3 of the
//     group's live runs (a warp maximum); under the paper's bound a run with n >= lambda_int
//     replaces the bits from the highest one where n and lambda_int differ with those of the
//     next attempt (Sec. 3, step 5(i) with the partial redraw of the bit-sliced kernel);
//   - the group's clock, the same integer product or floating-point clock as the bit-sliced
//     kernel, computed alike on every thread;
//   - per run, h_1 = A L, h_2 = A D, h_3 = L D (Eq. equation-as), the CDF walk n < S_r
//     (Sec. 3, step 5) and the count update of the fired reaction (Eq. equation-v).
// Rare events (a snapshot time or t_end passed, runs absorbed, the step budget, redraws given
// up) leave tail_lockstep and are handled by tail_run one group at a time.  The words, the
// integer rule and the clock are those of the bit-sliced step, so the runs, snapshots and
// absorption times are the same bit for bit.  Groups whose ensemble thins reactions
// (k_r < k_max) stay on the bit-sliced path.
#pragma once

#include <cstdint>

#include "frank_kernel.cuh"

namespace bitssa {


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
  static constexpr int W = 4 * NC0;                               // words of one step of a group
  static constexpr int kWarpWords = kTailSlots * kTailDepth * W;  // words per warp
};

// kTailDepth transposes side by side, stage by stage (their shuffles overlap).
__device__ __forceinline__ void warp_transpose32_x4(uint32_t (&x)[kTailDepth], int lane) {
#pragma unroll
  for (int j = 16; j >= 1; j >>= 1) {
    const uint32_t m = j == 16 ? 0x0000FFFFu : j == 8 ? 0x00FF00FFu : j == 4 ? 0x0F0F0F0Fu
                     : j == 2 ? 0x33333333u : 0x55555555u;
    const bool up = (lane & j) != 0;
    const uint32_t keep = up ? ~m : m;
    uint32_t y[kTailDepth];
#pragma unroll
    for (int d = 0; d < kTailDepth; ++d) y[d] = __shfl_xor_sync(0xFFFFFFFFu, x[d], j);
#pragma unroll
    for (int d = 0; d < kTailDepth; ++d) {
      const uint32_t moved = up ? (y[d] >> j) : (y[d] << j);
      x[d] = (x[d] & keep) | (moved & ~keep);
    }
  }
}

// The groups a warp finishes one run per thread.  Every thread keeps the scalars of every
// group (so that every decision on them is warp-uniform and needs no shuffle) and, for each
// group, the counts and flags of its own run (run `lane`).
template <bool PROD>
struct TailGroups {
  uint32_t sg[kTailSlots];              // stream group index
  int ens[kTailSlots];                  // ensemble
  int snap[kTailSlots];                 // next snapshot
  unsigned long long step[kTailSlots];
  Clock<PROD> clk[kTailSlots];
  int l[kTailSlots], d[kTailSlots];     // this thread's run: L and D (A = N - L - D)
  uint32_t live, valid;                 // bit s: this thread's run of group s can react / exists
  unsigned long long react, lsteps, redraws;  // this thread's share of the run counters
};

// arr[i] for a run-time i, without indexing a register array at run time.
template <typename T, int N>
__device__ __forceinline__ T pick(const T (&arr)[N], int i) {
  T v = arr[0];
#pragma unroll
  for (int k = 1; k < N; ++k)
    if (i == k) v = arr[k];
  return v;
}

template <typename T, int N>
__device__ __forceinline__ void put(T (&arr)[N], int i, T v) {
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (i == k) arr[k] = v;
}

// Moves the groups not in `fin` to the front, in order.
template <bool PROD>
__device__ __forceinline__ void tail_compact(TailGroups<PROD>& g, uint32_t fin, int ns) {
  const uint32_t keep = ~fin & ((1u << ns) - 1u);
  TailGroups<PROD> o = g;
  uint32_t live = 0u, valid = 0u;
#pragma unroll
  for (int dst = 0; dst < kTailSlots; ++dst) {
    if (dst < __popc(keep)) {
      const int src = nth_set_bit(keep, dst);
      g.sg[dst] = pick(o.sg, src);
      g.ens[dst] = pick(o.ens, src);
      g.snap[dst] = pick(o.snap, src);
      g.step[dst] = pick(o.step, src);
      g.clk[dst] = pick(o.clk, src);
      g.l[dst] = pick(o.l, src);
      g.d[dst] = pick(o.d, src);
      live |= ((o.live >> src) & 1u) << dst;
      valid |= ((o.valid >> src) & 1u) << dst;
    }
  }
  g.live = live;
  g.valid = valid;
}
// What stopped a run of tail_lockstep: the groups concerned (bits), and for an absorption the
// groups in which this thread's run absorbed.
struct TailEvent {
  int kind;       // kTailBudget, kTailRedraw, kTailCross, kTailAbsorb
  uint32_t slots;
  uint32_t mine;
  unsigned int rd[kTailSlots];  // kTailCross, kTailRedraw: each group's redraw rounds in the step
};
enum { kTailBudget = 0, kTailRedraw = 1, kTailCross = 2, kTailAbsorb = 3 };

// NS groups stepped in lockstep until a rare event: a group at its step budget or out of
// redraws (before its step), a group whose candidate event time passes a snapshot time or
// t_end (before any group commits the step), or runs that absorbed (after every group has
// committed the step).  A group's state changes only when it commits a step, so the caller
// handles the event and calls again: the groups that did not commit take up the same step,
// with the same words.
template <int K, bool BATCH, bool PROD, bool ADAPT, int NS>
__device__ __forceinline__ TailEvent tail_lockstep(const FrankLaunch& p, TailGroups<PROD>& g, uint32_t* W) {
  constexpr int NW = TailShape<K>::W, NC0 = TailShape<K>::NC0, NCR = TailShape<K>::NCR;
  constexpr int D = kTailDepth;
  constexpr uint32_t FULL = 0xFFFFFFFFu;
  constexpr uint32_t kMaskK = (1u << K) - 1u;
  const int lane = threadIdx.x & 31;
  const int precision = p.precision;
  const Ensemble* es[NS];
  int ntot[NS];
  bool rej[NS];
  uint32_t lam[NS];
  bool any_reject = false;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    es[s] = BATCH ? &p.ens_table[g.ens[s]] : &p.ens;
    ntot[s] = es[s]->n_tot;
    rej[s] = es[s]->reject != 0;
    lam[s] = es[s]->lambda_int;
    any_reject = any_reject || rej[s];
    const Threshold* th = BATCH ? p.thr + (long long)g.ens[s] * (p.n_snap + 1) : p.thr;
    g.clk[s].aim(th[g.snap[s]]);
  }
  for (;;) {
    // ---- the words of steps step[s] .. step[s] + D - 1 of every group: one Philox call per
    // thread and pass, stored by group and step
#pragma unroll
    for (int base = 0; base < NS * D * NC0; base += 32) {
      const int q = base + lane;
      const int s = q / (D * NC0), rem = q - s * (D * NC0);
      const int dd = rem / NC0, c = rem - dd * NC0;
      uint32_t sg = g.sg[0];
      unsigned long long st = g.step[0], seed = es[0]->seed;
#pragma unroll
      for (int k = 1; k < NS; ++k)
        if (s == k) {
          sg = g.sg[k];
          st = g.step[k];
          seed = es[k]->seed;
        }
      const PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
      const uint4 r = philox4x32_10(stream_counter(sg, st + (unsigned long long)dd, 0u, 0u, (uint32_t)c), key);
      if (q < NS * D * NC0) *reinterpret_cast<uint4*>(&W[(s * D + dd) * NW + 4 * c]) = r;
    }
    __syncwarp();
    // ---- the transposes, side by side: bit i of nr[s][dd] is bit `lane` of word i of the step
    uint32_t nr[NS][D], wk[NS][D], wk1[NS][D];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
      for (int dd = 0; dd < D; ++dd) {
        nr[s][dd] = lane < NW ? W[(s * D + dd) * NW + lane] : 0u;
        wk[s][dd] = W[(s * D + dd) * NW + K];
        wk1[s][dd] = W[(s * D + dd) * NW + K + 1];
      }
      warp_transpose32_x4(nr[s], lane);
    }
    __syncwarp();  // every read of W is done before the next batch writes it

    // ---- the steps, one at a time
    constexpr int kUnroll = NS == 1 ? D : 1;
#pragma unroll kUnroll
    for (int dd = 0; dd < D; ++dd) {
      if (p.step_budget > 0) {
        uint32_t over = 0u;
#pragma unroll
        for (int s = 0; s < NS; ++s)
          if ((long long)g.step[s] >= p.step_budget) over |= 1u << s;
        if (over) return TailEvent{kTailBudget, over, 0u, {}};
      }
      // n of every run; the state-following bound from the group's largest S_3
      uint32_t n[NS];
      int j[NS];
      unsigned int rd[NS];  // redraw rounds of this step per group, counted when it commits
      uint32_t need_mine = 0u;  // bit s: this thread's run of group s drew n >= lambda_int
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        rd[s] = 0u;
        n[s] = pick(nr[s], dd) & kMaskK;
        j[s] = 0;
        const bool live = (g.live >> s) & 1u;
        if constexpr (ADAPT) {
          const int l = g.l[s], d = g.d[s], a = ntot[s] - l - d;
          const uint32_t S3 = (uint32_t)(a * l) + (uint32_t)(a * d) + (uint32_t)(l * d);
          const uint32_t top = __reduce_max_sync(FULL, live ? S3 : 0u);
          const int bits = 32 - __clz((int)top);
          n[s] &= (1u << bits) - 1u;
          j[s] = K - bits;
        }
        if (rej[s] && live && n[s] >= lam[s]) need_mine |= 1u << s;
      }
      const uint32_t redo = any_reject ? __reduce_or_sync(FULL, need_mine) : 0u;
      if (redo) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          if (!((redo >> s) & 1u)) continue;
          // rare: redraws from the highest bit where n and lambda_int differ
          const PhiloxKey key{(uint32_t)es[s]->seed, (uint32_t)(es[s]->seed >> 32)};
          bool need = (need_mine >> s) & 1u;
          for (uint32_t attempt = 1u; __any_sync(FULL, need); ++attempt) {
            if (attempt >= 64u) {
              TailEvent ev{kTailRedraw, 1u << s, 0u, {}};
#pragma unroll
              for (int k = 0; k < NS; ++k) ev.rd[k] = rd[k];
              return ev;
            }
            ++rd[s];
            uint4 r = make_uint4(0u, 0u, 0u, 0u);
            if (lane < NCR) r = philox4x32_10(stream_counter(g.sg[s], g.step[s], attempt, 0u, (uint32_t)lane), key);
            const int wsrc = lane >> 2;
            const uint32_t a0 = __shfl_sync(FULL, r.x, wsrc), a1 = __shfl_sync(FULL, r.y, wsrc);
            const uint32_t a2 = __shfl_sync(FULL, r.z, wsrc), a3 = __shfl_sync(FULL, r.w, wsrc);
            const int comp = lane & 3;
            uint32_t xr = comp == 0 ? a0 : comp == 1 ? a1 : comp == 2 ? a2 : a3;
            xr = lane < K ? xr : 0u;
            xr = warp_transpose32(xr, lane) & kMaskK;
            if (need) {
              const int from = n[s] == lam[s] ? 0 : 31 - __clz((int)(n[s] ^ lam[s]));
              const uint32_t low = (1u << from) - 1u;
              n[s] = (n[s] & low) | (xr & ~low);
              need = n[s] >= lam[s];
            }
          }
        }
      }
      // the clocks (each the same on every thread): a snapshot time or t_end passed stops here
      Clock<PROD> nx[NS];
      uint32_t cross = 0u;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        bool c;
        if constexpr (ADAPT) c = clock_advance(g.clk[s], nx[s], pick(wk[s], dd), pick(wk1[s], dd), *es[s], precision, j[s]);
        else c = clock_advance(g.clk[s], nx[s], pick(wk[s], dd), pick(wk1[s], dd), *es[s], precision);
        cross |= c ? 1u << s : 0u;
      }
      if (cross) {
        TailEvent ev{kTailCross, cross, 0u, {}};
#pragma unroll
        for (int k = 0; k < NS; ++k) ev.rd[k] = rd[k];
        return ev;
      }
      // commit: the CDF walk and the update of every run (only live runs have S_3 > 0)
      uint32_t mine = 0u;  // bit s: this thread's run of group s absorbed at this step
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        g.redraws += rd[s];
        g.clk[s] = nx[s];
        ++g.step[s];
        const int n_tot = ntot[s];
        const bool live = (g.live >> s) & 1u;
        int l = g.l[s], d = g.d[s];
        const int a = n_tot - l - d;
        const uint32_t S1 = (uint32_t)(a * l), S2 = S1 + (uint32_t)(a * d), S3 = S2 + (uint32_t)(l * d);
        const bool f1 = n[s] < S1, f12 = n[s] < S2, f123 = n[s] < S3;
        const bool f3 = f123 && !f12, f2 = f12 && !f1;
        l += (int)f1 - (int)f3;
        d += (int)f2 - (int)f3;
        g.l[s] = l;
        g.d[s] = d;
        g.react += f123 ? 1u : 0u;
        // a run is absorbed when a single species is left (every rate is k_max here)
        if (live && (l != 0) + (d != 0) + (n_tot - l - d != 0) < 2) mine |= 1u << s;
      }
      g.live &= ~mine;
      const uint32_t newly = __reduce_or_sync(FULL, mine);
      if (newly) return TailEvent{kTailAbsorb, newly, mine, {}};
    }
  }
}

// The warp's running groups (the threads with `active` set, at most kTailSlots of them) as
// tail_run takes them: every group's scalars on every thread, and run `lane` of each group as
// integers.  Inlined into the kernel (it reads the bit-sliced state in registers); also hands
// over the counters the groups have so far.
template <int K, bool BATCH, bool PROD>
__device__ __forceinline__ TailGroups<PROD> tail_take(const FrankLaunch& p, const GroupState<K, PROD>& s, bool active,
                                                      int& ns) {
  using Sh = FrankShape<K>;
  constexpr int B = Sh::B, WP = Sh::WP;
  constexpr uint32_t FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const uint32_t alive = __ballot_sync(FULL, active);
  ns = __popc(alive);
  if (lane == 0) atomicOr(&p.counters[kLayoutUsed], (unsigned long long)kLayoutTail);
  // the group's counters so far; the rest is counted run by run in tail_run
  if (active) {
    atomicAdd(&p.counters[kReactions], s.reactions);
    atomicAdd(&p.counters[kLaneSteps], s.lane_steps);
    atomicAdd(&p.counters[kNullLaneSteps], s.lane_steps - s.reactions);  // modular: the tail adds the rest
    if (s.redraws) atomicAdd(&p.counters[kRedrawRounds], (unsigned long long)s.redraws);
  }
  TailGroups<PROD> g;
  g.live = g.valid = 0u;
  g.react = g.lsteps = g.redraws = 0ull;
#pragma unroll
  for (int k = 0; k < kTailSlots; ++k) {
    g.sg[k] = 0u;
    g.ens[k] = g.snap[k] = g.l[k] = g.d[k] = 0;
    g.step[k] = 0ull;
    g.clk[k].reset();
    if (k < ns) {  // warp-uniform
      const int src = nth_set_bit(alive, k);
      g.sg[k] = __shfl_sync(FULL, s.sgroup, src);
      g.ens[k] = __shfl_sync(FULL, s.ens, src);
      g.snap[k] = __shfl_sync(FULL, s.snap, src);
      g.step[k] = shfl64(s.step, src);
      shfl_clock(g.clk[k], s.clk, src);
      uint32_t l = 0u, u = 0u;
#pragma unroll
      for (int b = 0; b < B; ++b) l |= ((__shfl_sync(FULL, s.L[b], src) >> lane) & 1u) << b;
#pragma unroll
      for (int b = 0; b < WP; ++b) u |= ((__shfl_sync(FULL, s.U[b], src) >> lane) & 1u) << b;
      const int uv = (int)(u << (32 - WP)) >> (32 - WP);  // sign-extended U = N - 2 (L + D) - 1
      const uint32_t lv = __shfl_sync(FULL, s.live, src);
      const int nv = __shfl_sync(FULL, s.nvalid, src);
      const int n_tot = BATCH ? p.ens_table[g.ens[k]].n_tot : p.ens.n_tot;
      const int x = (n_tot - 1 - uv) / 2;
      g.l[k] = (int)l;
      g.d[k] = x - (int)l;
      if ((lv >> lane) & 1u) g.live |= 1u << k;
      if (lane < nv) g.valid |= 1u << k;
    }
  }
  return g;
}

// Runs the ns groups of g (from tail_take) to the end, writing every output a finished group
// writes.  Called by all 32 threads of the warp together; returns the error flags it raised.
// Not inlined, so that the bit-sliced loop's registers are allocated without it.
template <int K, bool BATCH, bool PROD, bool ADAPT>
__device__ __noinline__ unsigned int tail_run(const FrankLaunch& p, TailGroups<PROD> g, int ns, unsigned int* s_hist,
                                              uint32_t* wbuf) {
  constexpr uint32_t FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const int precision = p.precision;
  unsigned int errors = 0u;

  // the rare events, one group at a time (i run-time; its values picked from the arrays)
  auto ens_of = [&](int i) -> const Ensemble& {
    if constexpr (BATCH) return p.ens_table[pick(g.ens, i)];
    else return p.ens;
  };
  auto row_of = [&](int i) -> long long {
    const Ensemble& e = ens_of(i);
    return e.run_offset + ((long long)pick(g.sg, i) - e.group_base) * 32 + lane;
  };
  // the state of run `lane` of group i into snapshot `snap`
  auto capture = [&](int i, int snap) {
    if ((g.valid >> i) & 1u) {
      const int l = pick(g.l, i), d = pick(g.d, i), a = ens_of(i).n_tot - l - d;
      if (s_hist) atomicAdd(&s_hist[snap * kHistBins + ee_bin(l, d)], 1u);
      else atomicAdd(&p.hist[((long long)pick(g.ens, i) * p.n_snap + snap) * kHistBins + ee_bin(l, d)], 1ull);
      if (p.snap_counts) {
        int* o = p.snap_counts + ((long long)snap * p.n_runs_total + row_of(i)) * p.n_species;
        o[p.perm[0]] = l;
        o[p.perm[1]] = d;
        o[p.perm[2]] = a;
      }
    }
  };
  // the outputs of a finished group (every thread: its own run)
  auto finish = [&](int i) {
    const bool valid = (g.valid >> i) & 1u, live = (g.live >> i) & 1u;
    const unsigned long long step = pick(g.step, i);
    const int ens = pick(g.ens, i);
    int cls = 3;
    if (valid) {
      const int l = pick(g.l, i), d = pick(g.d, i), a = ens_of(i).n_tot - l - d;
      const long long row = row_of(i);
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
        g.lsteps += step;  // runs that never absorbed
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

  while (ns > 0) {
    TailEvent ev;
    switch (ns) {
      case 1: ev = tail_lockstep<K, BATCH, PROD, ADAPT, 1>(p, g, wbuf); break;
      case 2: ev = tail_lockstep<K, BATCH, PROD, ADAPT, 2>(p, g, wbuf); break;
      case 3: ev = tail_lockstep<K, BATCH, PROD, ADAPT, 3>(p, g, wbuf); break;
      default: ev = tail_lockstep<K, BATCH, PROD, ADAPT, kTailSlots>(p, g, wbuf); break;
    }
    uint32_t fin = 0u;  // groups that end here
    if (ev.kind == kTailBudget) {
      errors |= kErrTimeout;
      fin = ev.slots;
    } else if (ev.kind == kTailRedraw) {
      errors |= kErrRedraw;
      fin = ev.slots;
      g.redraws += pick(ev.rd, __ffs((int)fin) - 1);
    } else if (ev.kind == kTailCross) {
      // the state before the event into the snapshot whose time it passes, or t_end passed
#pragma unroll 1
      for (int i = 0; i < ns; ++i) {
        if (!((ev.slots >> i) & 1u)) continue;
        const int snap = pick(g.snap, i);
        if (snap >= p.n_snap) {  // t_end: the step is not applied, its redraws are counted
          fin |= 1u << i;
          g.redraws += pick(ev.rd, i);
        } else {
          capture(i, snap);
          put(g.snap, i, snap + 1);
        }
      }
    } else {
      // runs absorbed at the step just committed: their time is the group's clock; a group whose
      // every run has absorbed fills its remaining snapshots with its final state and ends
#pragma unroll 1
      for (int i = 0; i < ns; ++i) {
        if (!((ev.slots >> i) & 1u)) continue;
        if ((ev.mine >> i) & 1u) {
          p.t_abs[row_of(i)] = pick(g.clk, i).time(ens_of(i), precision);
          g.lsteps += pick(g.step, i);
        }
        if (!__any_sync(FULL, (g.live >> i) & 1u)) {
          for (int snap = pick(g.snap, i); snap < p.n_snap; ++snap) capture(i, snap);
          fin |= 1u << i;
        }
      }
    }
    if (fin) {
#pragma unroll 1
      for (int i = 0; i < ns; ++i)
        if ((fin >> i) & 1u) finish(i);
      tail_compact(g, fin, ns);
      ns -= __popc(fin);
    }
  }

  // the counters of the runs stepped here
  const unsigned long long react = warp_sum64(g.react);
  const unsigned long long lsteps = warp_sum64(g.lsteps);
  if (lane == 0) {
    atomicAdd(&p.counters[kReactions], react);
    atomicAdd(&p.counters[kLaneSteps], lsteps);
    atomicAdd(&p.counters[kNullLaneSteps], lsteps - react);
    if (g.redraws) atomicAdd(&p.counters[kRedrawRounds], g.redraws);
  }
  return errors;
}

}  // namespace bitssa
