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
// One group step (Sec. 3, steps 1-7 with steps 5-6 replaced by a-d):
//   1. Philox words of attempt 0: planes of the uniform integer n and the
//      group's waiting-time bits; lanes with n >= lambda_int redraw from the
//      next attempt.
//   2. Clock: tau ~ Exp(Lambda) (Eq. equation-tau).  Snapshots whose time is
//      passed record the state before the event; passing t_end stops the group.
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

// Largest N with N (N - 1) / 2 < 2^K, i.e. the largest Frank system whose
// lambda_int fits in K planes.
__host__ __device__ constexpr long long frank_nmax(int K) {
  long long lo = 1, hi = 1ll << 17;
  while (lo < hi) {
    const long long mid = (lo + hi + 1) / 2;
    if (mid * (mid - 1) / 2 < (1ll << K)) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__host__ __device__ constexpr int bit_length(long long v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

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

// Per-thread counters, flushed once per kernel.
struct FrankCounters {
  unsigned long long group_steps, lane_steps, reactions, null_steps, redraws, absorbed, groups;
};

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

template <int K>
__device__ __forceinline__ void run_group(const FrankLaunch& p, const Ensemble& e, const Threshold* thr,
                                          long long group_local, int ens_index, unsigned int* s_hist,
                                          FrankCounters& cnt, unsigned int& errors) {
  using Sh = FrankShape<K>;
  constexpr int B = Sh::B, WP = Sh::WP, WU3 = Sh::WU3, WR1 = Sh::WR1, WR3 = Sh::WR3;
  constexpr int NC0 = Sh::NC0, NCR = Sh::NCR;

  const long long run0 = group_local * 32;
  const long long left = e.n_runs - run0;
  const int nvalid = left >= 32 ? 32 : (int)left;
  const uint32_t valid = nvalid >= 32 ? 0xFFFFFFFFu : ((1u << nvalid) - 1u);
  const uint32_t sgroup = (uint32_t)(e.group_base + group_local);
  const PhiloxKey key{(uint32_t)e.seed, (uint32_t)(e.seed >> 32)};
  const long long row0 = e.run_offset + run0;
  const int n_tot = e.n_tot;

  // ---- initial planes (padding lanes hold (0, 0, N): absorbed, never counted)
  uint32_t Lp[B], Dp[B], Ap[B];
  if (p.init_counts) {
    bs::broadcast(Lp, 0);
    bs::broadcast(Dp, 0);
    bs::broadcast(Ap, n_tot);
    for (int l = 0; l < nvalid; ++l) {
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

  // ---- cumulative propensities by bit-sliced products (Eq. equation-as)
  uint32_t S1[K], S2[K], S3[K];
  {
    uint32_t h[K];
    bs::multiply(S1, Ap, Lp);
    bs::multiply(h, Ap, Dp);
#pragma unroll
    for (int i = 0; i < K; ++i) S2[i] = S1[i];
    bs::add_signed(S2, h, 0u);
    bs::multiply(h, Lp, Dp);
#pragma unroll
    for (int i = 0; i < K; ++i) S3[i] = S2[i];
    bs::add_signed(S3, h, 0u);
  }

  // ---- the linear forms, by ripple adds of (shifted, complemented) count planes
  uint32_t Lm[B], P[WP], U[WP], R1[WR1], R3[WR3];
#pragma unroll
  for (int i = 0; i < B; ++i) Lm[i] = Lp[i];
  {
    uint32_t c = 0u;  // P = A + ~L = A - L - 1
#pragma unroll
    for (int i = 0; i < WP; ++i) {
      const uint32_t a = bs::plane<false>(Ap, i), b = ~bs::plane<false>(Lp, i);
      P[i] = bs::xor3(a, b, c);
      c = bs::maj(a, b, c);
    }
    c = 0xFFFFFFFFu;  // U = P + ~D + 1 = A - L - D - 1
#pragma unroll
    for (int i = 0; i < WP; ++i) {
      const uint32_t a = P[i], b = ~bs::plane<false>(Dp, i);
      U[i] = bs::xor3(a, b, c);
      c = bs::maj(a, b, c);
    }
    // R1 = (L << 1) + ~A - 1 = 2L - A - 2
    c = 0u;
#pragma unroll
    for (int i = 0; i < WR1; ++i) {
      const uint32_t a = i == 0 ? 0u : bs::plane<false>(Lp, i - 1), b = ~bs::plane<false>(Ap, i);
      R1[i] = bs::xor3(a, b, c);
      c = bs::maj(a, b, c);
    }
    bs::add_select3<-1, -1, -1>(R1, 0xFFFFFFFFu, 0u, 0u);
    // R3 = L + D + (~A << 1) - 1 = L + D - 2A - 3
    c = 0u;
#pragma unroll
    for (int i = 0; i < WR3; ++i) {
      const uint32_t a = bs::plane<false>(Lp, i), b = bs::plane<false>(Dp, i);
      R3[i] = bs::xor3(a, b, c);
      c = bs::maj(a, b, c);
    }
    c = 0u;
#pragma unroll
    for (int i = 0; i < WR3; ++i) {
      const uint32_t a = R3[i], b = i == 0 ? 0u : ~bs::plane<false>(Ap, i - 1);
      R3[i] = bs::xor3(a, b, c);
      c = bs::maj(a, b, c);
    }
    bs::add_select3<-1, -1, -1>(R3, 0xFFFFFFFFu, 0u, 0u);
  }

  // ---- which lanes can still react: some reaction with k_r > 0 has h_r > 0
  const bool all_active = e.active == 7u;
  auto live_lanes = [&]() -> uint32_t {
    if (all_active) return bs::nonzero(S3);
    uint32_t m = 0u;
    if (e.active & 1u) m |= bs::nonzero(S1);
    if (e.active & 2u) m |= bs::differ(S2, S1);
    if (e.active & 4u) m |= bs::differ(S3, S2);
    return m;
  };
  uint32_t live = live_lanes() & valid;
  // runs that start absorbed are absorbed at t = 0
  {
    uint32_t at0 = valid & ~live;
    while (at0) {
      const int l = __ffs(at0) - 1;
      at0 &= at0 - 1;
      p.t_abs[row0 + l] = 0.0;
    }
  }

  // ---- snapshot capture: the current state of every valid lane
  const int n_snap = p.n_snap;
  auto capture = [&](int snap) {
    for (int l = 0; l < nvalid; ++l) {
      int cl, cd, ca;
      lane_counts<B, WP>(Lm, U, n_tot, l, cl, cd, ca);
      if (s_hist) atomicAdd(&s_hist[snap * kHistBins + ee_bin(cl, cd)], 1u);
      else atomicAdd(&p.hist[((long long)ens_index * n_snap + snap) * kHistBins + ee_bin(cl, cd)], 1ull);
      if (p.snap_counts) {
        int* o = p.snap_counts + ((long long)snap * p.n_runs_total + row0 + l) * p.n_species;
        o[p.perm[0]] = cl;
        o[p.perm[1]] = cd;
        o[p.perm[2]] = ca;
      }
    }
  };

  // ---- clock state
  const int precision = p.precision;
  double m = 1.0;        // product clock: exp(-Lambda t) = m 2^E
  long long E = 0;
  double t = 0.0;        // fp64 sum clocks
  float t_f = 0.0f, c_f = 0.0f;  // Kahan clock
  int snap = 0;
  Threshold cur = thr[0];
  auto group_time = [&]() -> double {
    if (precision == kP64) return -(log(m) + (double)E * kLn2) / e.lambda;
    if (precision == kP32Kahan) return (double)t_f;
    return t;
  };

  unsigned long long step = 0;
  unsigned long long reactions = 0, lane_steps = 0, redraws = 0;
  bool done = live == 0u;
  if (done)
    for (; snap < n_snap; ++snap) capture(snap);

  while (!done) {
    if (p.step_budget > 0 && (long long)step >= p.step_budget) {
      errors |= kErrTimeout;
      break;
    }
    // (1) the random words of attempt 0
    uint32_t w[4 * NC0];
#pragma unroll
    for (int c = 0; c < NC0; ++c) {
      const uint4 r = philox4x32_10(stream_counter(sgroup, step, 0u, 0u, (uint32_t)c), key);
      w[4 * c + 0] = r.x;
      w[4 * c + 1] = r.y;
      w[4 * c + 2] = r.z;
      w[4 * c + 3] = r.w;
    }
    uint32_t n[K];
#pragma unroll
    for (int i = 0; i < K; ++i) n[i] = w[i];
    uint32_t need = ~bs::less_than_const(n, e.lambda_int) & live;
    uint32_t attempt = 0u;
    while (need) {
      if (++attempt >= 64u) {
        errors |= kErrRedraw;
        break;
      }
      ++redraws;
      uint32_t wr[4 * NCR];
#pragma unroll
      for (int c = 0; c < NCR; ++c) {
        const uint4 r = philox4x32_10(stream_counter(sgroup, step, attempt, 0u, (uint32_t)c), key);
        wr[4 * c + 0] = r.x;
        wr[4 * c + 1] = r.y;
        wr[4 * c + 2] = r.z;
        wr[4 * c + 3] = r.w;
      }
#pragma unroll
      for (int i = 0; i < K; ++i) n[i] = (n[i] & ~need) | (wr[i] & need);
      need &= ~bs::less_than_const(n, e.lambda_int);
    }
    if (need) break;

    // (2) the clock: the candidate time of this step's event
    double m_new = m, t_new = t;
    long long E_new = E;
    float tf_new = t_f, cf_new = c_f;
    bool crossed;
    if (precision == kP64) {
      const unsigned long long x = ((unsigned long long)w[K + 1] << 21) | (w[K] >> 11);
      const double u = (double)(x + 1ull) * 0x1p-53;
      const double mm = m * u;
      const int hi = __double2hiint(mm), lo = __double2loint(mm);
      E_new = E + (long long)(((hi >> 20) & 0x7FF) - 1023);
      m_new = __hiloint2double((hi & 0x800FFFFF) | 0x3FF00000, lo);
      crossed = E_new < cur.E || (E_new == cur.E && m_new < cur.m);
    } else if (precision == kP64LogSum) {
      const unsigned long long x = ((unsigned long long)w[K + 1] << 21) | (w[K] >> 11);
      const double u = (double)(x + 1ull) * 0x1p-53;
      t_new = t + (-log(u) / e.lambda);
      crossed = t_new > cur.t;
    } else {
      const float u = (float)((w[K + 1] >> 8) + 1u) * 0x1p-24f;
      const float tau = -logf(u) * e.inv_lambda_f;
      if (precision == kP32Kahan) {
        const float y = tau - c_f;
        const float s = t_f + y;
        cf_new = (s - t_f) - y;
        tf_new = s;
        crossed = s > cur.t_f;
      } else {
        t_new = t + (double)tau;
        crossed = t_new > cur.t;
      }
    }
    if (crossed) {
      bool stop = false;
      for (;;) {
        if (snap >= n_snap) {
          stop = true;  // t_end passed: the event is not applied
          break;
        }
        capture(snap);
        ++snap;
        cur = thr[snap];
        if (precision == kP64) crossed = E_new < cur.E || (E_new == cur.E && m_new < cur.m);
        else if (precision == kP32Kahan) crossed = tf_new > cur.t_f;
        else crossed = t_new > cur.t;
        if (!crossed) break;
      }
      if (stop) break;
    }
    m = m_new;
    E = E_new;
    t = t_new;
    t_f = tf_new;
    c_f = cf_new;

    // (3) comparators and changer words
    const uint32_t lt1 = bs::less_than(n, S1);
    const uint32_t lt2 = bs::less_than(n, S2);
    const uint32_t lt3 = bs::less_than(n, S3);
    uint32_t x1 = lt1 & live, x2 = lt2 & ~lt1 & live, x3 = lt3 & ~lt2 & live;

    // (4) thinning for k_r < k_max: keep iff U < T_r, U read most significant bit first
    if (e.thin) {
      const uint32_t alw1 = (e.thin_always & 1u) ? ~0u : 0u;
      const uint32_t alw2 = (e.thin_always & 2u) ? ~0u : 0u;
      const uint32_t alw3 = (e.thin_always & 4u) ? ~0u : 0u;
      uint32_t und = (x1 & ~alw1) | (x2 & ~alw2) | (x3 & ~alw3);
      uint32_t rej = 0u;
      const int q = e.thin_bits;
      int i = 0;
      auto thin_bit = [&](uint32_t word) {
        const int pos = q - 1 - i;
        const uint32_t b1 = 0u - (uint32_t)(((unsigned long long)e.thin_T[0] >> pos) & 1ull);
        const uint32_t b2 = 0u - (uint32_t)(((unsigned long long)e.thin_T[1] >> pos) & 1ull);
        const uint32_t b3 = 0u - (uint32_t)(((unsigned long long)e.thin_T[2] >> pos) & 1ull);
        const uint32_t tb = (x1 & b1) | (x2 & b2) | (x3 & b3);
        const uint32_t lower = und & ~word & tb;   // U < T decided
        const uint32_t higher = und & word & ~tb;  // U > T decided
        rej |= higher;
        und &= ~(lower | higher);
        ++i;
      };
#pragma unroll
      for (int k = K + 2; k < 4 * NC0; ++k)
        if (i < q) thin_bit(w[k]);
      for (uint32_t c = NC0; und != 0u && i < q; ++c) {
        const uint4 r = philox4x32_10(stream_counter(sgroup, step, 0u, 0u, c), key);
        if (i < q) thin_bit(r.x);
        if (i < q) thin_bit(r.y);
        if (i < q) thin_bit(r.z);
        if (i < q) thin_bit(r.w);
      }
      rej |= und;  // U == T: not below
      x1 &= ~rej;
      x2 &= ~rej;
      x3 &= ~rej;
    }

    // (5) updates from the counts before the reaction (App. B)
    const uint32_t x12 = x1 | x2;
    {
      uint32_t T[WR1];
#pragma unroll
      for (int i = 0; i < WR1; ++i)
        T[i] = (x1 & bs::plane<true>(P, i)) | (x2 & ~bs::plane<false>(Lm, i)) | (x3 & R1[i]);
      bs::add_signed(S1, T, x2);  // -L = ~L + 1
    }
    {
      uint32_t U3[WU3];  // -U - 3 = ~U - 2
#pragma unroll
      for (int i = 0; i < WU3; ++i) U3[i] = ~bs::plane<true>(U, i);
      bs::add_select3<-2, -2, -2>(U3, 0xFFFFFFFFu, 0u, 0u);
      uint32_t T[WU3 + 1];
#pragma unroll
      for (int i = 0; i < WU3 + 1; ++i)
        T[i] = (x12 & bs::plane<true>(U, i)) | (x3 & (i == 0 ? 0u : U3[i - 1]));
      bs::add_signed(S2, T, 0u);
    }
    {
      uint32_t Q[WP];  // A - D - 1 = U + L
      uint32_t c = 0u;
#pragma unroll
      for (int i = 0; i < WP; ++i) {
        const uint32_t a = U[i], b = bs::plane<false>(Lm, i);
        Q[i] = bs::xor3(a, b, c);
        c = bs::maj(a, b, c);
      }
      uint32_t T[WR3];
#pragma unroll
      for (int i = 0; i < WR3; ++i)
        T[i] = (x1 & bs::plane<true>(P, i)) | (x2 & bs::plane<true>(Q, i)) | (x3 & R3[i]);
      bs::add_signed(S3, T, 0u);
    }
    bs::add_select3<1, 0, -1>(Lm, x1, x2, x3);
    bs::add_select3<-2, -1, 3>(P, x1, x2, x3);
    bs::add_select3<-2, -2, 4>(U, x1, x2, x3);
    bs::add_select3<3, 1, -4>(R1, x1, x2, x3);
    bs::add_select3<3, 3, -6>(R3, x1, x2, x3);
    const uint32_t fired = x12 | x3;
    reactions += (unsigned)__popc(fired);
    lane_steps += (unsigned)__popc(live);
    ++step;

    // (6) absorption
    const uint32_t now_live = live_lanes() & live;
    uint32_t newly = live & ~now_live;
    if (newly) {
      const double tn = group_time();
      while (newly) {
        const int l = __ffs(newly) - 1;
        newly &= newly - 1;
        p.t_abs[row0 + l] = tn;
      }
      live = now_live;
      if (!live) {
        done = true;
        for (; snap < n_snap; ++snap) capture(snap);
      }
    }
  }

  // ---- outputs of the group
  unsigned long long outc[4] = {0, 0, 0, 0};
  for (int l = 0; l < nvalid; ++l) {
    int cl, cd, ca;
    lane_counts<B, WP>(Lm, U, n_tot, l, cl, cd, ca);
    int* o = p.final_counts + (row0 + l) * p.n_species;
    o[p.perm[0]] = cl;
    o[p.perm[1]] = cd;
    o[p.perm[2]] = ca;
    signed char oc = -1;
    if (!((live >> l) & 1u)) {
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
      if (outc[k]) atomicAdd(&p.ens_absorbed[(long long)ens_index * 4 + k], outc[k]);
  }
  cnt.group_steps += step;
  cnt.lane_steps += lane_steps;
  cnt.reactions += reactions;
  cnt.null_steps += lane_steps - reactions;
  cnt.redraws += redraws;
  cnt.absorbed += (unsigned long long)__popc(valid & ~live);
  cnt.groups += 1;
}

// The persistent kernel: every thread takes work items (groups) from a queue
// until none is left; single-ensemble launches read the ensemble from the
// kernel parameters (warp-uniform), batches from a table.
template <int K, bool BATCH>
__global__ void __launch_bounds__(256) frank_kernel(const __grid_constant__ FrankLaunch p) {
  extern __shared__ unsigned int s_hist[];
  const bool smem_hist = !BATCH && p.n_snap > 0;
  if (smem_hist) {
    for (int i = threadIdx.x; i < p.n_snap * kHistBins; i += blockDim.x) s_hist[i] = 0u;
    __syncthreads();
  }
  FrankCounters cnt = {0, 0, 0, 0, 0, 0, 0};
  unsigned int errors = 0u;
  for (;;) {
    const long long item = (long long)atomicAdd(p.queue, 1ull) + p.item_begin;
    if (item >= p.item_end) break;
    if (!BATCH) {
      run_group<K>(p, p.ens, p.thr, item, 0, smem_hist ? s_hist : nullptr, cnt, errors);
    } else {
      const int ei = p.item_ens[item];
      const Ensemble e = p.ens_table[ei];
      run_group<K>(p, e, p.thr + (long long)ei * (p.n_snap + 1), p.item_group[item], ei, nullptr, cnt,
                   errors);
    }
  }
  // flush: warp sums, one atomic per warp per counter
  unsigned long long v[7] = {cnt.group_steps, cnt.lane_steps, cnt.reactions, cnt.null_steps,
                             cnt.redraws, cnt.absorbed, cnt.groups};
  const int ctr_index[7] = {kGroupSteps, kLaneSteps, kReactions, kNullLaneSteps, kRedrawRounds, kAbsorbed,
                            kGroupsDone};
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    unsigned long long x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&p.counters[ctr_index[k]], x);
  }
  unsigned int err = __reduce_or_sync(0xFFFFFFFFu, errors);
  if ((threadIdx.x & 31) == 0 && err) atomicOr(p.status, err);
  if (smem_hist) {
    __syncthreads();
    for (int i = threadIdx.x; i < p.n_snap * kHistBins; i += blockDim.x)
      if (s_hist[i]) atomicAdd(&p.hist[i], (unsigned long long)s_hist[i]);
  }
}

}  // namespace bitssa
