// general_reg.cuh -- the general-network step loop with every count plane and every kept
// propensity in registers, for networks of at most kRegSpecies species and kRegReactions
// reactions whose counts fit the planes the products read (every network with a reaction of
// order 2 does: lambda_int >= N (N - 1) / 2).
//
// The steps, streams and runs are those of general_kernel in incremental mode (the change of each
// h_r after an event is linear in the counts before it, App. A generalised).  A reaction's
// reactants are still found at run time, but every thread of a launch runs the same network, so
// "species a of reaction r" is a branch that is uniform over the launch, into code that names the
// registers of each candidate species: no plane is loaded from shared memory and no word is
// selected lane by lane.  The reaction loop is unrolled over kRegReactions slots, the species
// loops over kRegSpecies; slots beyond the network's R and S are skipped by uniform branches, and
// the planes of absent species are zero.
#pragma once

#include <cstdint>

#include "general_kernel.cuh"

namespace bitssa {

template <int K>
struct RegPlanes {
  static constexpr int BM = GeneralShape<K>::BM;
  uint32_t x[kRegSpecies][BM];   // count planes of each species (lane l: run 32 g + l)
  uint32_t h[kRegReactions][K];  // the kept propensities h_r
};

// v[s] for a launch-uniform s < N.
template <int N>
__device__ __forceinline__ uint32_t pick(const uint32_t (&v)[N], int s) {
  uint32_t r = 0u;
#pragma unroll
  for (int q = 0; q < N; ++q)
    if (q == s) r = v[q];
  return r;
}

// Count of species s in lane l.
template <int K>
__device__ __forceinline__ int reg_lane_count(const RegPlanes<K>& X, int s, int l) {
  int v = 0;
#pragma unroll
  for (int q = 0; q < kRegSpecies; ++q)
    if (q == s) {
#pragma unroll
      for (int i = 0; i < RegPlanes<K>::BM; ++i) v |= (int)((X.x[q][i] >> l) & 1u) << i;
    }
  return v;
}

// Lanes where some reaction with k_r > 0 has h_r > 0 (the rule of general_live).
template <int K>
__device__ __forceinline__ uint32_t reg_live(const Network& net, const Ensemble& e, const RegPlanes<K>& X) {
  constexpr int BM = RegPlanes<K>::BM;
  uint32_t nz[kRegSpecies], two[kRegSpecies];
#pragma unroll
  for (int q = 0; q < kRegSpecies; ++q) {
    nz[q] = two[q] = 0u;
    if (q < net.S) {
      uint32_t t = 0u;
#pragma unroll
      for (int i = 1; i < BM; ++i) t |= X.x[q][i];
      two[q] = t;
      nz[q] = X.x[q][0] | t;
    }
  }
  uint32_t m = 0u;
#pragma unroll
  for (int r = 0; r < kRegReactions; ++r) {
    if (r >= net.R || !((e.active >> r) & 1u)) continue;
    const int a = net.a[r], b = net.b[r];
    m |= net.order[r] == 1 ? pick(nz, a) : (b == a ? pick(two, a) : (pick(nz, a) & pick(nz, b)));
  }
  return m;
}

// h (K planes) = the propensity of reaction r from the count planes (set-up only: the reactants'
// planes are copied out by unrolled selects, then the products of general_propensity).
template <int K>
__device__ __forceinline__ void reg_propensity(uint32_t (&h)[K], const Network& net, int r, const RegPlanes<K>& X) {
  constexpr int BM = RegPlanes<K>::BM;
  const int a = net.a[r], b = net.b[r];
  uint32_t xa[BM], xb[BM];
#pragma unroll
  for (int i = 0; i < BM; ++i) xa[i] = xb[i] = 0u;
#pragma unroll
  for (int q = 0; q < kRegSpecies; ++q) {
#pragma unroll
    for (int i = 0; i < BM; ++i) {
      if (q == a) xa[i] = X.x[q][i];
      if (q == b) xb[i] = X.x[q][i];
    }
  }
  if (net.order[r] == 1) {  // h = x_a, zero-extended
#pragma unroll
    for (int i = 0; i < K; ++i) h[i] = i < BM ? xa[i] : 0u;
  } else if (b != a) {  // h = x_a x_b
    bs::multiply(h, xa, xb);
  } else {  // h = x_a (x_a - 1) / 2
    half_square(h, xa);
  }
}

template <int K, bool PROD>
__device__ __forceinline__ void reg_capture(const FrankLaunch& p, const GeneralState<PROD>& s, const Ensemble& e,
                                            int snap, const RegPlanes<K>& X, unsigned int* s_hist) {
  capture_counts(p, s, e, snap, s_hist, [&](int sp, int l) { return reg_lane_count(X, sp, l); });
}

// Set up a group (as general_init): counts into registers (padding lanes and absent species hold
// zero), every h_r by products, the live lanes, the clock.
template <int K, bool PROD>
__device__ __forceinline__ void reg_init(const FrankLaunch& p, GeneralState<PROD>& s, const Ensemble& e,
                                         const Threshold* thr, long long group_local, int ens_index,
                                         RegPlanes<K>& X, unsigned int* s_hist) {
  constexpr int BM = RegPlanes<K>::BM;
  const Network& net = p.net;
  const long long run0 = group_local * 32;
  const long long left = e.n_runs - run0;
  s.nvalid = left >= 32 ? 32 : (int)left;
  s.valid = s.nvalid >= 32 ? 0xFFFFFFFFu : ((1u << s.nvalid) - 1u);
  s.sgroup = (uint32_t)(e.group_base + group_local);
  s.ens = ens_index;
  const long long row0 = e.run_offset + run0;
#pragma unroll
  for (int q = 0; q < kRegSpecies; ++q) {
#pragma unroll
    for (int i = 0; i < BM; ++i) {
      uint32_t w = 0u;
      if (q < net.S) {
        if (p.init_counts) {
          for (int l = 0; l < s.nvalid; ++l) w |= (uint32_t)((p.init_counts[(row0 + l) * net.S + q] >> i) & 1) << l;
        } else if ((e.init[q] >> i) & 1) {
          w = s.valid;
        }
      }
      X.x[q][i] = w;
    }
  }
#pragma unroll
  for (int r = 0; r < kRegReactions; ++r) {
    if (r < net.R) {
      reg_propensity<K>(X.h[r], net, r, X);
    } else {
#pragma unroll
      for (int i = 0; i < K; ++i) X.h[r][i] = 0u;
    }
  }
  s.live = reg_live<K>(net, e, X) & s.valid;
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
    for (; s.snap < p.n_snap; ++s.snap) reg_capture<K, PROD>(p, s, e, s.snap, X, s_hist);
}

// One group step: the steps of general_step on registers.
template <int K, bool PROD>
__device__ __forceinline__ void reg_step(const FrankLaunch& p, GeneralState<PROD>& s, const Ensemble& e,
                                         const Threshold* thr, RegPlanes<K>& X, unsigned int* s_hist,
                                         unsigned int& errors) {
  using Sh = GeneralShape<K>;
  constexpr int BM = Sh::BM;
  const Network& net = p.net;
  uint32_t n[K], w[4 * Sh::NC0];
  if (!general_draw<K, PROD>(p, s, e, thr, n, w, errors,
                             [&](int snap) { reg_capture<K, PROD>(p, s, e, snap, X, s_hist); }))
    return;

  // (3) the CDF walk: xi_r = [S_{r-1} <= n < S_r], S_r = sum_{p<=r} h_p, as the borrow of
  // n - S_{r-1} - h_r (sub_borrow)
  uint32_t xi[kRegReactions];
#pragma unroll
  for (int r = 0; r < kRegReactions; ++r) xi[r] = r < net.R ? sub_borrow(n, X.h[r]) : 0u;

  // (4) thinning for k_r < k_max
  general_thin<K>(xi, w, e, s);

  // (5) the change of every species in every lane: d_s = sum_r xi_r nu_rs (three planes)
  uint32_t fired = 0u;
#pragma unroll
  for (int r = 0; r < kRegReactions; ++r) fired |= xi[r];
  ++s.step;
  if (!fired) return;
  uint32_t d[kRegSpecies][3];
#pragma unroll
  for (int q = 0; q < kRegSpecies; ++q) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      uint32_t v = 0u;
      if (q < net.S && ((net.changes >> q) & 1u)) {
        const unsigned int sel = net.nu_bits[q][b];
#pragma unroll
        for (int r = 0; r < kRegReactions; ++r)
          if ((sel >> r) & 1u) v |= xi[r];
      }
      d[q][b] = v;
    }
  }
  // h_r += its change, from the counts before the event: d_b x_a + d_a x_b + d_a d_b for a pair,
  // d_a x_a + d_a (d_a - 1) / 2 for a homodimer, d_a for a first-order reaction
#pragma unroll
  for (int r = 0; r < kRegReactions; ++r) {
    if (r >= net.R) continue;
    const int a = net.a[r], b = net.b[r];
    if (!(((net.changes >> a) & 1u) || (b >= 0 && ((net.changes >> b) & 1u)))) continue;
    uint32_t da[3], db[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      da[k] = db[k] = 0u;
#pragma unroll
      for (int q = 0; q < kRegSpecies; ++q) {
        if (q == a) da[k] = d[q][k];
        if (q == b) db[k] = d[q][k];
      }
    }
    uint32_t cst[4];
    if (net.order[r] == 1) {
      cst[0] = da[0];
      cst[1] = da[1];
      cst[2] = da[2];
      cst[3] = da[2];
    } else {
      // x_q scaled by the other reactant's change (its own for a homodimer)
#pragma unroll
      for (int q = 0; q < kRegSpecies; ++q) {
        if (q != a && q != b) continue;
        const bool other = q == a && b != a;
        const uint32_t f[3] = {other ? db[0] : da[0], other ? db[1] : da[1], other ? db[2] : da[2]};
        add_scaled(X.h[r], X.x[q], f);
      }
      if (b == a) same_constant(da, cst);
      else pair_constant(da, db, cst);
    }
    add_small(X.h[r], cst);
  }
  // the counts: x_s += d_s
#pragma unroll
  for (int q = 0; q < kRegSpecies; ++q) {
    if (q >= net.S || !((net.changes >> q) & 1u)) continue;
    uint32_t carry = 0u;
#pragma unroll
    for (int i = 0; i < BM; ++i) {
      const uint32_t di = d[q][i < 2 ? i : 2];
      const uint32_t xv = X.x[q][i];
      X.x[q][i] = bs::xor3(xv, di, carry);
      carry = bs::maj(xv, di, carry);
    }
  }
  s.reactions += (unsigned)__popc(fired);

  // (6) absorption
  const uint32_t now_live = reg_live<K>(net, e, X) & s.live;
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
      for (; s.snap < p.n_snap; ++s.snap) reg_capture<K, PROD>(p, s, e, s.snap, X, s_hist);
    }
  }
}

// The register-resident general kernel.  Dynamic shared memory: the histogram (single ensemble)
// only.
template <int K, bool BATCH, bool PROD>
__global__ void __launch_bounds__(256) general_reg_kernel(const __grid_constant__ FrankLaunch p) {
  extern __shared__ unsigned int s_mem[];
  RegPlanes<K> X;
  general_queue<BATCH, PROD>(
      p, s_mem,
      [&](GeneralState<PROD>& s, const Ensemble& e, const Threshold* thr, long long group, int ens,
          unsigned int* s_hist) { reg_init<K, PROD>(p, s, e, thr, group, ens, X, s_hist); },
      [&](GeneralState<PROD>& s, const Ensemble& e, const Threshold* thr, unsigned int* s_hist,
          unsigned int& errors) { reg_step<K, PROD>(p, s, e, thr, X, s_hist, errors); },
      [&](GeneralState<PROD>& s, const Ensemble& e) {
        finish_counts(p, s, e, [&](int sp, int l) { return reg_lane_count(X, sp, l); });
      });
}

}  // namespace bitssa
