// lattice_kernel.cuh -- Frank's model on a periodic lattice, 32 runs per word (sm_103a).
//
// One block runs one group of 32 runs at a time.  The group's lattice lives in global memory
// (L2-resident at the sizes this serves): per site one record of 3 P words, the count planes of L,
// D and A, plane i holding bit i of the 32 runs' counts (the binary-word representation of
// Sec. 4, one word per count plane, now per site).
//
// The steps of a group form one sequence: step s draws its words from the group's Philox stream
// at counter (group, s, tag 2), among them the site sigma_s shared by the group's runs and, per
// run, the K-bit number n that picks its event at sigma_s (a hop of one molecule to one of the
// four neighbours, one of Frank's three reactions, or nothing).  The site sequence does not
// depend on the state, so a window of consecutive steps (one per step thread) is drawn at once.
// A step changes only its site and the neighbours its runs hop to, so two steps whose closed
// neighbourhoods (the site and its four neighbours) are disjoint commute: the window's steps run
// in waves, a step waiting for every earlier step of the window whose neighbourhood meets its own
// (per-site stamps in shared memory find them).  Each step is the bit-sliced event of Sec. 4 at
// its site: comparisons of n with the hop slots and with the cumulative slots rho_r S_r (S_r
// from bit-sliced schoolbook products of the site's count planes, Sec. 4.1), masked count updates
// at the site (Eq. equation-v) and masked increments at the neighbours.  The group clock is summed
// in step order by a service warp, which also replays each window's event masks in step order to
// keep every run's lattice totals and the time its lattice first holds one species.  Every run
// therefore takes exactly the trajectory of the serial definition; only independent steps are
// reordered.  (The window's phases are listed above lattice_kernel.)
#pragma once

#include <cstdint>

#include "bitslice.cuh"
#include "internal.h"
#include "lattice.h"
#include "philox.cuh"

namespace bitssa {
namespace lat {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kNoStamp = 0xFFFFFFFFu;
constexpr int kCross = 1;  // window cut by a snapshot or t_end

// The four neighbours of site s: x + 1, x - 1, y + 1, y - 1 (periodic), the directions of a hop.
__device__ __forceinline__ void neighbours(const LatticeLaunch& p, int s, int (&nb)[4]) {
  const int x = s & (p.lx - 1), y = s >> p.lx_log;
  const int row = y << p.lx_log;
  nb[0] = ((x + 1) & (p.lx - 1)) + row;
  nb[1] = ((x - 1) & (p.lx - 1)) + row;
  nb[2] = x + (((y + 1) & (p.ly - 1)) << p.lx_log);
  nb[3] = x + (((y - 1) & (p.ly - 1)) << p.lx_log);
}

template <int P>
__device__ __forceinline__ void load_site(const uint32_t* rec, uint32_t (&L)[P], uint32_t (&D)[P],
                                          uint32_t (&A)[P]) {
  const uint4* r4 = reinterpret_cast<const uint4*>(rec);
  uint32_t w[3 * P];
#pragma unroll
  for (int i = 0; i < 3 * P / 4; ++i) {
    const uint4 v = r4[i];
    w[4 * i] = v.x;
    w[4 * i + 1] = v.y;
    w[4 * i + 2] = v.z;
    w[4 * i + 3] = v.w;
  }
#pragma unroll
  for (int i = 0; i < P; ++i) {
    L[i] = w[i];
    D[i] = w[P + i];
    A[i] = w[2 * P + i];
  }
}

template <int P>
__device__ __forceinline__ void store_site(uint32_t* rec, const uint32_t (&L)[P], const uint32_t (&D)[P],
                                           const uint32_t (&A)[P]) {
  uint32_t w[3 * P];
#pragma unroll
  for (int i = 0; i < P; ++i) {
    w[i] = L[i];
    w[P + i] = D[i];
    w[2 * P + i] = A[i];
  }
  uint4* r4 = reinterpret_cast<uint4*>(rec);
#pragma unroll
  for (int i = 0; i < 3 * P / 4; ++i) r4[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
}

// x += 1 on the lanes of inc (from plane `at`), x -= 1 on the lanes of dec; inc and dec disjoint,
// so each lane runs either a carry or a borrow chain.
template <int P>
__device__ __forceinline__ void add_pm(uint32_t (&x)[P], uint32_t inc, uint32_t dec, int at) {
  uint32_t carry = 0u, borrow = dec;
#pragma unroll
  for (int i = 0; i < P; ++i) {
    const uint32_t c = carry | (i == at ? inc : 0u);
    const uint32_t a = x[i];
    x[i] = a ^ c ^ borrow;
    carry = a & c;
    borrow = ~a & borrow;
  }
}

// s = x + y (W planes; the caller knows the sum fits).
template <int W>
__device__ __forceinline__ void add(uint32_t (&s)[W], const uint32_t (&x)[W], const uint32_t (&y)[W]) {
  uint32_t carry = 0u;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    const uint32_t a = x[i], b = y[i];
    s[i] = a ^ b ^ carry;
    carry = bs::maj(a, b, carry);
  }
}

// The largest value over the lanes of a bit-sliced number.
template <int W>
__device__ __forceinline__ unsigned lane_max(const uint32_t (&x)[W]) {
  uint32_t cand = kFull;
  unsigned v = 0;
#pragma unroll
  for (int i = W - 1; i >= 0; --i) {
    const uint32_t hit = x[i] & cand;
    if (hit) {
      v |= 1u << i;
      cand = hit;
    }
  }
  return v;
}

// R = rho * S modulo 2^KW, rho < 2^kLatRhoBits: shifted copies of S for the set bits of rho.
template <int KW, int SW>
__device__ __forceinline__ void scale(uint32_t (&R)[KW], const uint32_t (&S)[SW], uint32_t rho) {
#pragma unroll
  for (int i = 0; i < KW; ++i) R[i] = 0u;
  bool first = true;
#pragma unroll
  for (int j = 0; j < kLatRhoBits; ++j) {
    if ((rho >> j) & 1u) {
      if (first) {
#pragma unroll
        for (int i = j; i < KW; ++i) R[i] = (i - j < SW) ? S[i - j] : 0u;
        first = false;
      } else {
        uint32_t carry = 0u;
#pragma unroll
        for (int i = j; i < KW; ++i) {
          const uint32_t a = R[i], b = (i - j < SW) ? S[i - j] : 0u;
          R[i] = a ^ b ^ carry;
          carry = bs::maj(a, b, carry);
        }
      }
    }
  }
}

__device__ __forceinline__ uint32_t word_of(const uint4& w, int e) {
  return e == 0 ? w.x : (e == 1 ? w.y : (e == 2 ? w.z : w.w));
}

struct StepArgs {
  uint32_t group;        // stream group index
  long long step;        // the step's index in the group's sequence
  int sigma;             // its site
  uint32_t w3;           // word 3 of the stream (plane 0 of n)
  int bh, K;             // planes of the molecule index, planes of n
  uint32_t m;            // the cap
  uint32_t hop_slots;    // 4 rho_h 2^bh
  uint32_t* planes;      // the group's site records
};

struct StepOut {
  uint32_t x1, x2, x3, hop;  // runs that took reaction 1, 2, 3, or hopped
  bool overflow;             // a neighbour of some run went above the cap
  unsigned ub_sigma;         // largest site total at sigma after the step
};

// Planes 1 .. 4 NC of n (those below K; the rest stay zero) from calls 1 .. NC of the step's stream.
template <int KW, int NC>
__device__ __forceinline__ void draw_planes(uint32_t (&n)[KW], const StepArgs& a, PhiloxKey key) {
  uint32_t w[4 * NC];
  philox4x32_10_block<NC>(w, stream_counter(a.group, (unsigned long long)a.step, 0u, 2u, 0u), 1u, key);
#pragma unroll
  for (int j = 0; j < 4 * NC; ++j) {
    const int i = 1 + j;
    if (i < KW) n[i] = i < a.K ? w[j] : 0u;
  }
}

// One step of the group at its site, all 32 runs at once; updates the site and the neighbours
// a run hops to, and the cap table ub.
template <int P, int KW>
__device__ __forceinline__ StepOut step(const LatticeLaunch& p, const StepArgs& a, uint16_t* ub) {
  constexpr int SW = 2 * P - 1;  // S_3 <= m^2 / 3 < 2^(2P - 2)
  const PhiloxKey key{(uint32_t)p.seed, (uint32_t)(p.seed >> 32)};
  // (1) the planes of n: word 3 + i is plane i, i < K; planes at and above K are zero.  The calls
  //     beyond the first (planes 1 .. K - 1: calls 1 .. (K + 2) / 4) run as one interleaved block.
  uint32_t n[KW];
#pragma unroll
  for (int i = 0; i < KW; ++i) n[i] = 0u;
  n[0] = a.K > 0 ? a.w3 : 0u;
  const int nc = (a.K + 2) / 4;
  if (nc <= 2) draw_planes<KW, 2>(n, a, key);
  else if (nc <= 4) draw_planes<KW, 4>(n, a, key);
  else if (nc <= 6) draw_planes<KW, 6>(n, a, key);
  else draw_planes<KW, 8>(n, a, key);
  uint32_t* rec = a.planes + (size_t)a.sigma * p.rec;
  uint32_t L[P], D[P], A[P];
  load_site<P>(rec, L, D, A);

  // (2) hops: n < 4 rho_h m; direction n & 3, molecule (n >> 2) & (m - 1) against L, L + D, L + D + A
  const uint32_t is_hop = bs::less_than_const<KW>(n, a.hop_slots);
  uint32_t mol[P], LD[P], T[P];
#pragma unroll
  for (int i = 0; i < P; ++i) mol[i] = i < a.bh ? n[2 + i] : 0u;
  add<P>(LD, L, D);
  add<P>(T, LD, A);
  const uint32_t ltL = bs::less_than<P>(mol, L), ltLD = bs::less_than<P>(mol, LD), ltT = bs::less_than<P>(mol, T);
  const uint32_t hL = is_hop & ltL, hD = is_hop & ltLD & ~ltL, hA = is_hop & ltT & ~ltLD;

  // (3) reactions: 4 rho_h m + rho_r S_{r-1} <= n < 4 rho_h m + rho_r S_r with S_1 = A L,
  //     S_2 = A (L + D), S_3 = S_2 + L D
  uint32_t S1[SW], S2[SW], S3[SW], h3[SW];
  bs::multiply<SW, P, P>(S1, A, L);
  bs::multiply<SW, P, P>(S2, A, LD);
  bs::multiply<SW, P, P>(h3, L, D);
  add<SW>(S3, S2, h3);
  uint32_t y[KW];
  {
    uint32_t borrow = 0u;
#pragma unroll
    for (int i = 0; i < KW; ++i) {
      const uint32_t h = ((a.hop_slots >> i) & 1u) ? kFull : 0u;
      y[i] = n[i] ^ h ^ borrow;
      borrow = bs::maj(~n[i], h, borrow);
    }
  }
  uint32_t lt1, lt2, lt3;
  {
    uint32_t R[KW];
    scale<KW, SW>(R, S1, p.rho_r);
    lt1 = bs::less_than<KW>(y, R);
    scale<KW, SW>(R, S2, p.rho_r);
    lt2 = bs::less_than<KW>(y, R);
    scale<KW, SW>(R, S3, p.rho_r);
    lt3 = bs::less_than<KW>(y, R);
  }
  const uint32_t react = ~is_hop;
  uint32_t x1 = react & lt1, x2 = react & lt2 & ~lt1, x3 = react & lt3 & ~lt2;

  // (4) thinning: U from words 35.. (most significant bit first) against T_r
  if (p.thin) {
    const uint32_t c1 = (p.always & 1u) ? 0u : x1, c2 = (p.always & 2u) ? 0u : x2,
                   c3 = (p.always & 4u) ? 0u : x3;
    if (c1 | c2 | c3) {
      uint32_t lt[3] = {0u, 0u, 0u}, eq[3] = {kFull, kFull, kFull};
      uint4 buf = make_uint4(0u, 0u, 0u, 0u);
      int have = -1;
      for (int i = 0; i < p.q; ++i) {
        const int k = 35 + i;
        if ((k >> 2) != have) {
          have = k >> 2;
          buf = philox4x32_10(stream_counter(a.group, (unsigned long long)a.step, 0u, 2u, (uint32_t)have), key);
        }
        const uint32_t u = word_of(buf, k & 3);
        const int bit = p.q - 1 - i;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const uint32_t t = ((p.thin_T[r] >> bit) & 1ull) ? kFull : 0u;
          lt[r] |= eq[r] & ~u & t;
          eq[r] &= ~(u ^ t);
        }
        if (((c1 & eq[0]) | (c2 & eq[1]) | (c3 & eq[2])) == 0u) break;
      }
      x1 &= (p.always & 1u) ? kFull : lt[0];
      x2 &= (p.always & 2u) ? kFull : lt[1];
      x3 &= (p.always & 4u) ? kFull : lt[2];
    }
  }

  // (5) the site: L += x1 - x3 - hL, D += x2 - x3 - hD, A += 2 x3 - x1 - x2 - hA
  StepOut o;
  o.x1 = x1;
  o.x2 = x2;
  o.x3 = x3;
  const uint32_t hop = hL | hD | hA;
  o.hop = hop;
  o.overflow = false;
  if (x1 | x2 | x3 | hop) {
    add_pm<P>(L, x1, x3 | hL, 0);
    add_pm<P>(D, x2, x3 | hD, 0);
    add_pm<P>(A, x3, x1 | x2 | hA, 1);
    store_site<P>(rec, L, D, A);
  }
  if (hop) {
    add_pm<P>(T, 0u, hop, 0);
    ub[a.sigma] = (uint16_t)lane_max<P>(T);
    // (6) the neighbours a run hops to, one direction at a time (two directions may share a
    //     site on a side of length 2, and a side of length 1 sends a molecule back to sigma)
    int nb[4];
    neighbours(p, a.sigma, nb);
    const uint32_t n0 = n[0], n1 = n[1];
    const uint32_t dir[4] = {~n0 & ~n1, n0 & ~n1, ~n0 & n1, n0 & n1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t aL = hL & dir[k], aD = hD & dir[k], aA = hA & dir[k];
      if (aL | aD | aA) {
        uint32_t* r2 = a.planes + (size_t)nb[k] * p.rec;
        uint32_t L2[P], D2[P], A2[P], LD2[P], T2[P];
        load_site<P>(r2, L2, D2, A2);
        add_pm<P>(L2, aL, 0u, 0);
        add_pm<P>(D2, aD, 0u, 0);
        add_pm<P>(A2, aA, 0u, 0);
        store_site<P>(r2, L2, D2, A2);
        add<P>(LD2, L2, D2);
        add<P>(T2, LD2, A2);
        if (~bs::less_than_const<P>(T2, a.m + 1u)) o.overflow = true;  // a site above the cap
        ub[nb[k]] = (uint16_t)lane_max<P>(T2);
      }
    }
  }
  return o;
}

}  // namespace lat

// Shared-memory layout of a block (lat_smem_bytes in lattice.h sizes it): per site, the stamp and
// hop-count tables (uint32) and the cap table ub (uint16, the largest site total over the group's
// runs); per step, in a ring indexed by the step's index modulo kLatRing, its waiting time, site
// and plane 0 of n, the clock after it, its event masks and its done flag; the ready list.
struct LatSmem {
  uint32_t* stamp;
  uint32_t* hopcnt;
  uint16_t* ub;
  double* tnew;   // time after the step's event
  double* taud;   // fp64 waiting time
  float* tauf;    // fp32 waiting time
  float* tf;      // fp32 clock after the step (Kahan sum or plain sum)
  float* cf;      // Kahan compensation after the step
  int* sigma;
  uint32_t* w3;
  uint32_t* x1;
  uint32_t* x2;
  uint32_t* x3;
  uint32_t* hop;
  int* done;
  int* ready;     // [kLatSlots T]
};

__device__ __forceinline__ LatSmem lat_smem(unsigned char* base, int M) {
  constexpr int R = kLatRing;
  LatSmem s;
  s.stamp = reinterpret_cast<uint32_t*>(base);
  s.hopcnt = s.stamp + M;
  s.ub = reinterpret_cast<uint16_t*>(s.hopcnt + M);
  unsigned char* w = reinterpret_cast<unsigned char*>(s.ub + ((M + 3) & ~3));
  s.tnew = reinterpret_cast<double*>(w);
  s.taud = s.tnew + R;
  s.tauf = reinterpret_cast<float*>(s.taud + R);
  s.tf = s.tauf + R;
  s.cf = s.tf + R;
  s.sigma = reinterpret_cast<int*>(s.cf + R);
  s.w3 = reinterpret_cast<uint32_t*>(s.sigma + R);
  s.x1 = s.w3 + R;
  s.x2 = s.x1 + R;
  s.x3 = s.x2 + R;
  s.hop = s.x3 + R;
  s.done = reinterpret_cast<int*>(s.hop + R);
  s.ready = s.done + R;
  return s;
}

namespace lat {

constexpr long long kNoStop = 0x7FFFFFFFFFFFFFFFll;
enum StopReason { kStopNone = 0, kStopFlag = 1, kStopCross = 2, kStopBudget = 3 };

__device__ __forceinline__ int slot(long long s) { return (int)(s & (kLatRing - 1)); }

// Barrier of the step warps only; the service warp runs on meanwhile.
__device__ __forceinline__ void step_sync(int T) { asm volatile("bar.sync 1, %0;" ::"r"(T) : "memory"); }

// Run `lane` of the group, kept by the service warp: lattice totals, events, first single-species time.
struct RunBook {
  long long tot[3];
  long long reactions, hops;
  double t_h;
  int outcome;
};

// Column `lane` of the 32 x 32 bit matrix whose row j is lane j's word v: bit j of the result is bit
// `lane` of row j.  Five butterfly stages swap the off-diagonal blocks of width 16, 8, 4, 2, 1.
__device__ __forceinline__ uint32_t transpose32(uint32_t v, int lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int s = 0, k = 16; s < 5; ++s, k >>= 1) {
    const uint32_t m = masks[s];
    const uint32_t o = __shfl_xor_sync(kFull, v, k);
    v = (lane & k) ? ((v & ~m) | ((o >> k) & m)) : ((v & m) | ((o << k) & ~m));
  }
  return v;
}

// Adds the events of steps [a, b) to run `lane`'s book (every lane of the warp calls it; `mine` =
// the lane is a run of the group).  Each run's events over 32 steps are one column of the masks,
// so a bit transpose and a population count give the run's counts.  A species whose lattice total
// reaches zero stays at zero, so a run that still holds two species after the range held two
// throughout it; only a run left with one species replays the range in step order, to find the
// event after which its lattice first held one species.
__device__ __forceinline__ void replay(RunBook& r, const LatSmem& S, long long a, long long b, int lane, bool mine,
                                      bool f32) {
  int n1 = 0, n2 = 0, n3 = 0, nh = 0;
  for (long long base = a; base < b; base += 32) {
    const long long i = base + lane;
    const bool in = i < b;
    const int k = slot(i);
    n1 += __popc(transpose32(in ? S.x1[k] : 0u, lane));
    n2 += __popc(transpose32(in ? S.x2[k] : 0u, lane));
    n3 += __popc(transpose32(in ? S.x3[k] : 0u, lane));
    nh += __popc(transpose32(in ? S.hop[k] : 0u, lane));
  }
  if (!mine) return;
  const long long start[3] = {r.tot[0], r.tot[1], r.tot[2]};
  r.tot[0] += n1 - n3;
  r.tot[1] += n2 - n3;
  r.tot[2] += 2 * n3 - n1 - n2;
  r.reactions += n1 + n2 + n3;
  r.hops += nh;
  if (r.outcome != -1 || (r.tot[0] > 0) + (r.tot[1] > 0) + (r.tot[2] > 0) > 1) return;
  // the range holds the run's last extinction before a single species: find it in step order
  const uint32_t bit = 1u << lane;
  long long t0 = start[0], t1 = start[1], t2 = start[2];
  for (long long i = a; i < b; ++i) {
    const int k = slot(i);
    const uint32_t r1 = S.x1[k] & bit, r2 = S.x2[k] & bit, r3 = S.x3[k] & bit;
    if (!(r1 | r2 | r3)) continue;
    if (r1) {
      ++t0;
      --t2;
    } else if (r2) {
      ++t1;
      --t2;
    } else {
      --t0;
      --t1;
      t2 += 2;
    }
    if ((t0 > 0) + (t1 > 0) + (t2 > 0) == 1) {
      r.t_h = f32 ? (double)S.tf[k] : S.tnew[k];
      r.outcome = t0 ? 0 : (t1 ? 1 : 2);
      break;
    }
  }
}

struct Clock {
  double t;   // fp64 modes: the time; fp32 modes: (double) of the fp32 sum
  float tf;   // fp32 sum (Kahan or plain)
  float cf;   // Kahan compensation
};

// The group clock over steps [from, from + n), in step order (Eq. equation-tau, Eq.
// eq-update-time), from state c, computed by the 32 lanes of a warp together: each block of 32
// steps loads its waiting times in parallel, every lane runs the same recurrence on them (passed
// by shuffles, so no load waits on the chain), and lane j keeps the state after step j of the
// block and stores it with the others.  Records the clock after each step (the fp32 sum and its
// compensation in the fp32 modes, else the fp64 time).  With `detect`, stops before the first step
// whose event would pass the next snapshot (if any) or t_end and returns its offset with its time
// in *t_cut; otherwise returns n.  The fp32 sums compare against the largest floats at or below the
// time points, which decides exactly as comparing (double) of the sum with the time point.
__device__ __forceinline__ int clock_run(const LatticeLaunch& p, const LatSmem& S, long long from, int n, bool detect,
                                         bool has_snap, int next_snap, Clock c, double* t_cut, int lane) {
  if (p.precision == kP32Kahan || p.precision == kP32Plain) {
    const bool kahan = p.precision == kP32Kahan;
    const float snap_f = has_snap ? p.snap_f[next_snap] : 0.0f;
    float tf = c.tf, cf = c.cf;
    for (int base = 0; base < n; base += 32) {
      const int cnt = n - base < 32 ? n - base : 32;
      const int k = slot(from + base + lane);
      const float tau_l = lane < cnt ? S.tauf[k] : 0.0f;
      float my_tf = 0.0f, my_cf = 0.0f;
      int cut = -1;
      float tcut = 0.0f;
      for (int j = 0; j < cnt; ++j) {
        const float tau = __shfl_sync(kFull, tau_l, j);
        float tfn, cfn = 0.0f;
        if (kahan) {
          const float yk = tau - cf;
          const float sum = tf + yk;
          cfn = (sum - tf) - yk;
          tfn = sum;
        } else {
          tfn = tf + tau;
        }
        if (detect && ((has_snap && tfn > snap_f) || tfn > p.t_end_f)) {
          cut = j;
          tcut = tfn;
          break;
        }
        tf = tfn;
        cf = cfn;
        if (lane == j) {
          my_tf = tf;
          my_cf = cf;
        }
      }
      if (lane < (cut >= 0 ? cut : cnt)) {
        S.tf[k] = my_tf;
        S.cf[k] = my_cf;
      }
      if (cut >= 0) {
        *t_cut = (double)tcut;
        return base + cut;
      }
    }
    return n;
  }
  const double snap_next = has_snap ? p.snap[next_snap] : 0.0;
  double t = c.t;
  for (int base = 0; base < n; base += 32) {
    const int cnt = n - base < 32 ? n - base : 32;
    const int k = slot(from + base + lane);
    const double tau_l =
        lane < cnt ? (p.precision == kP64LogSum ? S.taud[k] : (double)S.tauf[k]) : 0.0;
    double my_t = 0.0;
    int cut = -1;
    double tcut = 0.0;
    for (int j = 0; j < cnt; ++j) {
      const double tn = t + __shfl_sync(kFull, tau_l, j);
      if (detect && ((has_snap && snap_next < tn) || tn > p.t_end)) {
        cut = j;
        tcut = tn;
        break;
      }
      t = tn;
      if (lane == j) my_t = t;
    }
    if (lane < (cut >= 0 ? cut : cnt)) S.tnew[k] = my_t;
    if (cut >= 0) {
      *t_cut = tcut;
      return base + cut;
    }
  }
  return n;
}

}  // namespace lat

// Block: T step threads and one service warp.  The group's pending steps (at most 2T, with
// consecutive indices [lo, hi), two pool offsets per step thread) sit in a ring; each round:
//   A  (step threads) admits new steps up to 2T pending: the first Philox call of each (waiting
//      time, site, plane 0 of n) and the sum of their waiting times, from which a bound on the
//      last new event time tells whether they can pass a snapshot or t_end at all;
//   B  (only if they can: the service warp, others waiting) the clock in step order up to the
//      first step that would pass it: no step from there on is admitted until the snapshot;
//   C  (step threads) the cap check: the first new step that might push a neighbour above the cap
//      m is the last admitted until it has run (only it can raise the cap, which changes K and
//      the rate of every later step);
//   D  (step threads) one wave: every pending step that no earlier pending step's closed
//      neighbourhood (site and four neighbours) meets runs, up to one per step thread, all at
//      once; lo moves to the first step still pending;
//   meanwhile the service warp sums the clock of the new steps (when B did not) and replays the
//   steps finished before this round into the runs' totals.
// When every step before a stop (snapshot or t_end, a possible cap raise, the step budget) has
// run, the stop is handled and admission resumes.
template <int P, int KW>
__global__ void __launch_bounds__(kLatMaxBlock + 32) lattice_kernel(const __grid_constant__ LatticeLaunch p) {
  using namespace lat;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NT = blockDim.x, T = NT - 32, W = T >> 5, C = kLatSlots * T;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool service = warp == W;
  const int M = p.M;
  const LatSmem S = lat_smem(smem_raw, M);
  __shared__ int s_wcnt[kLatMaxBlock / 32];
  __shared__ double s_wsum[kLatMaxBlock / 32];
  __shared__ float s_wsumf[kLatMaxBlock / 32];
  __shared__ unsigned s_dom[32][2];
  __shared__ unsigned long long s_tot[32][3];
  __shared__ struct {
    int fcut, overflow, n_max, ncut, newlo, hadm;
    double t_cut;
    Clock clk;
  } sh;
  const PhiloxKey key{(uint32_t)p.seed, (uint32_t)(p.seed >> 32)};
  const bool f32 = p.precision == kP32Kahan || p.precision == kP32Plain;  // the clock is an fp32 sum
  const long long budget_stop = p.step_budget > 0 ? p.step_budget : kNoStop;

  for (long long gi = blockIdx.x; gi < p.n_groups; gi += gridDim.x) {
    const long long run0 = gi * 32;
    const int lanes = (int)(p.n_runs - run0 < 32 ? p.n_runs - run0 : 32);
    const uint32_t active = lanes == 32 ? kFull : ((1u << lanes) - 1u);
    const uint32_t g = (uint32_t)(p.group_base + gi);
    uint32_t* planes = p.planes + (size_t)gi * (size_t)M * (size_t)p.rec;

    // ---- initial state: planes from the counts, the cap table, the cap
    if (tid < 32) s_tot[tid][0] = s_tot[tid][1] = s_tot[tid][2] = 0ull;
    if (tid == 0) {
      sh.n_max = 0;
      sh.overflow = 0;
      sh.clk.t = 0.0;
      sh.clk.tf = 0.0f;
      sh.clk.cf = 0.0f;
    }
    __syncthreads();
    for (int i = tid; i < M; i += NT) {
      uint32_t L[P], D[P], A[P];
#pragma unroll
      for (int k = 0; k < P; ++k) L[k] = D[k] = A[k] = 0u;
      unsigned mx = 0;
      for (int l = 0; l < lanes; ++l) {
        const int* c = p.init_per_run ? p.init + ((size_t)(run0 + l) * M + i) * 3 : p.init + (size_t)i * 3;
        const unsigned cl = (unsigned)c[0], cd = (unsigned)c[1], ca = (unsigned)c[2];
        const unsigned tot = cl + cd + ca;
        mx = tot > mx ? tot : mx;
#pragma unroll
        for (int k = 0; k < P; ++k) {
          L[k] |= ((cl >> k) & 1u) << l;
          D[k] |= ((cd >> k) & 1u) << l;
          A[k] |= ((ca >> k) & 1u) << l;
        }
      }
      store_site<P>(planes + (size_t)i * p.rec, L, D, A);
      S.ub[i] = (uint16_t)mx;
      S.stamp[i] = kNoStamp;
      S.hopcnt[i] = 0u;
      atomicMax(&sh.n_max, (int)mx);
    }
    RunBook rb;
    rb.tot[0] = rb.tot[1] = rb.tot[2] = 0;
    rb.reactions = rb.hops = 0;
    rb.t_h = __longlong_as_double(0x7FF0000000000000ll);  // +inf
    rb.outcome = -1;
    // each run's lattice totals: warp w sums run `lane`'s counts over its share of the sites
    {
      long long part[3] = {0, 0, 0};
      if (lane < lanes) {
        const int NW = NT >> 5;
        for (int i = warp; i < M; i += NW) {
          const int* c = p.init_per_run ? p.init + ((size_t)(run0 + lane) * M + i) * 3 : p.init + (size_t)i * 3;
          part[0] += c[0];
          part[1] += c[1];
          part[2] += c[2];
        }
        atomicAdd(&s_tot[lane][0], (unsigned long long)part[0]);
        atomicAdd(&s_tot[lane][1], (unsigned long long)part[1]);
        atomicAdd(&s_tot[lane][2], (unsigned long long)part[2]);
      }
    }
    __syncthreads();
    if (service && lane < lanes) {
      rb.tot[0] = (long long)s_tot[lane][0];
      rb.tot[1] = (long long)s_tot[lane][1];
      rb.tot[2] = (long long)s_tot[lane][2];
      const int kinds = (rb.tot[0] > 0) + (rb.tot[1] > 0) + (rb.tot[2] > 0);
      if (kinds <= 1) {
        rb.t_h = 0.0;
        rb.outcome = rb.tot[0] ? 0 : (rb.tot[1] ? 1 : (rb.tot[2] ? 2 : -1));
      }
    }
    const int n_max = sh.n_max;
    int b = 0;  // the cap's level: the first cap at or above every site count
    while (b + 1 < p.n_levels && p.cap[b].m < (unsigned)n_max) ++b;
    int status = p.cap[b].m < (unsigned)n_max || p.cap[b].m > (1u << (P - 1)) ? kLatBadInit : kLatOk;
    long long lo = 0, hi = 0, rep_lo = 0, stop = budget_stop;
    int reason = p.step_budget > 0 ? kStopBudget : kStopNone;
    double t_cut = 0.0;
    long long rounds = 0, flags = 0, slow_rounds = 0;
    int raises = 0, next_snap = 0;

    while (status == kLatOk) {
      // ---- a stop whose every earlier step has run
      if (lo == hi && hi == stop) {
        const bool raised = sh.overflow != 0;  // the last step, a possible cap raise, raised it
        if (raised) {
          ++b;
          ++raises;
        }
        if (reason == kStopBudget) {
          status = kLatTimeout;
          break;
        }
        // a crossing found at the old rate is found again at the new one
        if (reason == kStopCross && !raised) {
          // snapshots before the crossing step's event, after every earlier step's events
          if (service) replay(rb, S, rep_lo, lo, lane, lane < lanes, f32);
          rep_lo = lo;
          while (next_snap < p.n_snap && p.snap[next_snap] < t_cut) {
            if (tid < 32) s_dom[tid][0] = s_dom[tid][1] = 0u;
            __syncthreads();
            unsigned myL = 0, myD = 0;
            for (int base_s = warp * 32; base_s < M; base_s += NT) {
              const int i = base_s + lane;
              uint32_t gtL = 0u, gtD = 0u;
              if (i < M) {
                uint32_t L[P], D[P], A[P];
                load_site<P>(planes + (size_t)i * p.rec, L, D, A);
                gtL = bs::less_than<P>(D, L);
                gtD = bs::less_than<P>(L, D);
              }
              for (int l = 0; l < 32; ++l) {
                const unsigned cL = __popc(__ballot_sync(kFull, (gtL >> l) & 1u));
                const unsigned cD = __popc(__ballot_sync(kFull, (gtD >> l) & 1u));
                if (lane == l) {
                  myL += cL;
                  myD += cD;
                }
              }
            }
            atomicAdd(&s_dom[lane][0], myL);
            atomicAdd(&s_dom[lane][1], myD);
            __syncthreads();
            if (service && lane < lanes) {
              const size_t row = (size_t)next_snap * (size_t)p.n_runs + (size_t)(run0 + lane);
              if (p.snap_totals) {
                p.snap_totals[row * 3 + 0] = rb.tot[0];
                p.snap_totals[row * 3 + 1] = rb.tot[1];
                p.snap_totals[row * 3 + 2] = rb.tot[2];
              }
              if (p.snap_domains) {
                p.snap_domains[row * 2 + 0] = (int)s_dom[lane][0];
                p.snap_domains[row * 2 + 1] = (int)s_dom[lane][1];
              }
            }
            __syncthreads();
            ++next_snap;
          }
          if (t_cut > p.t_end) break;
        }
        __syncthreads();  // every thread has read sh.overflow
        if (tid == 0) sh.overflow = 0;
        stop = budget_stop;
        reason = p.step_budget > 0 ? kStopBudget : kStopNone;
      }
      const LatCap cp = p.cap[b < p.n_levels ? b : p.n_levels - 1];
      if (cp.K > 32) {
        status = kLatRange;
        break;
      }
      if (b >= p.n_levels || cp.m > (1u << (P - 1)) || cp.K > KW) {
        status = kLatCapacity;
        break;
      }
      // ---- A: admit new steps (pool offsets tid and tid + T of each step thread)
      long long room = (long long)C - (hi - lo);
      if (stop - hi < room) room = stop - hi;
      int n_new = (int)room;
      if (!service) {
        double tau = 0.0;
        float tauf = 0.0f;
#pragma unroll
        for (int j = 0; j < kLatSlots; ++j) {
          const int idx = tid + j * T;
          if (idx < n_new) {
            const long long s = hi + idx;
            const int k = slot(s);
            const uint4 w = philox4x32_10(stream_counter(g, (unsigned long long)s, 0u, 2u, 0u), key);
            if (p.precision == kP64LogSum) {
              const unsigned long long x = ((unsigned long long)w.y << 21) | (unsigned long long)(w.x >> 11);
              const double u = (double)(x + 1ull) * 0x1p-53;
              const double td = -log(u) / cp.lambda;
              S.taud[k] = td;
              tau += td;
            } else {
              const float u = (float)((w.y >> 8) + 1u) * 0x1p-24f;
              const float tf = -logf(u) * cp.inv_lambda_f;
              S.tauf[k] = tf;
              tauf += tf;
              if (p.precision == kP32D64Acc) tau += (double)tf;
            }
            S.sigma[k] = (int)(w.z & (uint32_t)(M - 1));
            S.w3[k] = w.w;
            S.done[k] = 0;
          }
        }
        if (f32) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) tauf += __shfl_xor_sync(kFull, tauf, o);
          if (lane == 0) s_wsumf[warp] = tauf;
        } else {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) tau += __shfl_xor_sync(kFull, tau, o);
          if (lane == 0) s_wsum[warp] = tau;
        }
        if (tid == 0) {
          sh.fcut = C;
          sh.newlo = C;
        }
      }
      __syncthreads();
      // a bound on the last new event time, above the sequential sum's rounding (at most one
      // rounding a step, and the tree sum's own, well inside the margin)
      const Clock c0 = sh.clk;
      const bool has_snap = next_snap < p.n_snap;
      bool slow;
      if (f32) {
        float sum = 0.0f;
        for (int w = 0; w < W; ++w) sum += s_wsumf[w];
        const float bound = (c0.tf + fabsf(c0.cf) + sum) * (1.0f + (float)(C + 2) * 0x1p-21f);
        slow = n_new > 0 && ((has_snap && !(bound <= p.snap_f[next_snap])) || !(bound <= p.t_end_f));
      } else {
        double sum = 0.0;
        for (int w = 0; w < W; ++w) sum += s_wsum[w];
        const double bound = (c0.t + sum) * (1.0 + (double)(C + 2) * 0x1p-50);
        const double snap_next = has_snap ? p.snap[next_snap] : 0.0;
        slow = n_new > 0 && ((has_snap && !(bound <= snap_next)) || !(bound <= p.t_end));
      }
      if (slow) {
        ++slow_rounds;
        // ---- B: the exact clock finds the first new step that would pass a time point
        if (service) {
          double tc = 0.0;
          const int nc = clock_run(p, S, hi, n_new, true, has_snap, next_snap, c0, &tc, lane);
          if (lane == 0) {
            sh.ncut = nc;
            sh.t_cut = tc;
          }
        }
        __syncthreads();
        if (sh.ncut < n_new) {
          n_new = sh.ncut;
          stop = hi + n_new;
          reason = kStopCross;
          t_cut = sh.t_cut;
        }
      }
      const int m = (int)cp.m;
      const long long lo0 = lo, hi0 = hi;
      if (!service) {
        // ---- C: the cap check of the new steps
        int nb[kLatSlots][4];
#pragma unroll
        for (int j = 0; j < kLatSlots; ++j) {
          const int idx = tid + j * T;
          if (idx < n_new) {
            neighbours(p, S.sigma[slot(hi0 + idx)], nb[j]);
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(&S.hopcnt[nb[j][k]], 1u);
          }
        }
        step_sync(T);
#pragma unroll
        for (int j = 0; j < kLatSlots; ++j) {
          const int idx = tid + j * T;
          if (idx < n_new) {
            bool flag = false;
#pragma unroll
            for (int k = 0; k < 4; ++k) flag |= (unsigned)S.ub[nb[j][k]] + S.hopcnt[nb[j][k]] > (unsigned)m;
            if (flag) atomicMin(&sh.fcut, idx);
          }
        }
        step_sync(T);
        const int f = sh.fcut;
        const int n_adm = f < n_new ? f + 1 : n_new;
#pragma unroll
        for (int j = 0; j < kLatSlots; ++j) {
          const int idx = tid + j * T;
          if (idx >= n_adm && idx < n_new) {
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicSub(&S.hopcnt[nb[j][k]], 1u);
          }
        }
        if (tid == 0) sh.hadm = n_adm;
        const long long hi1 = hi0 + n_adm;
        // ---- D: one wave over the pending steps [lo, hi1) (offsets tid and tid + T)
        const int np = (int)(hi1 - lo0);
        int ks[kLatSlots], c5[kLatSlots][5];
        bool mine[kLatSlots], ready[kLatSlots];
#pragma unroll
        for (int j = 0; j < kLatSlots; ++j) {
          const int off = tid + j * T;
          ks[j] = slot(lo0 + off);
          mine[j] = off < np && !S.done[ks[j]];
          if (mine[j]) {
            c5[j][0] = S.sigma[ks[j]];
            int n4[4];
            neighbours(p, c5[j][0], n4);
#pragma unroll
            for (int k = 0; k < 4; ++k) c5[j][k + 1] = n4[k];
#pragma unroll
            for (int k = 0; k < 5; ++k) atomicMin(&S.stamp[c5[j][k]], (uint32_t)off);
            if (off >= (int)(hi0 - lo0)) {  // admitted this round: bring its records to L1
#pragma unroll
              for (int k = 0; k < 5; ++k) {
                const uint32_t* r = planes + (size_t)c5[j][k] * p.rec;
                asm volatile("prefetch.global.L1 [%0];" ::"l"(r));
                asm volatile("prefetch.global.L1 [%0];" ::"l"(r + p.rec - 1));
              }
            }
          }
        }
        step_sync(T);
        uint32_t bal[kLatSlots];
        int mycount = 0;
#pragma unroll
        for (int j = 0; j < kLatSlots; ++j) {
          const int off = tid + j * T;
          ready[j] = mine[j];
          if (mine[j]) {
#pragma unroll
            for (int k = 0; k < 5; ++k) ready[j] &= S.stamp[c5[j][k]] == (uint32_t)off;
          }
          bal[j] = __ballot_sync(kFull, ready[j]);
          mycount += __popc(bal[j]);
        }
        if (lane == 0) s_wcnt[warp] = mycount;
        step_sync(T);
        int base_w = 0, total = 0;
        for (int w = 0; w < W; ++w) {
          const int cw = s_wcnt[w];
          base_w += w < warp ? cw : 0;
          total += cw;
        }
#pragma unroll
        for (int j = 0; j < kLatSlots; ++j) {
          if (ready[j]) S.ready[base_w + __popc(bal[j] & ((1u << lane) - 1u))] = tid + j * T;
          base_w += __popc(bal[j]);
          if (mine[j]) {
#pragma unroll
            for (int k = 0; k < 5; ++k) S.stamp[c5[j][k]] = kNoStamp;
          }
        }
        step_sync(T);
        // at most one ready step per thread runs; ready steps left over stay ready for the next round
        if (tid < total) {
          const long long s = lo0 + S.ready[tid];
          const int k = slot(s);
          StepArgs a;
          a.group = g;
          a.step = s;
          a.sigma = S.sigma[k];
          a.w3 = S.w3[k];
          a.bh = cp.bh;
          a.m = cp.m;
          a.K = cp.K;
          a.hop_slots = cp.hop_slots;
          a.planes = planes;
          const StepOut o = step<P, KW>(p, a, S.ub);
          S.x1[k] = o.x1 & active;
          S.x2[k] = o.x2 & active;
          S.x3[k] = o.x3 & active;
          S.hop[k] = o.hop & active;
          S.done[k] = 1;
          int n4[4];
          neighbours(p, a.sigma, n4);
#pragma unroll
          for (int j = 0; j < 4; ++j) atomicSub(&S.hopcnt[n4[j]], 1u);
          if (o.overflow) atomicOr(&sh.overflow, 1);
        }
        step_sync(T);
#pragma unroll
        for (int j = 0; j < kLatSlots; ++j)
          if (mine[j] && !S.done[ks[j]]) atomicMin(&sh.newlo, tid + j * T);
      } else {
        // the service warp: the clock of the new steps (unless B summed it), then the steps
        // finished before this round into the runs' totals
        if (!slow) {
          double tc = 0.0;
          clock_run(p, S, hi0, n_new, false, false, 0, c0, &tc, lane);
        }
        __syncwarp();
        if (lo0 > rep_lo) replay(rb, S, rep_lo, lo0, lane, lane < lanes, f32);
      }
      __syncthreads();
      // ---- advance
      const int n_adm = sh.hadm;
      hi = hi0 + n_adm;
      lo = sh.newlo < C ? lo0 + sh.newlo : hi;
      rep_lo = lo0;
      if (sh.fcut < n_new) {  // a possible cap raise, admitted last: nothing after it until it has run
        ++flags;
        if (hi < stop) {
          stop = hi;
          reason = kStopFlag;
        }
      }
      if (service && lane == 0 && n_adm > 0) {
        const int k = slot(hi - 1);
        if (f32) {
          sh.clk.tf = S.tf[k];
          sh.clk.cf = S.cf[k];
        } else {
          sh.clk.t = S.tnew[k];
        }
      }
      ++rounds;
      __syncthreads();  // every thread has read sh before it is written again
    }
    if (service && lo > rep_lo) replay(rb, S, rep_lo, lo, lane, lane < lanes, f32);

    // ---- outputs of the group
    if (service) {
      if (lane < lanes) {
        const size_t r = (size_t)(run0 + lane);
        p.t_homochiral[r] = rb.t_h;
        p.outcome[r] = (signed char)rb.outcome;
        p.events[2 * r] = rb.reactions;
        p.events[2 * r + 1] = rb.hops;
      }
      long long rs = lane < lanes ? rb.reactions : 0, hs = lane < lanes ? rb.hops : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        rs += __shfl_xor_sync(kFull, rs, o);
        hs += __shfl_xor_sync(kFull, hs, o);
      }
      if (lane == 0) {
        atomicAdd(&p.counters[kLatReactions], (unsigned long long)rs);
        atomicAdd(&p.counters[kLatHops], (unsigned long long)hs);
      }
    }
    if (tid == 0) {
      p.group_info[3 * gi] = lo;
      p.group_info[3 * gi + 1] = b < p.n_levels ? p.cap[b].m : 2 * p.cap[p.n_levels - 1].m;
      p.group_info[3 * gi + 2] = status;
      atomicAdd(&p.counters[kLatGroupSteps], (unsigned long long)lo);
      atomicAdd(&p.counters[kLatRounds], (unsigned long long)rounds);
      atomicAdd(&p.counters[kLatClockRounds], (unsigned long long)slow_rounds);
      atomicAdd(&p.counters[kLatCapRaises], (unsigned long long)raises);
      atomicAdd(&p.counters[kLatFlagged], (unsigned long long)flags);
      if (status != kLatOk) atomicAdd(&p.counters[kLatErrors], 1ull);
    }
    if (p.final_counts) {
      for (int i = tid; i < M; i += NT) {
        uint32_t L[P], D[P], A[P];
        load_site<P>(planes + (size_t)i * p.rec, L, D, A);
        for (int l = 0; l < lanes; ++l) {
          int cl = 0, cd = 0, ca = 0;
#pragma unroll
          for (int k = 0; k < P; ++k) {
            cl |= (int)((L[k] >> l) & 1u) << k;
            cd |= (int)((D[k] >> l) & 1u) << k;
            ca |= (int)((A[k] >> l) & 1u) << k;
          }
          int* out = p.final_counts + ((size_t)(run0 + l) * M + i) * 3;
          out[0] = cl;
          out[1] = cd;
          out[2] = ca;
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace bitssa
