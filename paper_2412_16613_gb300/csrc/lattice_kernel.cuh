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
// depend on the state, so a window of consecutive steps (one per thread) is drawn at once:
//   A. every thread draws its step's first Philox call: the waiting time and the site;
//   B. one thread adds the waiting times in step order (the group clock of Eq. equation-tau and
//      Eq. eq-update-time) and cuts the window before the first step whose event would pass a
//      snapshot or t_end, or that the step budget forbids;
//   C. the window is cut after the first step that might push a neighbour above the cap m (only
//      such a step can raise the cap, which changes K and the rate of every later step);
//   D. the steps run in waves: a step waits for every earlier step of the window whose closed
//      neighbourhood (the site and its four neighbours) meets its own, found with per-site
//      stamps in shared memory, so steps of one wave touch disjoint sites and commute with every
//      step left for later waves.  Each step is the bit-sliced event of Sec. 4 at its site:
//      comparisons of n with the hop slots and with the cumulative slots rho_r S_r (S_r from
//      bit-sliced schoolbook products of the site's count planes, Sec. 4.1), masked count updates
//      at the site (Eq. equation-v) and masked increments at the neighbours;
//   E. warp 0, thread l = run l, replays the window's event masks in step order to keep run l's
//      lattice totals and the time it first holds one species.
// Every run therefore takes exactly the trajectory of the serial definition; only independent
// steps are reordered.
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

// Lanes whose value exceeds 2^b (b < W).
template <int W>
__device__ __forceinline__ uint32_t above_pow2(const uint32_t (&x)[W], int b) {
  uint32_t high = 0u, low = 0u, at = 0u;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    if (i > b) high |= x[i];
    else if (i == b) at = x[i];
    else low |= x[i];
  }
  return high | (at & low);
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
  int b, K;              // cap bits, planes of n
  uint32_t hop_slots;    // 4 rho_h 2^b
  uint32_t* planes;      // the group's site records
};

struct StepOut {
  uint32_t x1, x2, x3, hop;  // runs that took reaction 1, 2, 3, or hopped
  bool overflow;             // a neighbour of some run went above the cap
  unsigned ub_sigma;         // largest site total at sigma after the step
};

// One step of the group at its site, all 32 runs at once; updates the site and the neighbours
// a run hops to, and the cap table ub.
template <int P, int KW>
__device__ __forceinline__ StepOut step(const LatticeLaunch& p, const StepArgs& a, uint16_t* ub) {
  constexpr int SW = 2 * P - 1;  // S_3 <= m^2 / 3 < 2^(2P - 2)
  const PhiloxKey key{(uint32_t)p.seed, (uint32_t)(p.seed >> 32)};
  // (1) the planes of n: word 3 + i is plane i, i < K; planes at and above K are zero
  uint32_t n[KW];
  n[0] = a.K > 0 ? a.w3 : 0u;
#pragma unroll
  for (int c = 1; 4 * c - 3 < KW; ++c) {
    if (4 * c - 3 < a.K) {
      const uint4 w = philox4x32_10(stream_counter(a.group, (unsigned long long)a.step, 0u, 2u, (uint32_t)c), key);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 4 * c - 3 + e;
        if (i < KW) n[i] = i < a.K ? word_of(w, e) : 0u;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 4 * c - 3 + e;
        if (i < KW) n[i] = 0u;
      }
    }
  }
  uint32_t* rec = a.planes + (size_t)a.sigma * p.rec;
  uint32_t L[P], D[P], A[P];
  load_site<P>(rec, L, D, A);

  // (2) hops: n < 4 rho_h m; direction n & 3, molecule (n >> 2) & (m - 1) against L, L + D, L + D + A
  const uint32_t is_hop = bs::less_than_const<KW>(n, a.hop_slots);
  uint32_t mol[P], LD[P], T[P];
#pragma unroll
  for (int i = 0; i < P; ++i) mol[i] = i < a.b ? n[2 + i] : 0u;
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
        if (above_pow2<P>(T2, a.b)) o.overflow = true;
        ub[nb[k]] = (uint16_t)lane_max<P>(T2);
      }
    }
  }
  return o;
}

}  // namespace lat

// Shared-memory layout of a block: per site, the stamp and hop-count tables (uint32) and the cap
// table ub (uint16, the largest site total over the group's runs); per step of a window, the clock
// and the event masks.
struct LatSmem {
  uint32_t* stamp;
  uint32_t* hopcnt;
  uint16_t* ub;
  double* tnew;   // time after step i's event
  double* taud;   // fp64 waiting times
  float* tauf;    // fp32 waiting times
  float* tf;      // fp32 clock after step i (Kahan sum or plain sum)
  float* cf;      // Kahan compensation after step i
  int* sigma;
  uint32_t* w3;
  uint32_t* x1;
  uint32_t* x2;
  uint32_t* x3;
  uint32_t* hop;
  int* ready;
  int* done;
};

__device__ __forceinline__ LatSmem lat_smem(unsigned char* base, int M, int T) {
  LatSmem s;
  s.stamp = reinterpret_cast<uint32_t*>(base);
  s.hopcnt = s.stamp + M;
  s.ub = reinterpret_cast<uint16_t*>(s.hopcnt + M);
  unsigned char* w = reinterpret_cast<unsigned char*>(s.ub + ((M + 3) & ~3));
  s.tnew = reinterpret_cast<double*>(w);
  s.taud = s.tnew + T;
  s.tauf = reinterpret_cast<float*>(s.taud + T);
  s.tf = s.tauf + T;
  s.cf = s.tf + T;
  s.sigma = reinterpret_cast<int*>(s.cf + T);
  s.w3 = reinterpret_cast<uint32_t*>(s.sigma + T);
  s.x1 = s.w3 + T;
  s.x2 = s.x1 + T;
  s.x3 = s.x2 + T;
  s.hop = s.x3 + T;
  s.ready = reinterpret_cast<int*>(s.hop + T);
  s.done = s.ready + T;
  return s;
}

__host__ __device__ constexpr int lat_smem_bytes(int M, int T) {
  return 4 * M + 4 * M + 2 * ((M + 3) & ~3) + T * (8 + 8 + 4 + 4 + 4 + 4 + 4 + 16 + 4 + 4);
}

template <int P, int KW>
__global__ void __launch_bounds__(kLatMaxBlock) lattice_kernel(const __grid_constant__ LatticeLaunch p) {
  using namespace lat;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int M = p.M;
  const LatSmem S = lat_smem(smem_raw, M, T);
  __shared__ int s_wcnt[kLatMaxBlock / 32];
  __shared__ unsigned s_dom[32][2];
  __shared__ struct {
    int cut, reason, ovcut, overflow, n_max;
    double t_cut;
  } sh;
  const PhiloxKey key{(uint32_t)p.seed, (uint32_t)(p.seed >> 32)};

  for (long long gi = blockIdx.x; gi < p.n_groups; gi += gridDim.x) {
    const long long run0 = gi * 32;
    const int lanes = (int)(p.n_runs - run0 < 32 ? p.n_runs - run0 : 32);
    const uint32_t active = lanes == 32 ? kFull : ((1u << lanes) - 1u);
    const uint32_t g = (uint32_t)(p.group_base + gi);
    uint32_t* planes = p.planes + (size_t)gi * (size_t)M * (size_t)p.rec;

    // ---- initial state: planes from the counts, the cap table, the cap
    if (tid == 0) sh.n_max = 0;
    __syncthreads();
    for (int i = tid; i < M; i += T) {
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
    // run `lane` of the group, kept by warp 0
    long long tot[3] = {0, 0, 0}, reactions = 0, hops = 0;
    double t_h = __longlong_as_double(0x7FF0000000000000ll);  // +inf
    int outcome = -1;
    if (warp == 0 && lane < lanes) {
      for (int i = 0; i < M; ++i) {
        const int* c = p.init_per_run ? p.init + ((size_t)(run0 + lane) * M + i) * 3 : p.init + (size_t)i * 3;
        tot[0] += c[0];
        tot[1] += c[1];
        tot[2] += c[2];
      }
      const int kinds = (tot[0] > 0) + (tot[1] > 0) + (tot[2] > 0);
      if (kinds <= 1) {
        t_h = 0.0;
        outcome = tot[0] ? 0 : (tot[1] ? 1 : (tot[2] ? 2 : -1));
      }
    }
    __syncthreads();
    const int n_max = sh.n_max;
    int b = n_max > 1 ? bit_length((long long)(n_max - 1)) : 0;
    int status = b > P - 1 ? kLatBadInit : kLatOk;
    long long s0 = 0, windows = 0, waves = 0, cuts = 0;
    int raises = 0, next_snap = 0;
    double t = 0.0;
    float t_f = 0.0f, c_f = 0.0f;

    while (status == kLatOk) {
      if (p.step_budget > 0 && s0 >= p.step_budget) {
        status = kLatTimeout;
        break;
      }
      const LatCap cp = p.cap[b];
      if (cp.K > 32) {
        status = kLatRange;
        break;
      }
      if (b > P - 1 || cp.K > KW) {
        status = kLatCapacity;
        break;
      }
      // ---- A: the waiting time, the site and plane 0 of n of each step of the window
      {
        const unsigned long long s = (unsigned long long)(s0 + tid);
        const uint4 w = philox4x32_10(stream_counter(g, s, 0u, 2u, 0u), key);
        if (p.precision == kP64LogSum) {
          const unsigned long long x = ((unsigned long long)w.y << 21) | (unsigned long long)(w.x >> 11);
          const double u = (double)(x + 1ull) * 0x1p-53;
          S.taud[tid] = -log(u) / cp.lambda;
        } else {
          const float u = (float)((w.y >> 8) + 1u) * 0x1p-24f;
          S.tauf[tid] = -logf(u) * cp.inv_lambda_f;
        }
        S.sigma[tid] = (int)(w.z & (uint32_t)(M - 1));
        S.w3[tid] = w.w;
        S.done[tid] = 0;
      }
      __syncthreads();
      // ---- B: the group clock in step order; the window ends before a crossing or the budget
      if (tid == 0) {
        int cut = T, reason = 0;
        double tc = 0.0, tt = t;
        float ttf = t_f, tcf = c_f;
        const double snap_next = next_snap < p.n_snap ? p.snap[next_snap] : 0.0;
        for (int i = 0; i < T; ++i) {
          if (p.step_budget > 0 && s0 + i >= p.step_budget) {
            cut = i;
            break;
          }
          double tn;
          float tfn = 0.0f, cfn = 0.0f;
          if (p.precision == kP64LogSum) {
            tn = tt + S.taud[i];
          } else {
            const float tau = S.tauf[i];
            if (p.precision == kP32Kahan) {
              const float yk = tau - tcf;
              const float sum = ttf + yk;
              cfn = (sum - ttf) - yk;
              tfn = sum;
              tn = (double)sum;
            } else if (p.precision == kP32Plain) {
              tfn = ttf + tau;
              tn = (double)tfn;
            } else {
              tn = tt + (double)tau;
            }
          }
          if ((next_snap < p.n_snap && snap_next < tn) || tn > p.t_end) {
            cut = i;
            reason = kCross;
            tc = tn;
            break;
          }
          S.tnew[i] = tn;
          S.tf[i] = tfn;
          S.cf[i] = tcf = cfn;
          tt = tn;
          ttf = tfn;
        }
        sh.cut = cut;
        sh.reason = reason;
        sh.t_cut = tc;
        sh.overflow = 0;
        sh.ovcut = T;
      }
      __syncthreads();
      const int cut = sh.cut;
      const int m = 1 << b;
      // ---- C: the first step that might raise the cap ends the window
      int nb[4] = {0, 0, 0, 0};
      if (tid < cut) {
        neighbours(p, S.sigma[tid], nb);
#pragma unroll
        for (int k = 0; k < 4; ++k) atomicAdd(&S.hopcnt[nb[k]], 1u);
      }
      __syncthreads();
      if (tid < cut) {
        bool flag = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) flag |= (unsigned)S.ub[nb[k]] + S.hopcnt[nb[k]] > (unsigned)m;
        if (flag) atomicMin(&sh.ovcut, tid);
      }
      __syncthreads();
      if (tid < cut) {
#pragma unroll
        for (int k = 0; k < 4; ++k) S.hopcnt[nb[k]] = 0u;
      }
      const int e = sh.ovcut + 1 < cut ? sh.ovcut + 1 : cut;
      if (e < cut) ++cuts;
      // ---- D: waves of steps whose closed neighbourhoods meet no earlier pending step's
      int done_n = 0;
      while (done_n < e) {
        const bool mine = tid < e && !S.done[tid];
        int c5[5];
        if (mine) {
          c5[0] = S.sigma[tid];
          int n4[4];
          neighbours(p, c5[0], n4);
#pragma unroll
          for (int k = 0; k < 4; ++k) c5[k + 1] = n4[k];
#pragma unroll
          for (int k = 0; k < 5; ++k) atomicMin(&S.stamp[c5[k]], (uint32_t)tid);
        }
        __syncthreads();
        bool ready = false;
        if (mine) {
          ready = true;
#pragma unroll
          for (int k = 0; k < 5; ++k) ready &= S.stamp[c5[k]] == (uint32_t)tid;
        }
        const uint32_t bal = __ballot_sync(kFull, ready);
        if (lane == 0) s_wcnt[warp] = __popc(bal);
        __syncthreads();
        int base = 0, total = 0;
        for (int w = 0; w < (T >> 5); ++w) {
          const int cw = s_wcnt[w];
          base += w < warp ? cw : 0;
          total += cw;
        }
        if (ready) S.ready[base + __popc(bal & ((1u << lane) - 1u))] = tid;
        if (mine) {
#pragma unroll
          for (int k = 0; k < 5; ++k) S.stamp[c5[k]] = kNoStamp;
        }
        __syncthreads();
        if (tid < total) {
          const int i = S.ready[tid];
          StepArgs a;
          a.group = g;
          a.step = s0 + i;
          a.sigma = S.sigma[i];
          a.w3 = S.w3[i];
          a.b = b;
          a.K = cp.K;
          a.hop_slots = cp.hop_slots;
          a.planes = planes;
          const StepOut o = step<P, KW>(p, a, S.ub);
          S.x1[i] = o.x1 & active;
          S.x2[i] = o.x2 & active;
          S.x3[i] = o.x3 & active;
          S.hop[i] = o.hop & active;
          S.done[i] = 1;
          if (o.overflow) atomicOr(&sh.overflow, 1);
        }
        __syncthreads();
        done_n += total;
        ++waves;
      }
      // ---- E: run `lane`'s totals and first single-species time, in step order
      if (warp == 0 && lane < lanes) {
        const uint32_t bit = 1u << lane;
        for (int i = 0; i < e; ++i) {
          const uint32_t r1 = S.x1[i] & bit, r2 = S.x2[i] & bit, r3 = S.x3[i] & bit;
          hops += (S.hop[i] & bit) ? 1 : 0;
          if (r1 | r2 | r3) {
            ++reactions;
            if (r1) {
              ++tot[0];
              --tot[2];
            } else if (r2) {
              ++tot[1];
              --tot[2];
            } else {
              --tot[0];
              --tot[1];
              tot[2] += 2;
            }
            if (outcome == -1 && (tot[0] > 0) + (tot[1] > 0) + (tot[2] > 0) == 1) {
              t_h = S.tnew[i];
              outcome = tot[0] ? 0 : (tot[1] ? 1 : 2);
            }
          }
        }
      }
      // ---- F: advance the group
      if (tid == 0 && e > 0) {
        t = S.tnew[e - 1];
        t_f = S.tf[e - 1];
        c_f = S.cf[e - 1];
      }
      s0 += e;
      ++windows;
      const bool overflow = sh.overflow != 0;
      const bool cross = e == cut && !overflow && sh.reason == kCross;
      const double t_cut = sh.t_cut;
      __syncthreads();  // every thread has read sh before thread 0 writes it again
      if (overflow) {
        ++b;
        ++raises;
        continue;
      }
      if (!cross) continue;
      // snapshots before the crossing step's event: lattice totals and domain counts of every run
      while (next_snap < p.n_snap && p.snap[next_snap] < t_cut) {
        if (tid < 32) s_dom[tid][0] = s_dom[tid][1] = 0u;
        __syncthreads();
        unsigned myL = 0, myD = 0;
        for (int base = warp * 32; base < M; base += T) {
          const int i = base + lane;
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
        if (warp == 0 && lane < lanes) {
          const size_t row = (size_t)next_snap * (size_t)p.n_runs + (size_t)(run0 + lane);
          if (p.snap_totals) {
            p.snap_totals[row * 3 + 0] = tot[0];
            p.snap_totals[row * 3 + 1] = tot[1];
            p.snap_totals[row * 3 + 2] = tot[2];
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

    // ---- outputs of the group
    if (warp == 0) {
      if (lane < lanes) {
        const size_t r = (size_t)(run0 + lane);
        p.t_homochiral[r] = t_h;
        p.outcome[r] = (signed char)outcome;
        p.events[2 * r] = reactions;
        p.events[2 * r + 1] = hops;
      }
      long long rs = lane < lanes ? reactions : 0, hs = lane < lanes ? hops : 0;
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
      p.group_info[3 * gi] = s0;
      p.group_info[3 * gi + 1] = b;
      p.group_info[3 * gi + 2] = status;
      atomicAdd(&p.counters[kLatGroupSteps], (unsigned long long)s0);
      atomicAdd(&p.counters[kLatWindows], (unsigned long long)windows);
      atomicAdd(&p.counters[kLatWaves], (unsigned long long)waves);
      atomicAdd(&p.counters[kLatCapRaises], (unsigned long long)raises);
      atomicAdd(&p.counters[kLatCutWindows], (unsigned long long)cuts);
      if (status != kLatOk) atomicAdd(&p.counters[kLatErrors], 1ull);
    }
    if (p.final_counts) {
      for (int i = tid; i < M; i += T) {
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
