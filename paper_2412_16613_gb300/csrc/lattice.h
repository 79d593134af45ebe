// lattice.h -- structures shared by the host runtime and the sm_103a kernel of Frank's model on
// a periodic lattice (ssa_lattice_* in bitssa.h).  Not part of the C ABI.
//
// The paper motivates compartments and non-well-mixed systems (Sec. 1, Sec. 6) without giving an
// algorithm.  The library's reading: sites (x, y) of an lx x ly torus, both powers of two, each
// with counts (L, D, A) and Frank's three reactions (Eqs. 1-3, Omega = 1 per site); every
// molecule hops to each of its four neighbours at rate d.  A group of 32 runs shares the site of
// each step, and each run draws its own event at that site from its bit of the step's words, the
// binary-word representation of Sec. 4 with one word per count plane per site.  Uniformisation
// is exact: with u = min(k_max, d), rho_r = k_max / u and rho_h = d / u integers and an
// occupancy cap m = 2^b at or above every site count of the group's runs, a site holds
// c(m) = 4 rho_h 2^bh + rho_r m (m - 1) / 2 slots (2^bh the power of two at or above m), the group
// draws K = bit_length(c(m) - 1) planes, and its steps come at rate Lambda = M 2^K u.  Caps are 1 .. 8
// and the numbers with a two-bit mantissa, (4 + j) 2^e; a hop that leaves a site of a run above m
// moves m to the next cap from the next step on.
#pragma once

#include <cstdint>

namespace bitssa {

constexpr int kLatMaxPlanes = 16;   // count planes of the widest instantiation (caps up to 2^15)
constexpr int kLatMaxSites = 16384; // per-site shared-memory tables of one block
constexpr int kLatMaxSnap = 64;
constexpr int kLatMaxBlock = 224;   // pending steps of a group at most (step threads of a block; one more warp serves)
constexpr int kLatDefaultWindow = 224;
constexpr int kLatRhoBits = 16;     // rho_r below 2^16
constexpr int kLatCounters = 8;
constexpr int kLatMaxLevels = 64;   // caps 1 .. 8 and four per octave up to 2^16
constexpr int kLatSlots = 2;        // pending steps per step thread: a group's pool holds kLatSlots T
// Steps of a group held at once in shared memory: the pending steps and the steps finished but not
// yet replayed into the runs' totals.  A power of two, at least twice the largest pool.
constexpr int kLatRing = 1024;
static_assert(kLatRing >= 2 * kLatSlots * kLatMaxBlock, "the ring must hold two pools");
// Bytes of one ring entry: the clock after the step (fp64), its waiting time in fp64 and fp32, the
// fp32 clock and compensation, the site, plane 0 of n, four event masks, the done flag.
constexpr int kLatRingEntryBytes = 8 + 8 + 4 + 4 + 4 + 4 + 4 + 16 + 4;
// Dynamic shared memory of a block with T step threads for a lattice of M sites: per site the stamp
// and hop-count tables (uint32) and the cap table (uint16), the ring, two ready-list entries per
// step thread.
__host__ __device__ constexpr int lat_smem_bytes(int M, int T) {
  return 4 * M + 4 * M + 2 * ((M + 3) & ~3) + kLatRing * kLatRingEntryBytes + 4 * kLatSlots * T;
}

// Indices into the lattice kernel's counter array (uint64).
enum LatCounter {
  kLatGroupSteps = 0,   // steps of every group
  kLatRounds = 1,       // rounds (admission of new steps and one wave of the ready ones)
  kLatClockRounds = 2,  // rounds whose new steps might pass a time point: the clock ran first
  kLatReactions = 3,    // reactions of every run
  kLatHops = 4,         // hops of every run
  kLatCapRaises = 5,    // raises of a group's occupancy cap
  kLatErrors = 6,       // groups that stopped with an error
  kLatFlagged = 7       // steps admitted as possible cap raises (nothing after them until they ran)
};

// Per-group stop status (LatticeLaunch::group_status).
enum LatStatus {
  kLatOk = 0,
  kLatTimeout = 1,   // the step budget ran out
  kLatRange = 2,     // the cap's K left the stream's 32 planes of n
  kLatCapacity = 3,  // the cap outgrew the planes of this launch
  kLatBadInit = 4    // an initial site count above the launch's capacity
};

// Constants of one occupancy cap m.
struct LatCap {
  double lambda;          // M 2^K u
  float inv_lambda_f;     // (float)(1 / lambda)
  int K;                  // bit length of c(m) - 1; above 32: outside the stream
  unsigned int hop_slots; // 4 rho_h 2^bh
  unsigned int m;         // the cap
  int bh;                 // bit length of m - 1: planes of the molecule index
};

struct LatticeLaunch {
  int lx, ly, lx_log, M;          // lattice; site index x + lx y
  int rec;                        // words of a site record (3 P, padded to a multiple of 4)
  int block;                      // pending steps at most (step threads; the block has one more warp)
  long long n_runs, n_groups;     // runs of the context, groups of 32
  long long group_base;           // stream index of the context's group 0
  unsigned long long seed;
  unsigned int rho_r, rho_h;
  int thin;                       // some k_r < k_max
  unsigned int always;            // bit r: k_r == k_max
  unsigned long long thin_T[3];   // floor(k_r / k_max 2^q)
  int q;
  int precision;                  // kP64LogSum (fp64), kP32Kahan, kP32D64Acc, kP32Plain
  double t_end;
  const double* snap;             // [n_snap]
  int n_snap;
  float t_end_f;                  // the largest float <= t_end: for an fp32 clock value f,
  float snap_f[kLatMaxSnap];      // f > t_end_f <=> (double)f > t_end; likewise each snapshot time
  long long step_budget;          // 0 = none
  LatCap cap[kLatMaxLevels];      // the caps in increasing order, from 1
  int n_levels;
  const int* init;                // [n_runs][M][3] or [M][3]
  int init_per_run;
  uint32_t* planes;               // [n_groups][M][rec] words of the group's count planes
  // outputs
  int* final_counts;              // [n_runs][M][3]
  double* t_homochiral;           // [n_runs]
  signed char* outcome;           // [n_runs]
  long long* events;              // [n_runs][2]: reactions, hops
  long long* group_info;          // [n_groups][3]: steps, final cap m, LatStatus
  long long* snap_totals;         // [n_snap][n_runs][3]
  int* snap_domains;              // [n_snap][n_runs][2]
  unsigned long long* counters;   // [kLatCounters]
};

// Launcher of the instantiation with P count planes (4, 8, 12 or 16); -1 if none.
int lattice_launch(int P, const LatticeLaunch& p, int grid, int block, int smem, void* stream);
// Draw planes the instantiation with P count planes handles (K above it is refused at create).
int lattice_draw_planes(int P);
// Dynamic shared memory of a block with T step threads for a lattice of M sites.
int lattice_smem_bytes(int M, int T);
int lattice_max_active_blocks(int P, int block, int smem, int* blocks);

}  // namespace bitssa
