// internal.h -- structures shared by the host runtime and the sm_103a kernels
// of libbitssa.  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <string>

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

constexpr int kMaxSnap = 64;
constexpr int kTailSlots = 4;          // the one-thread kernel's tail hand-off: groups a warp hands over at most
constexpr int kTailDepth = 4;          // steps whose random words it draws together
constexpr int kDefaultTailGroups = 2;  // FrankLaunch::tail_groups unless an option or the tuner sets it
constexpr int kHistBins = 65;  // 64 enantiomeric-excess bins + one for L + D == 0
constexpr int kCounters = 10;
constexpr int kMaxK = 31;      // random / propensity planes: N_tot (N_tot - 1) / 2 < 2^31
constexpr int kTrioBlock = 96; // threads of a block of the three-warp layout (32 groups)
constexpr int kMaxSpecies = 8;   // general networks: species
constexpr int kMaxReactions = 8; // general networks: reactions
constexpr int kMaxCountPlanes = 17;  // counts up to N_tot = 65536
constexpr int kGeneralScratch = 5 * kMaxSpecies;  // general kernel: scratch words per thread
// general networks whose count planes and propensities a thread keeps in registers
constexpr int kRegSpecies = 4;    // species
constexpr int kRegReactions = 4;  // reactions
constexpr int kRegMaxK = 22;      // propensity planes (larger K stays in shared memory)

// Clock precision modes (same values as SSA_P64 ... in bitssa.h).
enum Precision { kP64 = 0, kP32Kahan = 1, kP32D64Acc = 2, kP64LogSum = 3, kP32Plain = 4 };

// Indices into the device counter array (uint64).
enum Counter {
  kGroupSteps = 0,
  kLaneSteps = 1,
  kReactions = 2,
  kNullLaneSteps = 3,
  kRedrawRounds = 4,
  kAbsorbed = 5,
  kGroupsDone = 6,
  kErrorFlags = 7,
  kMaxGroupSteps = 8, // the longest group, in steps
  kLayoutUsed = 9     // set by the host: bit 0 one thread per group, bit 1 three warps per 32 groups,
                      // bit 2 the general kernel incrementing propensities, bit 3 it recomputing them,
                      // bit 4 (by the device) the one-thread kernel's tail hand-off ran
};
constexpr int kLayoutGeneralIncremental = 4;
constexpr int kLayoutGeneralProducts = 8;
constexpr int kLayoutTail = 16;  // set by the device: some groups were finished one run per thread
constexpr int kLayoutGeneralRegisters = 32;  // the general kernel kept its planes in registers

// Error flags (OR-ed into the status word).
enum ErrorFlag : uint32_t {
  kErrTimeout = 1u,      // step budget reached
  kErrRedraw = 2u,       // 64 redraws of n in a row
  kErrRange = 4u,        // a count or propensity left its range (internal check)
  kErrQueue = 8u         // work item without a valid ensemble
};

// Crossing threshold for one time point t of one ensemble, in the forms each
// clock compares against.
struct Threshold {
  double t;              // the time itself (fp64 sum clocks)
  unsigned long long M;  // exp(-Lambda t) = M 2^(E - 63), M in [2^63, 2^64) (product clock)
  long long E;
  float t_f;             // the largest float <= t (fp32 Kahan clock: f > t_f <=> (double)f > t)
  int pad;
};

// Per-ensemble constants.  For Frank's model species are in the kernel's canonical
// order (L, D, A): reactions A+L->2L, A+D->2D, L+D->2A; for a general network they
// are the caller's species and reactions.
struct Ensemble {
  unsigned long long seed;
  long long n_runs;        // runs of this ensemble in this context
  long long run_offset;    // row of the ensemble's first run in the output fields
  long long group_base;    // stream group index of the context's first group (first_run / 32)
  long long thin_T[kMaxReactions];  // thinning thresholds T_r (bit patterns of uint64)
  double lambda;           // k_max * lambda_int
  float inv_lambda_f;      // (float)(1 / lambda)
  unsigned int lambda_int; // N (N - 1) / 2 for Frank; m_pair C(N, 2) + u_max N in general
  int n_tot;
  int K;                   // bit length of lambda_int
  int init[kMaxSpecies];   // shared initial counts (canonical order for Frank)
  unsigned int thin_always;  // bit r: k_r == k_max
  unsigned int active;       // bit r: k_r > 0
  int thin;                  // any reaction with k_r < k_max
  int thin_bits;             // q
  int shared_n;              // 1: every lane of a group uses lane 0's n
  int reject;                // 1: lambda_int < 2^K, draws of n at or above it are redrawn;
                             // 0: the bound is padded to 2^K and every draw is accepted
  unsigned int top_ones;     // planes of the leading run of ones of lambda_int (bit i = plane i):
                             // n >= lambda_int needs all of them set (0: no pre-check)
  unsigned int top_mask[32]; // per plane: 0 on the run, ~0 elsewhere, so that the AND over planes
                             // of (n_i | top_mask[i]) is the lanes that pass the pre-check
};


// Fills top_ones and top_mask from lambda_int and K.
inline void set_precheck(Ensemble& e) {
  e.top_ones = 0u;
  for (int i = e.K - 1; i >= 0 && ((e.lambda_int >> i) & 1u); --i) e.top_ones |= 1u << i;
  for (int i = 0; i < 32; ++i) e.top_mask[i] = ((e.top_ones >> i) & 1u) ? 0u : 0xFFFFFFFFu;
}

// Per-ensemble constants of Frank's model in the kernel's species order (L, D, A) from their
// definitions: lambda_int = N (N - 1) / 2 (2^K when pad_pow2), K = the bit length of
// N (N - 1) / 2, the pre-check masks, the thinning thresholds T_r = floor(k_r / k_max 2^q).
Ensemble make_ensemble(long long n_tot, const int init[3], const double k[3], int q, unsigned long long seed,
                       long long n_runs, long long run_offset, long long group_base, int pad_pow2);
// The crossing threshold of time t for total rate lambda, in every form a clock compares.
Threshold make_threshold(double t, double lambda);

// A conserved mass-action network of order 1 or 2 (Sec. 2), in the caller's species and
// reaction order, for the general bit-sliced kernel.
struct Network {
  int S, R;
  int B;                             // count planes: bit length of N_tot
  int order[kMaxReactions];          // 1 or 2
  int a[kMaxReactions];              // first reactant
  int b[kMaxReactions];              // second reactant (a for 2X); -1 for first order
  int nu[kMaxReactions][kMaxSpecies];  // products - reactants, in [-2, 2]
  unsigned int nu_bits[kMaxSpecies][3];  // bit r of [s][p]: bit p of nu[r][s] in 3-bit two's complement
  unsigned int changes;              // bit s: some reaction changes species s
  int hist_x, hist_y;                // species binned by the ee histogram (x: "L", y: "D")
  int incremental;                   // 1: keep h_r and add its change every step; 0: products every step
  int regs;                          // 1: count planes and h_r in registers (general_reg_kernel)
};

// Per-ensemble constants of a general network from their definitions: lambda_int =
// m_pair C(N, 2) + u_max N (2^K when pad_pow2), K = the bit length of the unpadded bound,
// the thinning thresholds T_r = floor(k_r / k_max 2^q).
Ensemble make_general_ensemble(const Network& net, long long n_tot, const int* init, const double* k, int q,
                               unsigned long long seed, long long n_runs, long long run_offset,
                               long long group_base, int pad_pow2, unsigned long long* lambda_unpadded);

// One launch of the bit-sliced kernel for one K.
struct FrankLaunch {
  Ensemble ens;                   // used when ens_table == nullptr (one ensemble)
  const Ensemble* ens_table;      // [n_ens] (batch)
  const Threshold* thr;           // [n_ens][n_snap + 1]; entry n_snap is t_end
  const int* item_ens;            // [n_items] ensemble of each work item, or nullptr
  const int* item_group;          // [n_items] group inside its ensemble, or nullptr
  long long item_begin, item_end; // work items of this launch
  const int* init_counts;         // [n_runs_total][3] canonical order, or nullptr (shared init)
  int n_snap;
  int precision;
  long long step_budget;
  int perm[3];                    // canonical species c is written to column perm[c]
  int n_species;                  // columns of the count outputs
  // outputs
  int* final_counts;              // [n_runs_total][n_species]
  double* t_abs;                  // [n_runs_total]
  signed char* outcome;           // [n_runs_total]
  unsigned long long* hist;       // [n_ens][n_snap][65]
  unsigned long long* ens_absorbed; // [n_ens][4]
  int* snap_counts;               // [n_snap][n_runs_total][n_species] or nullptr
  long long n_runs_total;
  // scratch
  unsigned long long* counters;   // [kCounters]
  unsigned int* status;           // error flags
  unsigned long long* queue;      // work-item counter of this launch
  int adapt;                      // one-thread Frank kernel: 1 runs the instantiation with the
                                  // state-following bound (each step's bound 2^p, p the bit length
                                  // of the largest S_R over the group's live lanes; 2^K its ceiling)
  int lane_clock;                 // one-thread Frank kernel, single ensemble: 1 gives every run its own
                                  // clock (its records in dynamic shared memory from word lane_offset)
  int lane_offset;
  int tail_groups;                // one-thread Frank kernel: once the work queue is drained, a warp
                                  // with at most this many running groups (1..kTailSlots) finishes them with
                                  // one run per thread; 0 never
  int stage_offset;               // one-thread Frank kernel with a snapshot dump: the word of dynamic
                                  // shared memory where the per-thread staging rows start; -1: none
  Network net;                    // general kernel only
};

// Words of shared memory per thread for staging a group's snapshot rows (32 runs x 3 counts,
// padded so that rows start 16-byte aligned and neighbouring threads fall in different banks).
constexpr int kStageStride = 100;

// One launch of the one-thread-per-run baseline.
struct ThreadLaunch {
  Ensemble ens;
  const Threshold* thr;           // [n_snap + 1]
  const int* init_counts;         // [n_runs][3] or nullptr
  int n_snap;
  int precision;
  long long step_budget;
  double rates[3];
  int unit_rates;                 // all k_r equal: exact integer selection
  int perm[3];
  int n_species;
  int* final_counts;
  double* t_abs;
  signed char* outcome;
  unsigned long long* hist;
  unsigned long long* ens_absorbed;
  int* snap_counts;
  long long n_runs_total;
  unsigned long long* counters;
  unsigned int* status;
};

// Entry points implemented by the kernel translation units.
using FrankLauncher = int (*)(const FrankLaunch&, int grid, int block, int smem, void* stream);
FrankLauncher frank_launcher(int K);
// variant: bit 0 = batch (ensemble table), bit 1 = product clock (SSA_P64)
int frank_max_active_blocks(int K, int variant, int block, int smem, int* blocks);
int frank_registers(int K, int variant);
// The three-warp layout (block of kTrioBlock threads serving 32 groups).
using FrankTrioLauncher = int (*)(const FrankLaunch&, int grid, int smem, void* stream);
// The general-network kernel (one thread per group; counts in shared memory).
FrankLauncher general_launcher(int K);
int general_max_active_blocks(int K, int variant, int block, int smem, int* blocks);
int general_registers(int K, int variant);
// Shared memory of the general kernel per block of `block` threads, histogram excluded.
int general_smem_bytes(const Network& net, int K, int block);
FrankTrioLauncher frank_trio_launcher(int K);
int frank_trio_max_active_blocks(int K, int variant, int smem, int* blocks);
int frank_trio_registers(int K, int variant);
int thread_per_run_launch(const ThreadLaunch& p, int grid, int block, int smem, void* stream);
// Sets the calling thread's message returned by ssa_last_error(NULL).
void set_thread_error(const std::string& msg);
int thread_per_run_max_active_blocks(int block, int smem, int* blocks);

}  // namespace bitssa
