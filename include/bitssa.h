/*
 * bitssa.h -- C ABI of libbitssa, a GB300 (sm_103a) implementation of the
 * bit-sliced exact stochastic simulation algorithm of Castellana & Lacoste,
 * "Parallelization of Gillespie algorithm based on binary words"
 * (arXiv 2412.16613).
 *
 * The method (Sec. 4): M independent runs of a conserved mass-action network
 * are packed one per bit of a machine word, species counts live as bit-planes
 * (Eqs. eq3, eq1, eq2, eq4, eq6), and one Gillespie step for all M runs is
 * done with word-wide logic: a uniform integer n in [0, Lambda) per run, the
 * comparator / changer words that pick the reaction by walking the integer
 * CDF (steps a-d, Eq. equation-changer), masked count updates (Eq.
 * equation-v) and incremental propensity updates (Eqs. equation-a-1..3,
 * App. B).  Ghost reactions (Eqs. 4-6) make the total rate the constant
 * Lambda = k_max * N (N - 1) / 2 (Eq. equation-z), so the waiting time
 * tau ~ Exp(Lambda) (Eq. equation-tau) does not depend on the state.  Options
 * raise the bound to k_max 2^K or let it follow each group's state
 * (ssa_options.pad_pow2), and networks other than
 * Frank's use k_max (m_pair C(N, 2) + u_max N) (see ssa_create).
 *
 * Here a word is 32 bits and holds one *group* of 32 runs; run j is lane
 * j % 32 of group j / 32.  Every group draws its random bits from a Philox4x32-10
 * counter stream keyed by (seed, group, step), so results do not depend on the
 * launch shape: run j's trajectory is a fixed function of (network, N0, seed, j).
 * One waiting time is drawn per group and step: the 32 runs of a group share
 * their event times (each run is still an exact sample path; runs of
 * different groups are independent).
 *
 * Conventions for every entry point:
 *   - return value: an ssa_status (0 = SSA_OK, negative = error); no entry point
 *     aborts, throws or exits.  ssa_last_error() gives a message.
 *   - inputs are copied at the call; the caller keeps ownership of its arrays.
 *   - device buffers are owned by the context.  They come from the allocator
 *     set by ssa_set_allocator() (default cudaMalloc / cudaFree) and are used on
 *     the stream given in ssa_options.cuda_stream.
 *   - arrays are C order (row-major), integers little-endian, no padding.
 */
#ifndef BITSSA_H
#define BITSSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ssa_ctx ssa_ctx;

typedef enum {
  SSA_OK = 0,
  SSA_EINVAL = -1,        /* an argument is out of range or inconsistent */
  SSA_EUNSUPPORTED = -2,  /* valid input this library does not run (see ssa_create) */
  SSA_ENOMEM = -3,        /* the allocator returned NULL */
  SSA_ECUDA = -4,         /* a CUDA runtime call failed (no device, launch error, ...) */
  SSA_ETIMEOUT = -5,      /* a group hit ssa_options.step_budget */
  SSA_EOVERFLOW = -6,     /* 64 redraws of n in a row, or an internal range check failed */
  SSA_ESTATE = -7         /* call out of order (e.g. ssa_fetch before ssa_run) */
} ssa_status;

/* Precision of the waiting-time clock (the integer dynamics are exact in every mode). */
enum {
  SSA_P64 = 0,        /* fp64: u = (x + 1) 2^-53 from 53 random bits; the clock keeps
                         exp(-Lambda t) = prod u as a 64-bit integer mantissa and an
                         integer exponent, so no logarithm is taken per step */
  SSA_P32_KAHAN = 1,  /* fp32: u from the top 24 of those bits, tau = -logf(u) / Lambda,
                         Kahan-compensated fp32 time sum */
  SSA_P32_D64ACC = 2, /* fp32 tau as above, fp64 time accumulator */
  SSA_P64_LOGSUM = 3, /* fp64: tau = -log(u) / Lambda and t += tau every step, the
                         literal form of Eq. equation-tau and Eq. eq-update-time */
  SSA_P32_PLAIN = 4   /* fp32 tau, plain fp32 time sum without compensation (a control
                         for the precision comparison) */
};

/* Simulation engine. */
enum {
  SSA_ENGINE_BITSLICED = 0,      /* the method of the paper: 32 runs per word.  Frank's model
                                    (below) runs on kernels that keep the cumulative
                                    propensities and update them with App. A's increments; any
                                    other network on the general kernel */
  SSA_ENGINE_THREAD_PER_RUN = 1, /* comparison baseline: one GPU thread per run, direct
                                    method with integer propensities (Sec. 3, steps 1-7
                                    without ghosts) and its own per-run Philox stream;
                                    Frank's model only */
  SSA_ENGINE_GENERAL = 2         /* the method on the general kernel for every network, Frank's
                                    included: each step recomputes every propensity from the
                                    count planes with bit-sliced products (Sec. 4.1); same
                                    streams and runs as SSA_ENGINE_BITSLICED */
};

/* How the bit-sliced engine maps a group of 32 runs onto the GPU. */
enum {
  SSA_LAYOUT_AUTO = 0,   /* chosen by the library */
  SSA_LAYOUT_THREAD = 1, /* one thread keeps a group's whole state (S_1..S_3 and every
                            linear form) and runs its steps alone */
  SSA_LAYOUT_WARPS = 2   /* three warps of a 96-thread block serve 32 groups: warp r keeps
                            S_{r+1} and the forms of its increments, the comparisons
                            [n < S_r] and the updates of the three S_r run side by side
                            (same streams and results as SSA_LAYOUT_THREAD) */
};

typedef struct {
  int32_t precision;         /* SSA_P64 (default) | SSA_P32_KAHAN | SSA_P32_D64ACC | SSA_P64_LOGSUM |
                                SSA_P32_PLAIN */
  int32_t engine;            /* SSA_ENGINE_BITSLICED (default) | SSA_ENGINE_THREAD_PER_RUN |
                                SSA_ENGINE_GENERAL */
  int32_t block_size;        /* threads per block, 0 = default (SSA_LAYOUT_WARPS always uses 96) */
  int32_t blocks_per_sm;     /* resident blocks per SM to launch, 0 = occupancy limit */
  int32_t thin_bits;         /* q in [1, 64], bits of the thinning threshold (default 32) */
  int32_t keep_snap_counts;  /* 1: keep per-run counts at each snapshot (SSA_FIELD_SNAP_COUNTS) */
  int64_t step_budget;       /* group steps before SSA_ETIMEOUT, 0 = unlimited */
  int64_t first_run;         /* global index of this context's run 0 inside its ensembles
                                (a multiple of 32); lets several contexts shard one
                                ensemble with results identical to one context */
  void* cuda_stream;         /* cudaStream_t to use; NULL = the legacy default stream */
  int32_t device;            /* CUDA device ordinal, -1 = the current device */
  int32_t layout;            /* SSA_LAYOUT_AUTO (default) | SSA_LAYOUT_THREAD | SSA_LAYOUT_WARPS */
  int32_t shared_n;          /* 0 (default): every run draws its own n.  1: the paper's shared draw
                                (Sec. 4, step a): all 32 runs of a group use the n of the group's
                                run 0, drawn and redrawn whether or not that run is still live; with
                                identical initial states the runs of a group are then identical,
                                so it is meant for per-run initial states (n0_per_run = 1).
                                Bit-sliced engines; Frank's model runs it on the three-warp layout
                                (SSA_LAYOUT_AUTO takes it; SSA_LAYOUT_THREAD gives
                                SSA_EUNSUPPORTED), a general network on its one kernel. */
  int32_t pad_pow2;          /* 0 (default): n is uniform on [0, lambda_int), lambda_int = N (N - 1) / 2
                                (Eq. equation-z; Sec. 3 step 5), and a draw at or above it is redrawn.
                                1: the total rate is padded with further null events up to 2^K, K the
                                bit length of lambda_int, so that every K-bit draw is accepted and
                                Lambda = k_max 2^K.  Uniformisation at any bound at or above the largest
                                total propensity samples the same process: the runs are exact either
                                way, but not draw for draw the same.  Costs 2^K / lambda_int - 1 more
                                (null) steps, saves every redraw.  Bit-sliced engines only.
                                2: the bound follows the group's state: at each step it is 2^p, p the
                                bit length of the largest S_R (sum of the integer propensities) over
                                the group's live runs, n is the low p planes of the step's draw, and
                                the step's rate is k_max 2^p.  The state is constant between steps,
                                so this is uniformisation at a rate that changes with it: each run
                                still jumps by reaction r at rate k_r h_r and is an exact sample path.
                                Fewer null steps once a group's runs near absorption: at N = 10 000
                                a group takes about 40% of the padded bound's steps.  A run's draws
                                then depend on the other runs its group holds in this context, so
                                contexts split by first_run reproduce a single one when every part
                                but the last holds whole groups.  Frank's model
                                on one thread per group only
                                (SSA_LAYOUT_AUTO takes it; SSA_LAYOUT_WARPS, shared_n or a general
                                network give SSA_EUNSUPPORTED). */
  int32_t recompute;         /* general kernel (networks other than Frank's, SSA_ENGINE_GENERAL):
                                2 keeps every propensity h_r and adds its change after each event,
                                linear in the counts before it (App. A generalised to any
                                mass-action network); 1 recomputes every h_r by bit-sliced products
                                at every step (Sec. 4.1); 0 (default) incremental unless ssa_tune
                                found products faster on the caller's workload.  Incremental mode
                                keeps a group's count planes and every h_r in the thread's
                                registers when the network has at most 4 species and 4 reactions,
                                K is at most 22 and the counts fit the planes the products read
                                (every network with a reaction of order 2), else in shared memory;
                                3 is incremental mode with the planes in shared memory always.
                                Same runs in every mode. */
  int32_t clock;             /* SSA_CLOCK_GROUP (default): the 32 runs of a group share one clock (one
                                waiting time per group and step, the paper's one tau for all copies,
                                end of Sec. 4, Eq. equation-tau): each run is an exact sample path, but
                                the runs of a group are not independent of each other.
                                SSA_CLOCK_LANE: every run has its own clock: run j's waiting time at
                                step s comes from words 0 and 1 of its own Philox4x32-10 stream (key
                                the seed, counter (j lo 32, s lo 32, s hi 16 | (j >> 32) << 16 |
                                1 << 24, 0)), with u taken from them as for the group clock; it keeps
                                its own snapshots and stops alone at t_end, and the runs of a group are
                                independent.  The integer steps are those of the group clock.  About
                                four times the work per step (a Philox call and a clock per run).
                                Frank's model, single ensembles, one thread per group in blocks of at
                                most 128 threads (544 bytes of shared memory per thread), the paper's or
                                the padded bound (SSA_LAYOUT_AUTO takes it; otherwise
                                SSA_EUNSUPPORTED) */
  int32_t word_width;        /* lanes per word: 0 (default) or 32.  64 (two groups per thread) gives
                                SSA_EUNSUPPORTED: a thread's registers hold one group's state */
  int32_t tail_groups;       /* one-thread layout of Frank's model: once every group has started, a warp
                                with at most this many groups still running finishes them with one run
                                per thread and plain integer arithmetic on the same words (same runs,
                                bit for bit).  0 (default): the library's choice (2, or what ssa_tune
                                found); -1: never; 1..4.  Groups with thinned reactions (some
                                k_r < k_max) always stay bit-sliced */
  int32_t reserved[3];
} ssa_options;

/* Clock of the runs of a group (ssa_options.clock). */
enum {
  SSA_CLOCK_GROUP = 0,
  SSA_CLOCK_LANE = 1
};

/* Fields for ssa_fetch.  n_runs = the context's total number of runs (for a batch,
 * ensembles are concatenated in order); S = n_species, in the caller's species order. */
enum {
  SSA_FIELD_FINAL_COUNTS = 0,   /* int32[n_runs][S]: counts when the run stopped (absorbed or
                                   at t_end) */
  SSA_FIELD_ABSORB_TIME = 1,    /* double[n_runs]: time of the event after which no reaction
                                   with k_r > 0 can fire; +inf if that never happened by t_end */
  SSA_FIELD_ABSORB_OUTCOME = 2, /* int8[n_runs]: -1 not absorbed, else the index of the one
                                   species left (-2: absorbed with several species left) */
  SSA_FIELD_EE_HIST = 3,        /* uint64[n_ens][n_snap][65]: enantiomeric-excess histogram of
                                   (L, D) at each snapshot, L the species X of reaction 0
                                   (A + X -> 2X) and D the species Y of reaction 1 (A + Y -> 2Y):
                                   bin min(63, floor(64 L / (L + D))), bin 64 = L + D == 0.
                                   For a network that is not Frank's, L and D are species 0
                                   and 1 (D = 0 with a single species) */
  SSA_FIELD_SNAP_COUNTS = 4,    /* int32[n_snap][n_runs][S] (needs keep_snap_counts = 1) */
  SSA_FIELD_COUNTERS = 5,       /* uint64[10]: group steps, lane steps of live runs, real
                                   reactions, null lane steps, redraw rounds, absorbed runs,
                                   groups finished, error flags, steps of the longest group,
                                   the layouts that ran (bit 0 SSA_LAYOUT_THREAD, bit 1
                                   SSA_LAYOUT_WARPS: 1, 2, or 3 for a batch that used both;
                                   0 no bit-sliced launch; on the general kernel also bit 2
                                   with propensities incremented, bit 3 recomputed by products,
                                   bit 5 the planes kept in registers (ssa_options.recompute);
                                   bit 4: some groups were finished one run per thread, see
                                   ssa_options.tail_groups) */
  SSA_FIELD_ENS_ABSORBED = 6    /* uint64[n_ens][4]: runs absorbed with outcome species 0, 1, 2,
                                   and [3] the others: not absorbed, absorbed with several
                                   species left, or with one species of index 3 or above */
};
#define SSA_N_COUNTERS 10

void ssa_default_options(ssa_options* opt);

/*
 * Create a context for n_runs runs of one network.
 *   reactants, products: int32[n_reactions][n_species] multiplicities; every reaction
 *     has order 1 or 2 and conserves the total count (Sec. 2: the model conserves
 *     N_tot = N_L + N_R + N_A, which the method relies on, Sec. 4).
 *   rates: double[n_reactions], k_r >= 0 with max > 0.  Non-unit ratios k_r / k_max
 *     are applied by thinning: the drawn reaction is kept iff a q-bit uniform U is
 *     below T_r = floor(k_r / k_max 2^q) (the paper leaves general rates to future
 *     work, Sec. 6; this is an exact-in-the-limit integer form of it).
 *   N0: int64[n_species] shared initial counts (n0_per_run = 0) or
 *     int64[n_runs][n_species] (n0_per_run = 1); every run must have the same total
 *     (Sec. 4: the copies share N_tot).
 *   seed: the Philox key.
 * Frank's model (Eqs. 1-3) up to a relabelling of species -- three species X, Y, A
 * and, in this order, A + X -> 2X, A + Y -> 2Y, X + Y -> 2A -- runs on its own
 * kernels.  Any other network of at most 8 species and 8 reactions runs on the
 * general kernel: the uniformisation bound is lambda_int = m_pair C(N_tot, 2) +
 * u_max N_tot, with m_pair the most reactions on one unordered reactant pair and
 * u_max the most first-order reactions of one species, and reaction r takes the
 * integers [S_{r-1}, S_r) of the draw in the order given.  SSA_EUNSUPPORTED beyond
 * 8 species or reactions, for N_tot > 65536, and when lambda_int >= 2^31;
 * SSA_EUNSUPPORTED also for a general network with the thread-per-run engine or
 * SSA_LAYOUT_WARPS.  n_runs may be 0.  On success *out owns device memory until
 * ssa_destroy.
 */
int ssa_create(const int32_t* reactants, const int32_t* products, int32_t n_species,
               int32_t n_reactions, const double* rates, const int64_t* N0, int32_t n0_per_run,
               int64_t n_runs, uint64_t seed, const ssa_options* opt, ssa_ctx** out);

/*
 * Create a context for n_ens ensembles of the same network run in one launch
 * sequence.  Ensemble e has its own initial counts N0_ens[e] (int64[n_ens][S]),
 * rates rates_ens[e] (double[n_ens][R]), run count runs_ens[e] and seed
 * seed_ens[e]; its runs are numbered from 0 inside the ensemble (stream
 * groups restart at 0), and appear in the output fields after the runs of
 * ensembles 0..e-1.  Same restrictions as ssa_create.
 */
int ssa_create_batch(const int32_t* reactants, const int32_t* products, int32_t n_species,
                     int32_t n_reactions, int32_t n_ens, const int64_t* N0_ens,
                     const double* rates_ens, const int64_t* runs_ens, const uint64_t* seed_ens,
                     const ssa_options* opt, ssa_ctx** out);

/*
 * Simulate every run from its initial state (each call starts again from t = 0,
 * so repeated calls give identical results) until it is absorbed or its next
 * event would come after t_end.  snapshot_times: double[n_snap], ascending, each
 * in [0, t_end]; the snapshot at time t holds the state after every event with
 * time <= t.  n_snap in [0, 64].  Blocks until the work is done on the stream.
 */
int ssa_run(ssa_ctx* ctx, double t_end, const double* snapshot_times, int32_t n_snap);

/*
 * Autotuner: time the context's work under each launch configuration the library has and keep
 * the fastest for later ssa_run calls whose options leave layout = SSA_LAYOUT_AUTO, block_size =
 * 0, recompute = 0 and tail_groups = 0 (fixed options win).  Frank's model: the automatic layout
 * rule, one thread per group of 32 runs with blocks of 32, 64 and 128 threads, three warps per 32
 * groups; then, when one thread per group won, the tail hand-off off or at 1, 2 or 4 groups.  A
 * general network: blocks of 32, 64 and 128 threads, each with the propensities incremented and
 * with them recomputed by products.  Results do not depend on the configuration: every one draws
 * the same streams and gives the same runs.
 *   t_end, snapshot_times, n_snap: the workload to time, as for ssa_run.
 *   probe_steps: 0 times whole runs (exact, costs ten runs); > 0 stops every group after that
 *     many steps (a cheap probe of the early, crowded part of a run).
 *   choice: int32[2] or NULL; receives the chosen SSA_LAYOUT_* (SSA_LAYOUT_AUTO = the rule)
 *     and the block size of the one-thread layout.
 * Leaves the context without a run to fetch (SSA_ESTATE until the next ssa_run).  Errors as for
 * ssa_run; SSA_EUNSUPPORTED for the thread-per-run engine.
 */
int ssa_tune(ssa_ctx* ctx, double t_end, const double* snapshot_times, int32_t n_snap, int64_t probe_steps,
             int32_t* choice);

/* Size in bytes of a field after the last ssa_run (0 for an unknown field). */
int ssa_field_bytes(const ssa_ctx* ctx, int32_t field, size_t* bytes);

/*
 * Copy a field into dst (dst_bytes >= ssa_field_bytes).  dst_on_device = 1: dst is
 * device memory on the context's device, the copy runs on the context's stream
 * and is complete on return; 0: dst is host memory.
 */
int ssa_fetch(ssa_ctx* ctx, int32_t field, void* dst, size_t dst_bytes, int32_t dst_on_device);

/* Free the context and its device memory.  NULL is allowed. */
int ssa_destroy(ssa_ctx* ctx);

/* Message of the last failed call on ctx, or of the calling thread's last failed
 * ssa_create / ssa_create_batch / ssa_set_allocator when ctx is NULL.  Owned by
 * the library; valid until the next call on the same ctx / thread. */
const char* ssa_last_error(const ssa_ctx* ctx);

/*
 * Route device allocations through caller functions (e.g. a framework's caching
 * allocator).  alloc returns device memory of at least `bytes` on `device`
 * usable on `stream`, or NULL; release frees it.  NULL, NULL restores
 * cudaMalloc / cudaFree.  Affects contexts created afterwards.
 */
typedef void* (*ssa_alloc_fn)(size_t bytes, int device, void* stream, void* user);
typedef void (*ssa_free_fn)(void* ptr, size_t bytes, int device, void* stream, void* user);
int ssa_set_allocator(ssa_alloc_fn alloc, ssa_free_fn release, void* user);

/* ------------------------------------------------------------------------------------------ */
/* Frank's model on a periodic lattice (non-well-mixed).                                        */
/*                                                                                              */
/* The paper motivates compartments and systems that are not well mixed (Sec. 1, Sec. 6) but    */
/* gives no algorithm for them; what follows is this library's exact extension of the method.  */
/* ------------------------------------------------------------------------------------------ */
/*
 * Sites (x, y) with x < lx, y < ly (both powers of two; M = lx ly <= 16384 sites; site index
 * x + lx y) each hold counts (L, D, A) and run Frank's reactions A+L->2L, A+D->2D, L+D->2A (Eqs.
 * 1-3) with propensities k_r h_r per site (h = A L, A D, L D; Omega = 1 per site); every molecule
 * hops to each of its four neighbours (x +- 1 mod lx, y), (x, y +- 1 mod ly) at rate d.  The total
 * count is conserved over the lattice.
 *
 * The 32 runs of a group share one word per count plane per site (Sec. 4's binary words, one
 * set per site) and the site of every step; each run picks its own event there.  Uniformisation
 * is exact: with u = min(k_max, d), rho_r = k_max / u and rho_h = d / u must be integers
 * (rho_r < 65536); the group keeps an occupancy cap m at or above every site count of its runs,
 * one of 1 .. 8 or (4 + j) 2^e (j = 0 .. 3: 10, 12, 14, 16, 20, ...), initially the smallest such
 * cap; with bh = bit_length(m - 1), a site has c(m) = 4 rho_h 2^bh + rho_r m (m - 1) / 2 slots,
 * K = bit_length(c(m) - 1) <= 32, and the group's steps come at rate Lambda = M 2^K u.  Step s of
 * group g uses word k = element k % 4 of Philox4x32-10(key = seed, counter = (g, s lo 32,
 * s hi 16 | 2 << 24, k / 4)):
 *   w0, w1: the waiting time tau = -ln(u) / Lambda, u = (x + 1) 2^-53 from x = w1 2^21 + (w0 >> 11),
 *     or u = ((w1 >> 8) + 1) 2^-24 in the fp32 modes;
 *   w2: the site sigma = w2 & (M - 1) of every run of the group;
 *   w3 .. w3+K-1: plane i of run l's n is bit l of w_{3+i};
 *   w35 ..: thinning, the q-bit U whose bit q-1-i is bit l of w_{35+i}.
 * Run l with counts (L, D, A) at sigma: if n < H = 4 rho_h 2^bh, a hop in direction n & 3 (x+1,
 * x-1, y+1, y-1) of molecule i = (n >> 2) & (2^bh - 1): an L if i < L, a D if i < L + D, an A if
 * i < L + D + A, else nothing; otherwise reaction r if H + rho_r S_{r-1} <= n < H + rho_r S_r
 * (S_r = h_1 + .. + h_r), kept iff U < floor(k_r / k_max 2^q) when k_r < k_max, nothing above S_3.
 * A run thus jumps by reaction r at rate k_r h_r and moves a given molecule in a given direction at
 * rate d.  If a hop leaves a site of any run above m, m moves to the next cap from the next step.
 * Runs go on to t_end; the time at which a run's lattice first holds a single species is kept.
 *
 * Up to twice block_size consecutive steps of a group are pending at once; a step waits only
 * for earlier pending steps whose site or neighbours meet its own, so every run follows the serial
 * definition above exactly; results do not depend on the block size.
 */
typedef struct ssa_lattice ssa_lattice;

/* Fields for ssa_lattice_fetch (n_runs, M and n_snap of the context and its last run). */
enum {
  SSA_LAT_FINAL_COUNTS = 0,   /* int32[n_runs][M][3]: (L, D, A) of every site at t_end */
  SSA_LAT_HOMOCHIRAL_TIME = 1,/* double[n_runs]: first event time at which the run's lattice holds
                                 one species (0 if it did at the start); +inf if never by t_end */
  SSA_LAT_OUTCOME = 2,        /* int8[n_runs]: that species (0 L, 1 D, 2 A); -1 none */
  SSA_LAT_EVENTS = 3,         /* int64[n_runs][2]: reactions and hops of the run */
  SSA_LAT_SNAP_TOTALS = 4,    /* int64[n_snap][n_runs][3]: lattice totals of (L, D, A) at each
                                 snapshot (the state after every event with time <= t_snap) */
  SSA_LAT_SNAP_DOMAINS = 5,   /* int32[n_snap][n_runs][2]: sites with L > D and sites with D > L */
  SSA_LAT_GROUPS = 6,         /* int64[n_groups][3]: steps of the group, its final cap m (the cap
                                 it needed, when it stopped for want of planes), and its stop
                                 status (0 t_end, 1 step budget, 2 K above 32 planes, 3 cap above
                                 the context's planes) */
  SSA_LAT_COUNTERS = 7        /* uint64[8]: group steps, rounds (one wave of ready steps each),
                                 rounds whose new steps might pass a snapshot or t_end (the clock
                                 ran before admission), reactions, hops, cap raises, groups
                                 stopped by an error, steps admitted as possible cap raises */
};
#define SSA_LAT_N_COUNTERS 8

/*
 * Create a lattice context.
 *   lx, ly: powers of two, lx ly <= 16384.
 *   rates: double[3] (k_1, k_2, k_3) >= 0, max > 0; hop: d > 0.  max(k) / d or d / max(k) must be
 *     an integer (within 1e-9 relative).
 *   N0: int64[M][3] counts per site shared by every run (n0_per_run = 0) or int64[n_runs][M][3]
 *     (n0_per_run = 1); each site count in [0, 32768].
 *   n_runs >= 0, seed: as in ssa_create (run j is lane j % 32 of group j / 32).
 *   opt: precision (SSA_P64 and SSA_P64_LOGSUM both give tau = -log(u) / Lambda summed in fp64;
 *     SSA_P32_KAHAN, SSA_P32_D64ACC, SSA_P32_PLAIN as for ssa_create), thin_bits, block_size (step
 *     threads, each holding two pending steps; a multiple of 32 up to 224; 0 = 224), step_budget,
 *     first_run, cuda_stream, device.  Other fields must keep their defaults (SSA_EUNSUPPORTED
 *     otherwise).
 *   cap_bits_max: the runs may reach caps up to 2^cap_bits_max; 0 = what the count planes chosen
 *     for the initial cap hold; at most 15.  The planes per count are the smallest of 4, 8, 12, 16
 *     above it (caps up to 8, 128, 2048, 32768); a run whose cap would outgrow them stops with
 *     SSA_EOVERFLOW.
 * Returns SSA_EINVAL for bad arguments, SSA_EUNSUPPORTED beyond the limits above.
 */
int ssa_lattice_create(int32_t lx, int32_t ly, const double* rates, double hop, const int64_t* N0,
                       int32_t n0_per_run, int64_t n_runs, uint64_t seed, const ssa_options* opt,
                       int32_t cap_bits_max, ssa_lattice** out);

/*
 * Run every run from its initial state to t_end (each call starts again from t = 0).
 * snapshot_times: double[n_snap] ascending in [0, t_end], n_snap in [0, 64].  Blocks until done.
 * SSA_ETIMEOUT if a group hit the step budget, SSA_EOVERFLOW if a group's K left the stream's 32
 * planes or its cap outgrew the context's planes; the fields are still written (SSA_LAT_GROUPS
 * says which group stopped and why).
 */
int ssa_lattice_run(ssa_lattice* ctx, double t_end, const double* snapshot_times, int32_t n_snap);

/* Bytes of a field after the last run (0 for an unknown field). */
int ssa_lattice_field_bytes(const ssa_lattice* ctx, int32_t field, size_t* bytes);

/* Copy a field into dst (host memory, or device memory on the context's device when
 * dst_on_device = 1; complete on return). */
int ssa_lattice_fetch(ssa_lattice* ctx, int32_t field, void* dst, size_t dst_bytes, int32_t dst_on_device);

/* Free the context and its device memory.  NULL is allowed. */
int ssa_lattice_destroy(ssa_lattice* ctx);

/* Message of the last failed call on ctx; NULL: the calling thread's last failed create. */
const char* ssa_lattice_last_error(const ssa_lattice* ctx);

/*
 * ssa_run_frank_noalloc: one run of Frank's model that allocates no device memory.
 *
 * The paper has no counterpart; this is a service of the library.  Some callers
 * cannot allocate device memory at all: a plug-in hosted by a framework that owns
 * every byte of device memory (its pool hands out buffers, and memory taken
 * behind its back can make its own allocations fail), or a latency-critical loop
 * in which cudaMalloc, which can synchronise the whole device and has no bounded
 * latency, is not allowed.  They pass in every input and output buffer, and this
 * call runs the same one-thread bit-sliced kernel as ssa_run on a single ensemble
 * without a context.  It uses the paper's bound (pad_pow2 = 0: n uniform below
 * N (N - 1) / 2, draws above it redrawn), the group clock and blocks of 64 threads;
 * ssa_run with those options gives the same runs.
 *
 * The kernel's own scratch (work-queue counter, run counters, error word and the
 * crossing thresholds of up to 64 snapshot times plus t_end, about 2.2 KB) is a
 * fixed device array inside the library: every GPU that loads the library holds a
 * copy until the process exits.  The first call on a device looks up that copy's
 * address, with the device current.  Every call clears what must start at zero and
 * overwrites the thresholds, so calls share the array: two calls that overlap on
 * one GPU (other streams, other host threads) race, and the caller must serialise
 * them.
 *
 *   N0: int64[3] host, the shared initial counts of L, D and A for the reactions
 *       A+L->2L, A+D->2D, L+D->2A; total in [1, 65536].
 *   rates: double[3] host, k >= 0 with max > 0 (thinning as in ssa_create, q = thin_bits).
 *   n_runs >= 0, seed: as in ssa_create (run j is lane j % 32 of group j / 32).
 *   t_end, snapshot_times (double[n_snap] host, ascending, in [0, t_end]), n_snap in
 *       [0, 64]: as in ssa_run.  n_snap above 64, the capacity of the fixed scratch,
 *       is rejected with SSA_EINVAL before any GPU work.
 *   precision: SSA_P64 ... SSA_P32_PLAIN.
 *   outputs, device memory on the current device, written on cuda_stream:
 *       final_counts int32[n_runs][3], t_abs double[n_runs], outcome int8[n_runs]
 *       (as SSA_FIELD_FINAL_COUNTS / ABSORB_TIME / ABSORB_OUTCOME, species order L, D, A;
 *       may be NULL when n_runs == 0), ee_hist uint64[n_snap][65] (cleared by the call;
 *       may be NULL when n_snap == 0).
 *   counters_out: uint64[10] host (as SSA_FIELD_COUNTERS) or NULL.
 *   cuda_stream: cudaStream_t, NULL = the legacy default stream.
 * The thresholds are copied from host memory and the counters read back into it, and
 * the call waits for the stream before it returns.  Returns an ssa_status; the message
 * of a failure is given by ssa_last_error(NULL) on the calling thread.  Calls no
 * cudaMalloc, cudaFree or other allocating routine.
 */
int ssa_run_frank_noalloc(const int64_t* N0, const double* rates, int64_t n_runs, uint64_t seed,
                          int32_t thin_bits, double t_end, const double* snapshot_times, int32_t n_snap,
                          int32_t precision, int32_t* final_counts, double* t_abs, int8_t* outcome,
                          uint64_t* ee_hist, uint64_t* counters_out, void* cuda_stream);

/* Library version as major * 10000 + minor * 100 + patch. */
int ssa_version(void);

#ifdef __cplusplus
}
#endif
#endif
