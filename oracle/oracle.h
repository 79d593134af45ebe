/*
 * oracle.h -- CPU oracle for the bit-sliced Gillespie method
 *             (Castellana & Lacoste, "Parallelization of Gillespie algorithm
 *             based on binary words", arXiv 2412.16613).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (libbitssa) never links, loads or calls it, and the two share no code.
 *
 * What it computes: one run at a time, a plain serial Gillespie simulation of
 * a conserved mass-action network with integer counts (Sec. 2-3), driven by a
 * fixed counter-based random stream so that any single run can be recomputed
 * on its own:
 *
 *   run j lives in group g = j / 32 at lane l = j % 32;
 *   word k of the (g, step s, attempt a, tag) stream is element k % 4 of
 *     Philox4x32-10(key = (seed lo, seed hi),
 *                   ctr = (g, s lo32, (s hi16) | a << 16 | tag << 24, k / 4));
 *   n   = sum_{i<K} bit_l(w_i) 2^i; while n >= Lambda_int, its bits from p up (p the
 *         highest bit where n and Lambda_int differ, 0 if equal) are replaced by the
 *         same bits of attempt a+1 (a uniform integer in [0, Lambda_int), Sec. 3 step
 *         5(i) and step a); with pad_pow2 = 1, Lambda_int = 2^K and no draw is rejected;
 *         with pad_pow2 = 2 the bound of step s is 2^p, p = the bit length of the largest
 *         S_R over the live runs of the group, and n = sum_{i<p} bit_l(w_i) 2^i;
 *   tau = -log(u) / Lambda (Lambda = k_max 2^p with pad_pow2 = 2) from the whole
 *         words w_K, w_{K+1} of attempt 0 (with lane_clock = 1, from the words v_0, v_1 of
 *         run j's own stream: element k of Philox4x32-10(key as above, ctr = (j lo 32,
 *         s lo 32, s hi 16 | (j >> 32) << 16 | 1 << 24, 0)); so every run has its own clock)
 *         (Eq. equation-tau, with the uniformisation rate of Eq. equation-z):
 *         fp64 u = (x + 1) 2^-53 with x = w_{K+1} << 21 | w_K >> 11; the fp32
 *         modes take u = ((w_{K+1} >> 8) + 1) 2^-24, the top 24 of those bits;
 *   the fired reaction is the smallest r with n < S_r = sum_{p<=r} h_p
 *         (the CDF walk of Sec. 3 step 5 / Fig. 2); none fires when n >= S_R
 *         (a ghost reaction, Eqs. 4-6);
 *   non-unit rates: reaction r is kept iff U < T_r = floor(k_r / k_max 2^q), U
 *         the q-bit number whose bit q-1-i is bit_l(w_{K+2+i}) of attempt 0.
 *
 * Everything here is fp64 (or fp32 where a precision mode asks for it),
 * compiled with -ffp-contract=off so that x86-64 and aarch64 hosts agree.
 */
#ifndef BITSSA_ORACLE_H
#define BITSSA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_SPECIES 8
#define ORC_MAX_REACTIONS 8

/* precision modes of the waiting-time clock */
#define ORC_P64 0        /* u from 53 bits, tau = -log(u)/Lambda, double sum */
#define ORC_P32_KAHAN 1  /* u from 24 bits, tau = -logf(u)*(float)(1/Lambda), Kahan float sum */
#define ORC_P32_D64ACC 2 /* float tau as above, double accumulator */
#define ORC_P32_PLAIN 3  /* float tau as above, plain float sum (no compensation) */

/* status codes */
#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ETIMEOUT -5
#define ORC_ERANGE -6    /* 64 redraw attempts exhausted, or a count left its range */

typedef struct {
  int32_t n_species;        /* S, 1..ORC_MAX_SPECIES */
  int32_t n_reactions;      /* R, 1..ORC_MAX_REACTIONS */
  const int32_t* reactants; /* [R][S] reactant multiplicities, order <= 2 */
  const int32_t* products;  /* [R][S] product multiplicities */
  const double* rates;      /* [R] k_r >= 0, max > 0 */
  int64_t n_tot;            /* conserved total count, >= 1 */
  uint64_t seed;            /* Philox key */
  int32_t precision;        /* ORC_P64 | ORC_P32_KAHAN | ORC_P32_D64ACC | ORC_P32_PLAIN */
  int32_t thin_bits;        /* q, 1..64 */
  double t_end;             /* stop before the first event later than t_end */
  const double* snap_times; /* [n_snap] ascending, <= t_end (may be NULL if n_snap == 0) */
  int32_t n_snap;
  int64_t step_budget;      /* max steps per run, 0 = unlimited */
  int32_t shared_n;         /* 1: every run of a group of 32 uses the n of the group's lane 0 (one n
                               for all copies, Sec. 4 step a), drawn whether or not lane 0 is live */
  int32_t pad_pow2;         /* 1: the uniformisation bound is raised from lambda_int to 2^K with
                               further null events, so that every K-bit draw of n is accepted;
                               2: the bound follows the group's state (2^p at each step, p the
                               bit length of the largest S_R over the group's live runs), so the
                               32 runs of a group are stepped together */
  int64_t ensemble_runs;    /* pad_pow2 = 2: runs in the ensemble, which fixes how many lanes the
                               last group holds; 0 = every group holds 32 runs */
  int32_t lane_clock;       /* 0: one clock per group of 32 runs (the waiting-time words K, K+1 of
                               the group's stream); 1: every run has its own clock, the waiting time
                               of run j at step s from words 0 and 1 of its own stream (below).
                               Not with pad_pow2 = 2 */
} orc_problem;

/* Derived constants of a problem, computed from their definitions. */
typedef struct {
  uint64_t lambda_int;      /* integer uniformisation bound: sum_r h_r <= lambda_int (2^K when
                               pad_pow2 is set) */
  int32_t K;                /* random planes for n: bit length of the unpadded bound */
  double k_max;
  double lambda;            /* k_max * lambda_int */
  int32_t thin_always[ORC_MAX_REACTIONS]; /* 1: T_r = 2^q, always kept */
  uint64_t thin_T[ORC_MAX_REACTIONS];     /* T_r when not always kept */
  int32_t any_thinning;
} orc_derived;

/* Per-run result. */
typedef struct {
  int64_t final_counts[ORC_MAX_SPECIES];
  double t_abs;        /* time of the event that made every real propensity 0; +inf if none */
  double t_last;       /* time of the last committed step */
  int32_t outcome;     /* -1 not absorbed; >= 0 the one species left; -2 absorbed with several */
  int32_t status;
  int64_t steps;       /* committed steps, null ones included */
  int64_t reactions;   /* real reactions */
  int64_t redraws;     /* extra attempts spent on n >= lambda_int */
  double margin;       /* smallest relative gap between a snapshot / t_end and the
                          committed event times on either side of it */
} orc_result;

int orc_derive(const orc_problem* p, orc_derived* d);

/* Philox4x32-10 block function (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Word k of a stream, as defined above. */
uint32_t orc_stream_word(uint64_t seed, uint64_t group, uint64_t step, uint32_t attempt,
                         uint32_t tag, uint32_t k);

/* h_r(state) for every r, and the reaction the CDF walk picks for integer n
 * (-1 = none).  Exposed for the exhaustive tests of the selection rule. */
int orc_propensities(const orc_problem* p, const int64_t* state, int64_t* h);
int32_t orc_select(const orc_problem* p, const int64_t* state, uint64_t n);

/* One run.  snap_counts: [n_snap][S] or NULL. */
int orc_run(const orc_problem* p, const orc_derived* d, int64_t run_index,
            const int64_t* init, orc_result* out, int64_t* snap_counts);

/* The lanes of one group stepped together (pad_pow2 = 2).  init is [S] (init_per_lane = 0)
 * or [lanes][S]; out is [lanes]; snap_counts is [lanes][n_snap][S] or NULL. */
int orc_run_group(const orc_problem* p, const orc_derived* d, uint64_t group, int32_t lanes,
                  const int64_t* init, int32_t init_per_lane, orc_result* out, int64_t* snap_counts);

/* Many runs on n_threads host threads.  Run i is global run run_ids[i] (or
 * first_run + i when run_ids is NULL).  init is [S] (init_per_run = 0) or
 * [n_runs][S]; with pad_pow2 = 2 a per-run init is indexed by the run's global index
 * instead, and holds a row for every run of the groups asked for.  Outputs are per run,
 * indexed by i; any may be NULL except out.  snap_counts is [n_snap][n_runs][S].
 * Returns the first non-OK status. */
int orc_run_many(const orc_problem* p, int64_t first_run, const int64_t* run_ids, int64_t n_runs,
                 const int64_t* init, int32_t init_per_run, orc_result* out,
                 int64_t* snap_counts, int32_t n_threads);

/* ------------------------------------------------------------------------ */
/* Frank's model on a periodic lattice (non-well-mixed; the paper's Sec. 1   */
/* and Sec. 6 motivate compartments but give no algorithm: this is the      */
/* library's reading, stated here in full).                                  */
/* ------------------------------------------------------------------------ */
/* Sites (x, y), x < lx, y < ly, both powers of two, M = lx ly sites, site index x + lx y.  Each
 * site holds counts (L, D, A) and runs Frank's three reactions with propensities k_r h_r
 * (h_1 = A L, h_2 = A D, h_3 = L D; Omega = 1 per site); every molecule hops to each of its four
 * neighbours (x +- 1 mod lx, y) and (x, y +- 1 mod ly) at rate d.  The total count is conserved
 * over the lattice, not per site.
 *
 * Uniformisation, exact: with u = min(k_max, d), rho_r = k_max / u and rho_h = d / u must be
 * integers.  The runs of a group of 32 share an occupancy cap m with every site count of every
 * run <= m, m one of 1 .. 8 or a number with a two-bit mantissa (4 + j) 2^e (j = 0 .. 3: 10, 12,
 * 14, 16, 20, 24, ...); with bh = bit_length(m - 1) (2^bh >= m), a site has c(m) = 4 rho_h 2^bh +
 * rho_r m (m - 1) / 2 slots, K = bit_length(c(m) - 1), and the rate of a step is Lambda = M 2^K u.  One step of group g at step s uses word k = element k % 4 of
 * Philox4x32-10(key = seed, ctr = (g, s lo 32, s hi 16 | 2 << 24, k / 4)):
 *   w0, w1: the waiting time, as for the well-mixed group clock (u53 or its top 24 bits);
 *   w2: the site, sigma = w2 & (M - 1), shared by the runs of the group;
 *   w3 .. w3+K-1: the planes of n (run l: n = sum_i bit_l(w_{3+i}) 2^i), uniform on [0, 2^K);
 *   w35 ..: thinning, U = the q-bit number whose bit q-1-i is bit_l(w_{35+i}).
 * Run l with counts (L, D, A) at sigma, n_s = L + D + A:
 *   n < H = 4 rho_h 2^bh: a hop: direction n & 3 (x+1, x-1, y+1, y-1), molecule
 *     i = (n >> 2) & (2^bh - 1); i < L: an L hops, i < L + D: a D, i < n_s: an A, else nothing;
 *   else the reaction r with H + rho_r S_{r-1} <= n < H + rho_r S_r (S_r = sum_{p<=r} h_p), kept
 *     iff U < T_r = floor(k_r / k_max 2^q) (always when k_r = k_max); none if n is at or above
 *     H + rho_r S_3.
 * A run then jumps by reaction r at sigma at rate (Lambda / M)(rho_r h_r / 2^K)(k_r / k_max) =
 * k_r h_r and moves a given molecule in a given direction at rate (Lambda / M)(1 / 2^K) = d.  After
 * the step, if a hop left a site of any run above m, m becomes the next cap for the next steps
 * (a bound that changes with the state, between steps).  Initially m is the smallest cap at or
 * above every site count of the group's runs.  Runs do not stop before t_end: the output keeps
 * the time at which a run's whole lattice first holds a single species (global homochirality). */
typedef struct {
  int32_t lx, ly;           /* sides, powers of two, lx ly <= 65536 */
  const double* rates;      /* [3] k_r >= 0, max > 0 */
  double hop;               /* d > 0 */
  uint64_t seed;
  int32_t precision;        /* ORC_P64 | ORC_P32_KAHAN | ORC_P32_D64ACC | ORC_P32_PLAIN */
  int32_t thin_bits;        /* q, 1..64 */
  double t_end;             /* finite */
  const double* snap_times; /* [n_snap] ascending, <= t_end */
  int32_t n_snap;
  int64_t step_budget;      /* 0 = unlimited */
} orc_lattice;

typedef struct {
  double t_homochiral;      /* first event time at which the lattice holds one species; +inf */
  int32_t outcome;          /* that species (0 L, 1 D, 2 A), -1 none */
  int32_t status;
  int64_t steps;            /* the group's steps */
  int64_t reactions;        /* this run's reactions */
  int64_t hops;             /* this run's hops */
  int32_t cap;              /* the group's final cap m */
  int32_t pad;
  double margin;            /* smallest relative gap between a snapshot / t_end and an event time */
} orc_lattice_result;

/* The `lanes` runs of group g.  init: int64[lanes][M][3]; out: [lanes]; final: int64[lanes][M][3];
 * snap_totals: int64[lanes][n_snap][3] lattice totals of (L, D, A) at each snapshot;
 * snap_domains: int64[lanes][n_snap][2] sites with L > D and sites with D > L.  The last three
 * may be NULL. */
int orc_lattice_group(const orc_lattice* p, uint64_t group, int32_t lanes, const int64_t* init,
                      orc_lattice_result* out, int64_t* final_counts, int64_t* snap_totals,
                      int64_t* snap_domains);

/* Enantiomeric-excess bin of (L, D): 64 bins over [-1, 1] by floor(64 L / (L + D)),
 * the top edge folded into bin 63; bin 64 holds L + D == 0. */
int32_t orc_ee_bin(int64_t L, int64_t D);

#ifdef __cplusplus
}
#endif
#endif
