/*
 * oracle.c -- CPU oracle for the bit-sliced Gillespie method (arXiv 2412.16613).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product library.
 *
 * Plain serial Gillespie, one run at a time, integer counts, propensities
 * recomputed from their definition at every step.  Under the state-following
 * bound (pad_pow2 = 2) the 32 runs of a group are stepped together, since the
 * bound of each step depends on all of them.  The random stream and the
 * integer reaction-choice rule are described in oracle.h.  Compile with
 * -ffp-contract=off.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from the description in Salmon, Moraes, Dror and   */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of */
/* two 32x32->64 multiplications whose high halves are xored into the other  */
/* words together with the round key; the key is bumped by the two Weyl      */
/* constants between rounds.                                                  */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_MUL_A = 0xD2511F53u;
static const uint32_t PHILOX_MUL_B = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL_A = 0x9E3779B9u;
static const uint32_t PHILOX_WEYL_B = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) {
      k0 += PHILOX_WEYL_A;
      k1 += PHILOX_WEYL_B;
    }
    uint64_t prod_a = (uint64_t)PHILOX_MUL_A * (uint64_t)x0;
    uint64_t prod_b = (uint64_t)PHILOX_MUL_B * (uint64_t)x2;
    uint32_t n0 = (uint32_t)(prod_b >> 32) ^ x1 ^ k0;
    uint32_t n1 = (uint32_t)prod_b;
    uint32_t n2 = (uint32_t)(prod_a >> 32) ^ x3 ^ k1;
    uint32_t n3 = (uint32_t)prod_a;
    x0 = n0;
    x1 = n1;
    x2 = n2;
    x3 = n3;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

static void stream_counter(uint64_t group, uint64_t step, uint32_t attempt, uint32_t tag,
                           uint32_t call, uint32_t ctr[4]) {
  ctr[0] = (uint32_t)group;
  ctr[1] = (uint32_t)(step & 0xFFFFFFFFu);
  ctr[2] = (uint32_t)((step >> 32) & 0xFFFFu) | (attempt << 16) | (tag << 24);
  ctr[3] = call;
}

uint32_t orc_stream_word(uint64_t seed, uint64_t group, uint64_t step, uint32_t attempt,
                         uint32_t tag, uint32_t k) {
  uint32_t ctr[4], key[2], out[4];
  stream_counter(group, step, attempt, tag, k / 4, ctr);
  key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
  key[1] = (uint32_t)(seed >> 32);
  orc_philox4x32_10(ctr, key, out);
  return out[k % 4];
}

/* A one-entry cache so that the four words of a Philox call are not
 * recomputed four times; it changes nothing but speed. */
typedef struct {
  uint32_t key[2];
  uint32_t ctr[4];
  uint32_t out[4];
  int valid;
} word_source;

static uint32_t word_at(word_source* ws, uint64_t group, uint64_t step, uint32_t attempt,
                        uint32_t tag, uint32_t k) {
  uint32_t ctr[4];
  stream_counter(group, step, attempt, tag, k / 4, ctr);
  if (!ws->valid || memcmp(ctr, ws->ctr, sizeof ctr) != 0) {
    memcpy(ws->ctr, ctr, sizeof ctr);
    orc_philox4x32_10(ctr, ws->key, ws->out);
    ws->valid = 1;
  }
  return ws->out[k % 4];
}

static uint32_t lane_bit(uint32_t word, int lane) { return (word >> lane) & 1u; }

/* The two waiting-time words of run j at step s under the per-run clock: words 0 and 1 of
 * Philox4x32-10 with counter (j lo 32, s lo 32, s hi 16 | (j >> 32) << 16 | 1 << 24, 0). */
static void lane_clock_words(const word_source* ws, int64_t run, int64_t step, uint32_t* w0, uint32_t* w1) {
  uint32_t ctr[4], out[4];
  ctr[0] = (uint32_t)((uint64_t)run & 0xFFFFFFFFu);
  ctr[1] = (uint32_t)((uint64_t)step & 0xFFFFFFFFu);
  ctr[2] = (uint32_t)(((uint64_t)step >> 32) & 0xFFFFu) | (uint32_t)((((uint64_t)run >> 32) & 0xFFu) << 16) |
           (1u << 24);
  ctr[3] = 0u;
  orc_philox4x32_10(ctr, ws->key, out);
  *w0 = out[0];
  *w1 = out[1];
}

/* ------------------------------------------------------------------------ */
/* The network: propensities (Eq. equation-as generalised to order <= 2     */
/* mass action), the uniformisation bound, thinning thresholds.              */
/* ------------------------------------------------------------------------ */
static int reaction_order(const orc_problem* p, int r) {
  int order = 0;
  for (int i = 0; i < p->n_species; i++) order += p->reactants[r * p->n_species + i];
  return order;
}

/* h_r = prod_i C(n_i, m_i): n_i n_j, n_i (n_i - 1) / 2 or n_i. */
static int64_t propensity(const orc_problem* p, int r, const int64_t* n) {
  int64_t h = 1;
  for (int i = 0; i < p->n_species; i++) {
    int m = p->reactants[r * p->n_species + i];
    if (m == 1) h *= n[i];
    if (m == 2) h *= n[i] * (n[i] - 1) / 2;
  }
  return h;
}

int orc_propensities(const orc_problem* p, const int64_t* state, int64_t* h) {
  for (int r = 0; r < p->n_reactions; r++) h[r] = propensity(p, r, state);
  return ORC_OK;
}

/* The CDF walk of Sec. 3 step 5: m runs over the partial sums S_r, and the
 * first reaction whose partial sum exceeds n fires. */
int32_t orc_select(const orc_problem* p, const int64_t* state, uint64_t n) {
  uint64_t partial = 0;
  for (int r = 0; r < p->n_reactions; r++) {
    partial += (uint64_t)propensity(p, r, state);
    if (n < partial) return r;
  }
  return -1;
}

static int64_t real_propensity_sum(const orc_problem* p, const int64_t* n) {
  int64_t total = 0;
  for (int r = 0; r < p->n_reactions; r++)
    if (p->rates[r] > 0.0) total += propensity(p, r, n);
  return total;
}

static int bit_length(uint64_t v) {
  int b = 0;
  while (v) {
    b++;
    v >>= 1;
  }
  return b;
}

int orc_derive(const orc_problem* p, orc_derived* d) {
  memset(d, 0, sizeof *d);
  if (p->n_species < 1 || p->n_species > ORC_MAX_SPECIES) return ORC_EINVAL;
  if (p->n_reactions < 1 || p->n_reactions > ORC_MAX_REACTIONS) return ORC_EINVAL;
  if (p->n_tot < 1 || p->n_tot > (1 << 20)) return ORC_EINVAL;
  if (p->thin_bits < 1 || p->thin_bits > 64) return ORC_EINVAL;
  if (p->precision < ORC_P64 || p->precision > ORC_P32_PLAIN) return ORC_EINVAL;
  if (!(p->t_end >= 0.0) || p->n_snap < 0) return ORC_EINVAL;
  for (int s = 0; s < p->n_snap; s++) {
    if (!(p->snap_times[s] >= 0.0) || p->snap_times[s] > p->t_end) return ORC_EINVAL;
    if (s > 0 && p->snap_times[s] < p->snap_times[s - 1]) return ORC_EINVAL;
  }
  int pair_count[ORC_MAX_SPECIES][ORC_MAX_SPECIES];
  int uni_count[ORC_MAX_SPECIES];
  memset(pair_count, 0, sizeof pair_count);
  memset(uni_count, 0, sizeof uni_count);
  double k_max = 0.0;
  for (int r = 0; r < p->n_reactions; r++) {
    int order = reaction_order(p, r), made = 0;
    if (order < 1 || order > 2) return ORC_EINVAL;
    for (int i = 0; i < p->n_species; i++) {
      if (p->reactants[r * p->n_species + i] < 0 || p->products[r * p->n_species + i] < 0)
        return ORC_EINVAL;
      made += p->products[r * p->n_species + i];
    }
    if (made != order) return ORC_EINVAL; /* the total count must be conserved (Sec. 2) */
    double k = p->rates[r];
    if (!(k >= 0.0) || isinf(k)) return ORC_EINVAL;
    if (k > k_max) k_max = k;
    int first = -1, second = -1;
    for (int i = 0; i < p->n_species; i++) {
      int m = p->reactants[r * p->n_species + i];
      if (m == 2) first = second = i;
      if (m == 1) {
        if (first < 0) first = i;
        else second = i;
      }
    }
    if (order == 2) pair_count[first][second]++;
    else uni_count[first]++;
  }
  if (!(k_max > 0.0)) return ORC_EINVAL;
  int m_pair = 0, u_max = 0;
  for (int i = 0; i < p->n_species; i++) {
    if (uni_count[i] > u_max) u_max = uni_count[i];
    for (int j = 0; j < p->n_species; j++)
      if (pair_count[i][j] > m_pair) m_pair = pair_count[i][j];
  }
  /* Over all states with sum_i n_i = N, sum_{i<j} n_i n_j + sum_i C(n_i, 2) = C(N, 2)
   * (Eq. equation-z); each unordered reactant pair carries at most m_pair reactions
   * and each species at most u_max first-order ones. */
  uint64_t N = (uint64_t)p->n_tot;
  d->lambda_int = (uint64_t)m_pair * (N * (N - 1) / 2) + (uint64_t)u_max * N;
  d->K = bit_length(d->lambda_int);
  /* Uniformisation at any bound at or above the largest total propensity samples the same
   * process; padding the bound to 2^K with further null events makes every K-bit n valid. */
  if (p->pad_pow2 < 0 || p->pad_pow2 > 2 || p->ensemble_runs < 0) return ORC_EINVAL;
  if (p->lane_clock != 0 && p->lane_clock != 1) return ORC_EINVAL;
  if (p->lane_clock && p->pad_pow2 == 2) return ORC_EINVAL; /* not built */
  if (p->pad_pow2) d->lambda_int = (uint64_t)1 << d->K;
  d->k_max = k_max;
  d->lambda = k_max * (double)d->lambda_int;
  for (int r = 0; r < p->n_reactions; r++) {
    if (p->rates[r] == k_max) {
      d->thin_always[r] = 1;
    } else {
      d->thin_always[r] = 0;
      d->thin_T[r] = (uint64_t)floor(ldexp(p->rates[r] / k_max, p->thin_bits));
      d->any_thinning = 1;
    }
  }
  return ORC_OK;
}

int32_t orc_ee_bin(int64_t L, int64_t D) {
  if (L + D == 0) return 64;
  int64_t bin = (64 * L) / (L + D);
  return bin > 63 ? 63 : (int32_t)bin;
}

static int32_t outcome_of(const orc_problem* p, const int64_t* n) {
  int32_t who = -1, alive = 0;
  for (int i = 0; i < p->n_species; i++)
    if (n[i] != 0) {
      who = i;
      alive++;
    }
  return alive == 1 ? who : -2;
}

static double relative_gap(double a, double b, double scale) {
  double gap = fabs(a - b);
  return scale > 0.0 ? gap / scale : gap;
}

/* ------------------------------------------------------------------------ */
/* One run.                                                                  */
/* ------------------------------------------------------------------------ */
int orc_run(const orc_problem* p, const orc_derived* d, int64_t run_index, const int64_t* init,
            orc_result* out, int64_t* snap_counts) {
  const int S = p->n_species;
  const int K = d->K;
  const uint64_t group = (uint64_t)run_index / 32;
  const int lane = (int)(run_index % 32);
  int64_t n[ORC_MAX_SPECIES];
  int64_t total = 0;

  memset(out, 0, sizeof *out);
  out->t_abs = INFINITY;
  out->outcome = -1;
  out->margin = INFINITY;
  if (p->pad_pow2 == 2) return out->status = ORC_EINVAL; /* needs the whole group: orc_run_group */
  for (int i = 0; i < S; i++) {
    n[i] = init[i];
    total += n[i];
    if (n[i] < 0) return out->status = ORC_EINVAL;
  }
  if (total != p->n_tot) return out->status = ORC_EINVAL;

  word_source ws;
  memset(&ws, 0, sizeof ws);
  ws.key[0] = (uint32_t)(p->seed & 0xFFFFFFFFu);
  ws.key[1] = (uint32_t)(p->seed >> 32);

  double t = 0.0;        /* P64 and P32_D64ACC clock */
  float t_f = 0.0f, c_f = 0.0f; /* P32_KAHAN clock and its compensation */
  const float inv_lambda_f = (float)(1.0 / d->lambda);
  int has_event = 0;     /* whether t is the time of a committed step */
  int next_snap = 0;
  int64_t step = 0;

  if (real_propensity_sum(p, n) == 0) {
    out->t_abs = 0.0;
    out->outcome = outcome_of(p, n);
    goto fill_snapshots;
  }

  for (;;) {
    if (p->step_budget > 0 && step >= p->step_budget) {
      out->status = ORC_ETIMEOUT;
      break;
    }
    /* (1) the integer n, uniform in [0, lambda_int), by per-lane rejection.  A rejected
     * draw (draw >= lambda_int) redraws its bits from position p up, p being the highest
     * bit where it differs from lambda_int (all bits when it equals lambda_int), and keeps
     * the bits below p: they are uniform and independent of the rejection, so the new
     * draw is again uniform on [0, 2^K) and the accepted one uniform on [0, lambda_int). */
    const int n_lane = p->shared_n ? 0 : lane;  /* whose bits make n */
    uint64_t draw = 0;
    for (int i = 0; i < K; i++)
      draw |= (uint64_t)lane_bit(word_at(&ws, group, (uint64_t)step, 0, 0, (uint32_t)i), n_lane) << i;
    uint32_t attempt = 0;
    while (draw >= d->lambda_int) {
      attempt++;
      if (attempt >= 64) return out->status = ORC_ERANGE;
      int from = draw == d->lambda_int ? 0 : bit_length(draw ^ d->lambda_int) - 1;
      draw &= ((uint64_t)1 << from) - 1;
      for (int i = from; i < K; i++)
        draw |= (uint64_t)lane_bit(word_at(&ws, group, (uint64_t)step, attempt, 0, (uint32_t)i),
                                   n_lane) << i;
    }
    out->redraws += attempt;

    /* (2) the waiting time, from the whole words K and K+1 of attempt 0 (per-run clock: the
     * words 0 and 1 of the run's own stream) */
    uint32_t wk0, wk1;
    if (p->lane_clock) {
      lane_clock_words(&ws, run_index, step, &wk0, &wk1);
    } else {
      wk0 = word_at(&ws, group, (uint64_t)step, 0, 0, (uint32_t)K);
      wk1 = word_at(&ws, group, (uint64_t)step, 0, 0, (uint32_t)K + 1);
    }
    double t_new;
    float t_f_new = 0.0f, c_f_new = 0.0f;
    if (p->precision == ORC_P64) {
      uint64_t x = ((uint64_t)wk1 << 21) | (uint64_t)(wk0 >> 11);
      double u = (double)(x + 1) * 0x1p-53;
      double tau = -log(u) / d->lambda;
      t_new = t + tau;
    } else {
      /* the top 24 of the 53 bits above: the fp32 clock is a rounding of the fp64 one */
      float u = (float)((wk1 >> 8) + 1u) * 0x1p-24f;
      float tau = -logf(u) * inv_lambda_f;
      if (p->precision == ORC_P32_KAHAN) {
        float y = tau - c_f;
        float sum = t_f + y;
        c_f_new = (sum - t_f) - y;
        t_f_new = sum;
        t_new = (double)sum;
      } else if (p->precision == ORC_P32_PLAIN) {
        t_f_new = t_f + tau;
        t_new = (double)t_f_new;
      } else {
        t_new = t + (double)tau;
      }
    }

    /* (3) snapshots hold the state after every event no later than their time */
    while (next_snap < p->n_snap && p->snap_times[next_snap] < t_new) {
      double ts = p->snap_times[next_snap];
      double gap = relative_gap(t_new, ts, ts);
      if (gap < out->margin) out->margin = gap;
      if (has_event) {
        gap = relative_gap(ts, t, ts);
        if (gap < out->margin) out->margin = gap;
      }
      if (snap_counts)
        for (int i = 0; i < S; i++) snap_counts[(int64_t)next_snap * S + i] = n[i];
      next_snap++;
    }
    if (t_new > p->t_end) {
      double gap = relative_gap(t_new, p->t_end, p->t_end);
      if (gap < out->margin) out->margin = gap;
      if (has_event) {
        gap = relative_gap(p->t_end, t, p->t_end);
        if (gap < out->margin) out->margin = gap;
      }
      break;
    }
    t = t_new;
    t_f = t_f_new;
    c_f = c_f_new;
    has_event = 1;

    /* (4) the reaction: CDF walk on the integer propensities */
    int32_t r = orc_select(p, n, draw);
    if (r >= 0 && !d->thin_always[r]) {
      uint64_t U = 0;
      for (int i = 0; i < p->thin_bits; i++) {
        uint32_t w = word_at(&ws, group, (uint64_t)step, 0, 0, (uint32_t)(K + 2 + i));
        U |= (uint64_t)lane_bit(w, lane) << (p->thin_bits - 1 - i);
      }
      if (!(U < d->thin_T[r])) r = -1;
    }
    if (r >= 0) {
      int64_t check = 0;
      for (int i = 0; i < S; i++) {
        n[i] += p->products[r * S + i] - p->reactants[r * S + i];
        if (n[i] < 0) return out->status = ORC_ERANGE;
        check += n[i];
      }
      if (check != p->n_tot) return out->status = ORC_ERANGE;
      out->reactions++;
    }
    step++;

    /* (5) absorption: no real reaction can fire any more */
    if (r >= 0 && real_propensity_sum(p, n) == 0) {
      out->t_abs = t;
      out->outcome = outcome_of(p, n);
      break;
    }
  }

fill_snapshots:
  /* an absorbed run keeps its state for ever */
  if (out->outcome != -1 && snap_counts)
    for (; next_snap < p->n_snap; next_snap++)
      for (int i = 0; i < S; i++) snap_counts[(int64_t)next_snap * S + i] = n[i];
  for (int i = 0; i < S; i++) out->final_counts[i] = n[i];
  out->steps = step;
  out->t_last = (p->precision == ORC_P32_KAHAN || p->precision == ORC_P32_PLAIN) ? (double)t_f : t;
  return out->status;
}

/* ------------------------------------------------------------------------ */
/* A group of runs under a bound that follows the group's state.             */
/* ------------------------------------------------------------------------ */
/* Uniformisation samples the process at any rate that is at least the total
 * propensity, and the rate may change with the state, which is constant between
 * steps.  With pad_pow2 = 2 the bound of a step is 2^p, p the bit length of the
 * largest S_R over the group's live runs, so S_R < 2^p for every live run and a
 * p-bit n always lands in [0, 2^p).  A run still jumps by reaction r at rate
 * (k_max 2^p) (h_r / 2^p) (k_r / k_max) = k_r h_r, whatever the other runs hold. */
static int group_bound_bits(const orc_problem* p, int lanes, const int64_t (*n)[ORC_MAX_SPECIES],
                            const int* live) {
  uint64_t top = 0;
  for (int l = 0; l < lanes; l++) {
    if (!live[l]) continue;
    uint64_t sum = 0;
    for (int r = 0; r < p->n_reactions; r++) sum += (uint64_t)propensity(p, r, n[l]);
    if (sum > top) top = sum;
  }
  return bit_length(top);
}

int orc_run_group(const orc_problem* p, const orc_derived* d, uint64_t group, int32_t lanes,
                  const int64_t* init, int32_t init_per_lane, orc_result* out, int64_t* snap_counts) {
  const int S = p->n_species;
  const int K = d->K;
  if (p->pad_pow2 != 2 || lanes < 1 || lanes > 32) return ORC_EINVAL;
  int64_t n[32][ORC_MAX_SPECIES];
  int live[32];
  int n_live = 0;
  for (int l = 0; l < lanes; l++) {
    memset(&out[l], 0, sizeof out[l]);
    out[l].t_abs = INFINITY;
    out[l].outcome = -1;
    out[l].margin = INFINITY;
    const int64_t* c = init + (init_per_lane ? (int64_t)l * S : 0);
    int64_t total = 0;
    for (int i = 0; i < S; i++) {
      n[l][i] = c[i];
      total += c[i];
      if (c[i] < 0) return ORC_EINVAL;
    }
    if (total != p->n_tot) return ORC_EINVAL;
    live[l] = real_propensity_sum(p, n[l]) > 0;
    if (!live[l]) {
      out[l].t_abs = 0.0;
      out[l].outcome = outcome_of(p, n[l]);
    }
    n_live += live[l];
  }

  word_source ws;
  memset(&ws, 0, sizeof ws);
  ws.key[0] = (uint32_t)(p->seed & 0xFFFFFFFFu);
  ws.key[1] = (uint32_t)(p->seed >> 32);
  double t = 0.0;
  float t_f = 0.0f, c_f = 0.0f;
  int has_event = 0, next_snap = 0, status = ORC_OK;
  int64_t step = 0;

  while (n_live > 0) {
    if (p->step_budget > 0 && step >= p->step_budget) {
      status = ORC_ETIMEOUT;
      break;
    }
    /* (1) this step's bound from the group's state */
    const int bits = group_bound_bits(p, lanes, (const int64_t(*)[ORC_MAX_SPECIES])n, live);
    const double lambda_s = ldexp(d->k_max, bits);

    /* (2) the waiting time at rate lambda_s, from the words K and K+1 of attempt 0 */
    uint32_t wk0 = word_at(&ws, group, (uint64_t)step, 0, 0, (uint32_t)K);
    uint32_t wk1 = word_at(&ws, group, (uint64_t)step, 0, 0, (uint32_t)K + 1);
    double t_new;
    float t_f_new = 0.0f, c_f_new = 0.0f;
    if (p->precision == ORC_P64) {
      uint64_t x = ((uint64_t)wk1 << 21) | (uint64_t)(wk0 >> 11);
      double u = (double)(x + 1) * 0x1p-53;
      t_new = t + (-log(u) / lambda_s);
    } else {
      float u = (float)((wk1 >> 8) + 1u) * 0x1p-24f;
      float tau = -logf(u) * (float)(1.0 / lambda_s);
      if (p->precision == ORC_P32_KAHAN) {
        float y = tau - c_f;
        float sum = t_f + y;
        c_f_new = (sum - t_f) - y;
        t_f_new = sum;
        t_new = (double)sum;
      } else if (p->precision == ORC_P32_PLAIN) {
        t_f_new = t_f + tau;
        t_new = (double)t_f_new;
      } else {
        t_new = t + (double)tau;
      }
    }

    /* (3) snapshots and t_end, as for a single run */
    int stop = 0;
    for (;;) {
      const int at_end = !(next_snap < p->n_snap && p->snap_times[next_snap] < t_new);
      if (at_end && !(t_new > p->t_end)) break;
      const double ts = at_end ? p->t_end : p->snap_times[next_snap];
      double gap = relative_gap(t_new, ts, ts);
      double gap_before = has_event ? relative_gap(ts, t, ts) : INFINITY;
      if (gap_before < gap) gap = gap_before;
      for (int l = 0; l < lanes; l++)
        if (live[l] && gap < out[l].margin) out[l].margin = gap;
      if (at_end) {
        stop = 1;
        break;
      }
      if (snap_counts)
        for (int l = 0; l < lanes; l++)
          for (int i = 0; i < S; i++)
            snap_counts[((int64_t)l * p->n_snap + next_snap) * S + i] = n[l][i];
      next_snap++;
    }
    if (stop) break;
    t = t_new;
    t_f = t_f_new;
    c_f = c_f_new;
    has_event = 1;

    /* (4) every live run draws its n from the low `bits` planes and reacts */
    for (int l = 0; l < lanes; l++) {
      if (!live[l]) continue;
      const int n_lane = p->shared_n ? 0 : l;
      uint64_t draw = 0;
      for (int i = 0; i < bits; i++)
        draw |= (uint64_t)lane_bit(word_at(&ws, group, (uint64_t)step, 0, 0, (uint32_t)i), n_lane) << i;
      int32_t r = orc_select(p, n[l], draw);
      if (r >= 0 && !d->thin_always[r]) {
        uint64_t U = 0;
        for (int i = 0; i < p->thin_bits; i++) {
          uint32_t w = word_at(&ws, group, (uint64_t)step, 0, 0, (uint32_t)(K + 2 + i));
          U |= (uint64_t)lane_bit(w, l) << (p->thin_bits - 1 - i);
        }
        if (!(U < d->thin_T[r])) r = -1;
      }
      if (r < 0) continue;
      int64_t check = 0;
      for (int i = 0; i < S; i++) {
        n[l][i] += p->products[r * S + i] - p->reactants[r * S + i];
        if (n[l][i] < 0) return ORC_ERANGE;
        check += n[l][i];
      }
      if (check != p->n_tot) return ORC_ERANGE;
      out[l].reactions++;
    }
    step++;

    /* (5) absorption, run by run */
    for (int l = 0; l < lanes; l++) {
      if (!live[l] || real_propensity_sum(p, n[l]) != 0) continue;
      live[l] = 0;
      n_live--;
      out[l].t_abs = t;
      out[l].outcome = outcome_of(p, n[l]);
      out[l].steps = step;
      out[l].t_last = (p->precision == ORC_P32_KAHAN || p->precision == ORC_P32_PLAIN) ? (double)t_f : t;
    }
  }

  for (int l = 0; l < lanes; l++) {
    if (out[l].outcome != -1 && snap_counts)  /* an absorbed run keeps its state for ever */
      for (int s = next_snap; s < p->n_snap; s++)
        for (int i = 0; i < S; i++) snap_counts[((int64_t)l * p->n_snap + s) * S + i] = n[l][i];
    for (int i = 0; i < S; i++) out[l].final_counts[i] = n[l][i];
    if (live[l]) {
      out[l].steps = step;
      out[l].t_last = (p->precision == ORC_P32_KAHAN || p->precision == ORC_P32_PLAIN) ? (double)t_f : t;
      out[l].status = status;
    }
  }
  return status;
}

/* ------------------------------------------------------------------------ */
/* Many runs over host threads.                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_problem* p;
  const orc_derived* d;
  int64_t first_run;
  const int64_t* run_ids;
  int64_t n_runs;
  const int64_t* init;
  int32_t init_per_run;
  orc_result* out;
  int64_t* snap_counts;
  int64_t next; /* shared work counter */
  int status;
  pthread_mutex_t lock;
} batch_job;

/* pad_pow2 = 2: a run's result comes out of its whole group, which is kept while the
 * following runs asked for fall in the same group. */
static void* group_worker(void* arg) {
  batch_job* job = (batch_job*)arg;
  const orc_problem* p = job->p;
  const int S = p->n_species;
  const int64_t per_group = (int64_t)p->n_snap * S;
  orc_result res[32];
  int64_t lane_init[32 * ORC_MAX_SPECIES];
  int64_t* snaps = NULL;
  if (job->snap_counts && p->n_snap > 0) snaps = (int64_t*)malloc(sizeof(int64_t) * 32 * (size_t)per_group);
  int64_t held = -1; /* the group in res, -1 none */
  int held_status = ORC_OK, held_lanes = 0;
  for (;;) {
    int64_t i = __atomic_fetch_add(&job->next, 16, __ATOMIC_RELAXED);
    if (i >= job->n_runs) break;
    int64_t stop = i + 16 < job->n_runs ? i + 16 : job->n_runs;
    for (; i < stop; i++) {
      const int64_t run = job->run_ids ? job->run_ids[i] : job->first_run + i;
      const int64_t g = run / 32;
      int st = ORC_OK;
      if (run < 0 || (p->ensemble_runs > 0 && run >= p->ensemble_runs)) {
        st = ORC_EINVAL;
      } else {
        if (g != held) {
          int64_t left = p->ensemble_runs > 0 ? p->ensemble_runs - 32 * g : 32;
          held_lanes = left < 32 ? (int)left : 32;
          for (int l = 0; l < held_lanes; l++)
            for (int k = 0; k < S; k++)
              lane_init[l * S + k] = job->init[(job->init_per_run ? (32 * g + l) * S : 0) + k];
          held_status = orc_run_group(p, job->d, (uint64_t)g, held_lanes, lane_init, 1, res, snaps);
          held = g;
        }
        const int lane = (int)(run % 32);
        job->out[i] = res[lane];
        if (held_status != ORC_OK && held_status != ORC_ETIMEOUT) st = held_status;
        else st = res[lane].status;
        if (snaps)
          for (int s = 0; s < p->n_snap; s++)
            for (int k = 0; k < S; k++)
              job->snap_counts[((int64_t)s * job->n_runs + i) * S + k] = snaps[lane * per_group + s * S + k];
      }
      if (st != ORC_OK) {
        job->out[i].status = st;
        pthread_mutex_lock(&job->lock);
        if (job->status == ORC_OK) job->status = st;
        pthread_mutex_unlock(&job->lock);
      }
    }
  }
  free(snaps);
  return NULL;
}

static void* batch_worker(void* arg) {
  batch_job* job = (batch_job*)arg;
  const int S = job->p->n_species;
  if (job->p->pad_pow2 == 2) return group_worker(arg);
  int64_t* snaps = NULL;
  if (job->snap_counts && job->p->n_snap > 0)
    snaps = (int64_t*)malloc(sizeof(int64_t) * (size_t)job->p->n_snap * (size_t)S);
  for (;;) {
    int64_t i = __atomic_fetch_add(&job->next, 16, __ATOMIC_RELAXED);
    if (i >= job->n_runs) break;
    int64_t stop = i + 16 < job->n_runs ? i + 16 : job->n_runs;
    for (; i < stop; i++) {
      int64_t run = job->run_ids ? job->run_ids[i] : job->first_run + i;
      const int64_t* init = job->init + (job->init_per_run ? i * S : 0);
      int st = orc_run(job->p, job->d, run, init, &job->out[i], snaps);
      if (snaps)
        for (int s = 0; s < job->p->n_snap; s++)
          for (int k = 0; k < S; k++)
            job->snap_counts[((int64_t)s * job->n_runs + i) * S + k] = snaps[(int64_t)s * S + k];
      if (st != ORC_OK) {
        pthread_mutex_lock(&job->lock);
        if (job->status == ORC_OK) job->status = st;
        pthread_mutex_unlock(&job->lock);
      }
    }
  }
  free(snaps);
  return NULL;
}

int orc_run_many(const orc_problem* p, int64_t first_run, const int64_t* run_ids, int64_t n_runs,
                 const int64_t* init, int32_t init_per_run, orc_result* out,
                 int64_t* snap_counts, int32_t n_threads) {
  orc_derived d;
  int st = orc_derive(p, &d);
  if (st != ORC_OK) return st;
  if (n_runs <= 0) return ORC_OK;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  batch_job job;
  memset(&job, 0, sizeof job);
  job.p = p;
  job.d = &d;
  job.first_run = first_run;
  job.run_ids = run_ids;
  job.n_runs = n_runs;
  job.init = init;
  job.init_per_run = init_per_run;
  job.out = out;
  job.snap_counts = snap_counts;
  pthread_mutex_init(&job.lock, NULL);
  pthread_t threads[256];
  int started = 0;
  for (int i = 1; i < n_threads; i++)
    if (pthread_create(&threads[started], NULL, batch_worker, &job) == 0) started++;
  batch_worker(&job);
  for (int i = 0; i < started; i++) pthread_join(threads[i], NULL);
  pthread_mutex_destroy(&job.lock);
  return job.status;
}
