/*
 * lattice.c -- CPU oracle for Frank's model on a periodic lattice (the non-well-mixed
 *              configuration), with the uniformisation and random stream defined in
 *              oracle.h (orc_lattice).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests and the benchmark's CPU-baseline leg,
 * never by the product library.  Plain serial stepping of one group of runs with integer
 * counts per site; propensities recomputed from their definition at every step.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define LAT_MAX_LANES 32

static int lat_bit_length(uint64_t v) {
  int b = 0;
  while (v) {
    b++;
    v >>= 1;
  }
  return b;
}

static int is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

/* The smallest occupancy cap at or above v >= 1: caps are 1 .. 8 and then the numbers with a two-bit
 * mantissa, (4 + j) 2^e for j = 0 .. 3 (10, 12, 14, 16, 20, 24, 28, 32, 40, ...). */
static int64_t lat_cap_at_or_above(int64_t v) {
  if (v <= 8) return v < 1 ? 1 : v;
  const int e = lat_bit_length((uint64_t)(v - 1)) - 3; /* 4 2^e < v <= 8 2^e */
  const int64_t unit = (int64_t)1 << e;
  return (v + unit - 1) / unit * unit;
}

/* Word k of the lattice stream of group g at step s (tag 2). */
typedef struct {
  uint32_t key[2];
  uint32_t ctr[4];
  uint32_t out[4];
  int valid;
} lat_words;

static uint32_t lat_word(lat_words* ws, uint64_t group, uint64_t step, uint32_t k) {
  uint32_t ctr[4];
  ctr[0] = (uint32_t)group;
  ctr[1] = (uint32_t)(step & 0xFFFFFFFFu);
  ctr[2] = (uint32_t)((step >> 32) & 0xFFFFu) | (2u << 24);
  ctr[3] = k / 4;
  if (!ws->valid || memcmp(ctr, ws->ctr, sizeof ctr) != 0) {
    memcpy(ws->ctr, ctr, sizeof ctr);
    orc_philox4x32_10(ctr, ws->key, ws->out);
    ws->valid = 1;
  }
  return ws->out[k % 4];
}

/* The neighbour of site i in direction dir: 0 x+1, 1 x-1, 2 y+1, 3 y-1 (periodic). */
static int64_t neighbour(const orc_lattice* p, int64_t i, int dir) {
  int64_t x = i % p->lx, y = i / p->lx;
  if (dir == 0) x = (x + 1) % p->lx;
  if (dir == 1) x = (x + p->lx - 1) % p->lx;
  if (dir == 2) y = (y + 1) % p->ly;
  if (dir == 3) y = (y + p->ly - 1) % p->ly;
  return x + (int64_t)p->lx * y;
}

static double gap_rel(double a, double b, double scale) {
  double g = fabs(a - b);
  return scale > 0.0 ? g / scale : g;
}

int orc_lattice_group(const orc_lattice* p, uint64_t group, int32_t lanes, const int64_t* init,
                      orc_lattice_result* out, int64_t* final_counts, int64_t* snap_totals,
                      int64_t* snap_domains) {
  if (!p || !init || !out || lanes < 1 || lanes > LAT_MAX_LANES) return ORC_EINVAL;
  if (!is_pow2(p->lx) || !is_pow2(p->ly) || (int64_t)p->lx * p->ly > 65536) return ORC_EINVAL;
  if (!(p->hop > 0.0) || !p->rates || p->thin_bits < 1 || p->thin_bits > 64) return ORC_EINVAL;
  if (!(p->t_end >= 0.0) || isinf(p->t_end) || p->n_snap < 0 || (p->n_snap > 0 && !p->snap_times))
    return ORC_EINVAL;
  if (p->precision < ORC_P64 || p->precision > ORC_P32_PLAIN) return ORC_EINVAL;
  const int64_t M = (int64_t)p->lx * p->ly;
  double k_max = 0.0;
  for (int r = 0; r < 3; r++) {
    if (!(p->rates[r] >= 0.0)) return ORC_EINVAL;
    if (p->rates[r] > k_max) k_max = p->rates[r];
  }
  if (!(k_max > 0.0)) return ORC_EINVAL;
  /* integer weights of a reaction slot and of a hop slot, in units of u = min(k_max, d) */
  const double unit = k_max < p->hop ? k_max : p->hop;
  const double rr = k_max / unit, rh = p->hop / unit;
  const int64_t rho_r = (int64_t)llround(rr), rho_h = (int64_t)llround(rh);
  if (fabs(rr - (double)rho_r) > 1e-9 * rr || fabs(rh - (double)rho_h) > 1e-9 * rh) return ORC_EINVAL;
  /* thinning thresholds */
  const int q = p->thin_bits;
  int always[3];
  uint64_t T[3];
  for (int r = 0; r < 3; r++) {
    always[r] = p->rates[r] == k_max;
    T[r] = always[r] ? 0 : (uint64_t)floor(p->rates[r] / k_max * ldexp(1.0, q));
  }
  /* Frank's reactions in (L, D, A): A+L -> 2L, A+D -> 2D, L+D -> 2A */
  static const int nu[3][3] = {{1, 0, -1}, {0, 1, -1}, {-1, -1, 2}};

  int64_t* n = (int64_t*)malloc(sizeof(int64_t) * (size_t)lanes * (size_t)M * 3);
  if (!n) return ORC_EINVAL;
  int64_t tot[LAT_MAX_LANES][3];
  int64_t n_max = 0;
  for (int l = 0; l < lanes; l++) {
    memset(&out[l], 0, sizeof out[l]);
    out[l].t_homochiral = INFINITY;
    out[l].outcome = -1;
    out[l].margin = INFINITY;
    tot[l][0] = tot[l][1] = tot[l][2] = 0;
    for (int64_t i = 0; i < M; i++) {
      int64_t site = 0;
      for (int c = 0; c < 3; c++) {
        const int64_t v = init[((int64_t)l * M + i) * 3 + c];
        if (v < 0) {
          free(n);
          return ORC_EINVAL;
        }
        n[((int64_t)l * M + i) * 3 + c] = v;
        tot[l][c] += v;
        site += v;
      }
      if (site > n_max) n_max = site;
    }
    const int kinds = (tot[l][0] > 0) + (tot[l][1] > 0) + (tot[l][2] > 0);
    if (kinds <= 1) {
      out[l].t_homochiral = 0.0;
      out[l].outcome = tot[l][0] ? 0 : (tot[l][1] ? 1 : (tot[l][2] ? 2 : -1));
    }
  }
  int64_t m = lat_cap_at_or_above(n_max); /* the cap: every site count of every run <= m */

  lat_words ws;
  memset(&ws, 0, sizeof ws);
  ws.key[0] = (uint32_t)(p->seed & 0xFFFFFFFFu);
  ws.key[1] = (uint32_t)(p->seed >> 32);
  double t = 0.0;
  float t_f = 0.0f, c_f = 0.0f;
  int has_event = 0, next_snap = 0, status = ORC_OK;
  int64_t step = 0;

  for (;;) {
    if (p->step_budget > 0 && step >= p->step_budget) {
      status = ORC_ETIMEOUT;
      break;
    }
    const int bh = lat_bit_length((uint64_t)(m - 1)); /* molecule index bits: 2^bh >= m */
    const int64_t hop_slots = 4 * rho_h * ((int64_t)1 << bh);
    const uint64_t c_m = (uint64_t)hop_slots + (uint64_t)rho_r * (uint64_t)(m * (m - 1) / 2);
    const int K = lat_bit_length(c_m - 1);
    if (K > 32) { /* the cap no longer fits the stream's 32 planes of n */
      status = ORC_ERANGE;
      break;
    }
    const double lambda = (double)M * ldexp(unit, K);

    /* (1) the waiting time from w0, w1 */
    const uint32_t w0 = lat_word(&ws, group, (uint64_t)step, 0), w1 = lat_word(&ws, group, (uint64_t)step, 1);
    double t_new;
    float t_f_new = 0.0f, c_f_new = 0.0f;
    if (p->precision == ORC_P64) {
      uint64_t x = ((uint64_t)w1 << 21) | (uint64_t)(w0 >> 11);
      double u = (double)(x + 1) * 0x1p-53;
      t_new = t + (-log(u) / lambda);
    } else {
      float u = (float)((w1 >> 8) + 1u) * 0x1p-24f;
      float tau = -logf(u) * (float)(1.0 / lambda);
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

    /* (2) snapshots: the lattice before the event; t_end stops the group */
    int stop = 0;
    for (;;) {
      const int at_end = !(next_snap < p->n_snap && p->snap_times[next_snap] < t_new);
      if (at_end && !(t_new > p->t_end)) break;
      const double ts = at_end ? p->t_end : p->snap_times[next_snap];
      double g = gap_rel(t_new, ts, ts);
      const double g_before = has_event ? gap_rel(ts, t, ts) : INFINITY;
      if (g_before < g) g = g_before;
      for (int l = 0; l < lanes; l++)
        if (g < out[l].margin) out[l].margin = g;
      if (at_end) {
        stop = 1;
        break;
      }
      for (int l = 0; l < lanes; l++) {
        if (snap_totals)
          for (int c = 0; c < 3; c++) snap_totals[((int64_t)l * p->n_snap + next_snap) * 3 + c] = tot[l][c];
        if (snap_domains) {
          int64_t lsites = 0, dsites = 0;
          for (int64_t i = 0; i < M; i++) {
            const int64_t* si = &n[((int64_t)l * M + i) * 3];
            lsites += si[0] > si[1];
            dsites += si[1] > si[0];
          }
          snap_domains[((int64_t)l * p->n_snap + next_snap) * 2 + 0] = lsites;
          snap_domains[((int64_t)l * p->n_snap + next_snap) * 2 + 1] = dsites;
        }
      }
      next_snap++;
    }
    if (stop) break;
    t = t_new;
    t_f = t_f_new;
    c_f = c_f_new;
    has_event = 1;

    /* (3) the site, shared by the group, and every run's event there */
    const int64_t sigma = (int64_t)(lat_word(&ws, group, (uint64_t)step, 2) & (uint32_t)(M - 1));
    int overflow = 0;
    for (int l = 0; l < lanes; l++) {
      int64_t* sv = &n[((int64_t)l * M + sigma) * 3];
      uint64_t draw = 0;
      for (int i = 0; i < K; i++)
        draw |= (uint64_t)((lat_word(&ws, group, (uint64_t)step, 3 + (uint32_t)i) >> l) & 1u) << i;
      if (draw < (uint64_t)hop_slots) {
        /* a hop: direction from the low two bits, the molecule from the next bh bits */
        const int dir = (int)(draw & 3u);
        const int64_t mol = (int64_t)((draw >> 2) & (((uint64_t)1 << bh) - 1));
        int species = -1;
        if (mol < sv[0]) species = 0;
        else if (mol < sv[0] + sv[1]) species = 1;
        else if (mol < sv[0] + sv[1] + sv[2]) species = 2;
        if (species < 0) continue;
        int64_t* nb = &n[((int64_t)l * M + neighbour(p, sigma, dir)) * 3];
        sv[species]--;
        nb[species]++;
        out[l].hops++;
        if (nb[0] + nb[1] + nb[2] > m) overflow = 1;
        continue;
      }
      /* a reaction: the CDF walk over rho_r S_r above the hop slots */
      const int64_t h[3] = {sv[2] * sv[0], sv[2] * sv[1], sv[0] * sv[1]};
      uint64_t partial = (uint64_t)hop_slots;
      int r = -1;
      for (int k = 0; k < 3; k++) {
        partial += (uint64_t)rho_r * (uint64_t)h[k];
        if (draw < partial) {
          r = k;
          break;
        }
      }
      if (r < 0) continue;
      if (!always[r]) {
        uint64_t U = 0;
        for (int i = 0; i < q; i++) {
          uint32_t w = lat_word(&ws, group, (uint64_t)step, 35 + (uint32_t)i);
          U |= (uint64_t)((w >> l) & 1u) << (q - 1 - i);
        }
        if (!(U < T[r])) continue;
      }
      for (int c = 0; c < 3; c++) {
        sv[c] += nu[r][c];
        tot[l][c] += nu[r][c];
        if (sv[c] < 0) {
          free(n);
          return ORC_ERANGE;
        }
      }
      out[l].reactions++;
      if (out[l].outcome == -1 && (tot[l][0] > 0) + (tot[l][1] > 0) + (tot[l][2] > 0) == 1) {
        out[l].t_homochiral = t;
        out[l].outcome = tot[l][0] ? 0 : (tot[l][1] ? 1 : 2);
      }
    }
    step++;
    if (overflow) m = lat_cap_at_or_above(m + 1);
  }

  for (int l = 0; l < lanes; l++) {
    out[l].steps = step;
    out[l].cap = (int32_t)m;
    out[l].status = status;
    if (final_counts)
      memcpy(&final_counts[(int64_t)l * M * 3], &n[(int64_t)l * M * 3], sizeof(int64_t) * (size_t)M * 3);
  }
  free(n);
  return status;
}
