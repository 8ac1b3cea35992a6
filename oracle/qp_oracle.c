/*
 * qp_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-thread-per-replica CPU oracle for the one-hot UAV path
 * QUBO of "GPU-Accelerated Quantum Annealing-Inspired UAV Path Planning for
 * Smart Agriculture" (Sections II and III-B, Eqs. 1-6, Algorithm 1) and for the
 * many-replica Metropolis annealer that samples it.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load this file.  It shares no
 * code, header, table or constant generator with the CUDA library: every step is
 * written here again from the paper's definitions.
 *
 * Readings of the paper taken here (the paper is silent or garbled on these):
 *  R1 cells: free cells numbered in row-major grid order, integer (row, col)
 *     coordinates at unit pitch (Section II; w_grid/v = 1 s cancels).
 *  R2 distance: d_ij = round(scale * sqrt(dr^2 + dc^2)), computed exactly in
 *     integers (Section II defines d_ij as the Euclidean distance, t_ij = d*tau).
 *  R3 weights: A multiplies the one-hot penalties (the paper's lambda_p) and B
 *     the distance term (the paper's A in Eq. 6).
 *  R4 every t-range in the penalties of Eqs. 1c, 4, 5 runs over 0..C-1; the
 *     distance term of Eq. 3 over t = 0..C-2 (open path).
 *  R5 start clamp (Section II, x_{0,0} = 1): x_{0,s} = 1 for the start cell s,
 *     the rest of row 0 and of column s are frozen at 0 and never proposed.
 *  R6 Metropolis sweep: sweep s visits free k = t*C + i in increasing order,
 *     accepts iff dE <= 0 or (dE < len_s and u < thr_s[dE]) with
 *     thr_s[dE] = floor(2^32 exp(-dE/T_s)), T_s = T0 (T1/T0)^(s/(S-1)).
 *  R7 random numbers: Philox4x32-10 (Salmon et al., SC'11) with key
 *     (seed_lo, seed_hi) and counter (k>>2, s, replica, 0x51505448); the draw of
 *     variable k is output word k&3.
 *  R8 best energy: the minimum of E over the ends of the sweeps run in which
 *     the state is feasible (every row and column sum is 1); INT64_MAX if none.
 *     A QUBO without path structure has no feasibility test: every sweep end
 *     counts.
 *  R9 extended objective (Section V names battery capacity and the pesticide
 *     amount as the next objectives and gives no formula): the distance term
 *     of Eq. 3 with one integer weight per leg, sum_t w_t d_ij x_{t,i}
 *     x_{t+1,j} (w_t = B for every t is Eq. 3 itself).  With a fixed amount
 *     sprayed per cell the mass carried on leg t falls with t, and a leg's
 *     flight energy is taken as proportional to mass times distance; the
 *     weights are that mass in integer units.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_RNG_TAG 0x51505448u
#define OR_E_NONE INT64_MAX

/* ------------------------------------------------------------------------ */
/* Section II: the field.  Free cells are the waypoints, numbered row-major.  */
/* Returns C; fills the integer coordinates and the cell id of grid cell      */
/* `start` (-1 if it is not free).                                            */
int32_t or_cells(int32_t rows, int32_t cols, const uint8_t *free_mask,
                 int32_t start, int32_t *cell_r, int32_t *cell_c,
                 int32_t *start_cell) {
  int32_t C = 0;
  *start_cell = -1;
  for (int32_t r = 0; r < rows; ++r) {
    for (int32_t c = 0; c < cols; ++c) {
      int32_t g = r * cols + c;
      if (free_mask && !free_mask[g]) continue;
      if (g == start) *start_cell = C;
      cell_r[C] = r;
      cell_c[C] = c;
      ++C;
    }
  }
  return C;
}

/* Section II (t_ij = d_ij * tau, d Euclidean), reading R2: round(scale*sqrt(q))
 * without floating point.  With N = scale^2 q and r = floor(sqrt(N)), sqrt(N)
 * rounds up iff N >= r^2 + r + 1/4, i.e. iff N - r^2 > r.  A tie cannot occur
 * because N is an integer.                                                   */
int64_t or_round_scaled_sqrt(int64_t q, int64_t scale) {
  int64_t N = scale * scale * q;
  int64_t r = 0;
  /* integer square root by bisection: the largest r with r*r <= N */
  int64_t lo = 0, hi = 1;
  while (hi * hi <= N) hi *= 2;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) / 2;
    if (mid * mid <= N) lo = mid; else hi = mid - 1;
  }
  r = lo;
  return (N - r * r > r) ? r + 1 : r;
}

/* Section II, Algorithm 1 first step: the travel-cost matrix d (C x C). */
void or_distances(int32_t C, const int32_t *cell_r, const int32_t *cell_c,
                  int32_t scale, int32_t *d) {
  for (int32_t i = 0; i < C; ++i) {
    for (int32_t j = 0; j < C; ++j) {
      int64_t dr = cell_r[i] - cell_r[j];
      int64_t dc = cell_c[i] - cell_c[j];
      d[(int64_t)i * C + j] = (int32_t)or_round_scaled_sqrt(dr * dr + dc * dc, scale);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Eqs. 3-6 written out term by term, readings R3/R4.  x is C x C, t-major.   */
int64_t or_energy_terms(int32_t C, const int32_t *d, int32_t A, int32_t B,
                        const uint8_t *x, int64_t *h_dist, int64_t *h_visit,
                        int64_t *h_time) {
  int64_t hd = 0, hv = 0, ht = 0;
  /* Eq. 3: sum over consecutive steps of d_ij x_{t,i} x_{t+1,j} */
  for (int32_t t = 0; t + 1 < C; ++t)
    for (int32_t i = 0; i < C; ++i)
      for (int32_t j = 0; j < C; ++j)
        hd += (int64_t)d[(int64_t)i * C + j] * x[(int64_t)t * C + i] *
              x[(int64_t)(t + 1) * C + j];
  /* Eq. 4: every cell visited once */
  for (int32_t i = 0; i < C; ++i) {
    int64_t s = 0;
    for (int32_t t = 0; t < C; ++t) s += x[(int64_t)t * C + i];
    hv += (1 - s) * (1 - s);
  }
  /* Eq. 5: one cell per step */
  for (int32_t t = 0; t < C; ++t) {
    int64_t s = 0;
    for (int32_t i = 0; i < C; ++i) s += x[(int64_t)t * C + i];
    ht += (1 - s) * (1 - s);
  }
  if (h_dist) *h_dist = hd;
  if (h_visit) *h_visit = hv;
  if (h_time) *h_time = ht;
  /* Eq. 6 */
  return (int64_t)B * hd + (int64_t)A * (hv + ht);
}

/* Eq. 6 expanded into one symmetric matrix S (n = C^2) and a constant c0 such
 * that E(x) = sum_k S_kk x_k + sum_{k<l} S_kl x_k x_l + c0.  Expanding
 * (1 - sum x)^2 with x^2 = x gives 1 - sum x + 2 sum_{pairs} x_a x_b, so each
 * variable gets -2A on the diagonal (one row and one column penalty), each pair
 * sharing a row or a column gets +2A, consecutive-step pairs get B*d_ij, and
 * c0 = 2AC (C row penalties plus C column penalties).                         */
void or_dense_qubo(int32_t C, const int32_t *d, int32_t A, int32_t B,
                   int32_t *S, int64_t *c0) {
  int64_t n = (int64_t)C * C;
  memset(S, 0, sizeof(int32_t) * n * n);
  for (int32_t t = 0; t < C; ++t) {
    for (int32_t i = 0; i < C; ++i) {
      int64_t k = (int64_t)t * C + i;
      S[k * n + k] = -2 * A;
      for (int32_t u = 0; u < C; ++u) {
        for (int32_t j = 0; j < C; ++j) {
          int64_t l = (int64_t)u * C + j;
          if (l == k) continue;
          int32_t v = 0;
          if (u == t) v += 2 * A;            /* same step: Eq. 5 */
          if (j == i) v += 2 * A;            /* same cell: Eq. 4 */
          if (u == t + 1 || u == t - 1) v += B * d[(int64_t)i * C + j]; /* Eq. 3 */
          S[k * n + l] = v;
        }
      }
    }
  }
  *c0 = 2 * (int64_t)A * C;
}

/* R9: Eq. 6 with the distance term weighted per leg, w[t] on the leg from
 * step t to step t+1 (t = 0..C-2); the penalty terms as in Eqs. 4-5.        */
int64_t or_energy_terms_weighted(int32_t C, const int32_t *d, int32_t A, const int32_t *w,
                                 const uint8_t *x) {
  int64_t hd = 0, hv = 0, ht = 0;
  for (int32_t t = 0; t + 1 < C; ++t)
    for (int32_t i = 0; i < C; ++i)
      for (int32_t j = 0; j < C; ++j)
        hd += (int64_t)w[t] * d[(int64_t)i * C + j] * x[(int64_t)t * C + i] *
              x[(int64_t)(t + 1) * C + j];
  for (int32_t i = 0; i < C; ++i) {
    int64_t s = 0;
    for (int32_t t = 0; t < C; ++t) s += x[(int64_t)t * C + i];
    hv += (1 - s) * (1 - s);
  }
  for (int32_t t = 0; t < C; ++t) {
    int64_t s = 0;
    for (int32_t i = 0; i < C; ++i) s += x[(int64_t)t * C + i];
    ht += (1 - s) * (1 - s);
  }
  return hd + (int64_t)A * (hv + ht);
}

/* R9: the dense form of or_energy_terms_weighted, expanded as or_dense_qubo
 * expands Eq. 6: the pair of consecutive steps t, t+1 gets w[t] d_ij.        */
void or_dense_qubo_weighted(int32_t C, const int32_t *d, int32_t A, const int32_t *w,
                            int32_t *S, int64_t *c0) {
  int64_t n = (int64_t)C * C;
  memset(S, 0, sizeof(int32_t) * n * n);
  for (int32_t t = 0; t < C; ++t) {
    for (int32_t i = 0; i < C; ++i) {
      int64_t k = (int64_t)t * C + i;
      S[k * n + k] = -2 * A;
      for (int32_t u = 0; u < C; ++u) {
        for (int32_t j = 0; j < C; ++j) {
          int64_t l = (int64_t)u * C + j;
          if (l == k) continue;
          int32_t v = 0;
          if (u == t) v += 2 * A;
          if (j == i) v += 2 * A;
          if (u == t + 1) v += w[t] * d[(int64_t)i * C + j];
          if (u == t - 1) v += w[u] * d[(int64_t)i * C + j];
          S[k * n + l] = v;
        }
      }
    }
  }
  *c0 = 2 * (int64_t)A * C;
}

/* Energy of a generic QUBO in the convention above. */
int64_t or_energy_dense(int64_t n, const int32_t *S, int64_t c0, const uint8_t *x) {
  int64_t e = c0;
  for (int64_t k = 0; k < n; ++k) {
    if (!x[k]) continue;
    e += S[k * n + k];
    for (int64_t l = k + 1; l < n; ++l)
      if (x[l]) e += S[k * n + l];
  }
  return e;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32   */
/* S-box, each multiplying words 0 and 2 by the round constants and mixing the */
/* high halves with words 1, 3 and the key; the key is bumped by the Weyl      */
/* constants between rounds.                                                   */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* R7: the uniform 32-bit draw of variable k in sweep s of replica r. */
static uint32_t or_draw(uint64_t seed, int64_t k, int32_t s, int32_t r) {
  uint32_t ctr[4] = {(uint32_t)(k >> 2), (uint32_t)s, (uint32_t)r, OR_RNG_TAG};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  or_philox4x32_10(ctr, key, out);
  return out[k & 3];
}

/* ------------------------------------------------------------------------ */
/* R6: geometric schedule, one temperature per sweep. */
double or_temperature(int32_t n_sweeps, double T0, double T1, int32_t s) {
  if (n_sweeps <= 1) return T0;
  return T0 * pow(T1 / T0, (double)s / (double)(n_sweeps - 1));
}

/* R6: thr[dE] = floor(2^32 exp(-dE/T)) for dE = 1, 2, ... until the first zero.
 * Entry 0 is unused and set to 0xFFFFFFFF.  Returns len (the first dE whose
 * threshold is 0), or -1 if the table would not fit in `cap` entries; with
 * out == NULL only the length is computed.                                    */
int32_t or_thresholds(double T, uint32_t *out, int32_t cap) {
  if (out && cap > 0) out[0] = 0xFFFFFFFFu;
  for (int32_t de = 1;; ++de) {
    double p = exp(-(double)de / T);
    double v = floor(ldexp(p, 32));
    if (v <= 0.0) return de;
    if (de >= cap && out) return -1;
    if (out) out[de] = (uint32_t)v;
  }
}

/* The acceptance rule R6 for one proposal. */
static int or_accept(int64_t de, const uint32_t *thr, int32_t len, uint64_t seed,
                     int64_t k, int32_t s, int32_t r) {
  if (de <= 0) return 1;
  if (de >= len) return 0;
  return or_draw(seed, k, s, r) < thr[de];
}

/* ------------------------------------------------------------------------ */
/* The annealer.  One description covers both problem forms:
 *   structured: the path QUBO given by (C, d, A, B, start cell), n = C^2;
 *   dense:      a generic symmetric S (n x n) with constant c0, an optional
 *               frozen mask, and optionally the path structure C (C*C == n)
 *               used only for the feasibility test of R8.                    */
typedef struct {
  int32_t structured;
  int64_t n;
  /* structured */
  int32_t C, A, B, start_cell;
  const int32_t *d;
  /* dense */
  const int32_t *S;
  int64_t c0;
  const uint8_t *frozen;      /* may be NULL */
  const uint8_t *frozen_val;  /* may be NULL */
  /* schedule */
  int32_t n_sweeps, sweep_begin, sweep_end;
  double T0, T1;
  uint64_t seed;
  /* replicas: global indices */
  int32_t n_rep;
  const int32_t *rep_index;
  const uint8_t *init_states; /* n_rep x n or NULL */
  uint8_t *states_out;        /* n_rep x n */
  int64_t *energy_out;        /* n_rep */
  int64_t *best_out;          /* n_rep */
  int64_t *accepts_out;       /* n_rep, may be NULL */
  /* per-sweep threshold tables, built once */
  uint32_t **thr;
  int32_t *thr_len;
} or_job;

static int or_is_frozen(const or_job *J, int64_t k) {
  if (J->structured) {
    int32_t t = (int32_t)(k / J->C), i = (int32_t)(k % J->C);
    return t == 0 || i == J->start_cell;
  }
  return J->frozen ? J->frozen[k] != 0 : 0;
}

static uint8_t or_frozen_value(const or_job *J, int64_t k) {
  if (J->structured) {
    int32_t t = (int32_t)(k / J->C), i = (int32_t)(k % J->C);
    return (uint8_t)(t == 0 && i == J->start_cell);
  }
  return J->frozen_val ? J->frozen_val[k] : 0;
}

/* Per-replica state of the plain sweep: the spins, the row and column sums of
 * the one-hot grid, and for each row the list of its cells that are 1 (used to
 * add up the distance field; its order does not matter, sums are integers).  */
typedef struct {
  uint8_t *x;
  int32_t *rowsum, *colsum;
  int32_t *hot, *hot_n;   /* hot[t*C + m] = m-th cell with x_{t,i} = 1 */
  int64_t *hot_var;       /* dense: list of k with x_k = 1 */
  int64_t *hot_pos;       /* dense: position of k in hot_var, or -1 */
  int64_t hot_var_n;
} or_state;

static void or_hot_add(or_state *st, int32_t C, int32_t t, int32_t i) {
  st->hot[(int64_t)t * C + st->hot_n[t]] = i;
  st->hot_n[t] += 1;
}

static void or_hot_remove(or_state *st, int32_t C, int32_t t, int32_t i) {
  int32_t *row = st->hot + (int64_t)t * C;
  for (int32_t m = 0; m < st->hot_n[t]; ++m) {
    if (row[m] == i) {
      row[m] = row[st->hot_n[t] - 1];
      st->hot_n[t] -= 1;
      return;
    }
  }
}

/* Structured dE of flipping x_{t,i} (from Eq. 6 with readings R3/R4):
 *   dE = (1 - 2x) [ B sum_j d_ij (x_{t-1,j} + x_{t+1,j})
 *                   + A (2 r' - 1) + A (2 c' - 1) ]
 * where r', c' are the row-t and column-i sums without x_{t,i}.              */
static int64_t or_delta_structured(const or_job *J, const or_state *st,
                                   int32_t t, int32_t i) {
  int32_t C = J->C;
  int64_t x = st->x[(int64_t)t * C + i];
  int64_t nb = 0;
  for (int32_t dt = -1; dt <= 1; dt += 2) {
    int32_t u = t + dt;
    if (u < 0 || u >= C) continue;
    for (int32_t m = 0; m < st->hot_n[u]; ++m)
      nb += J->d[(int64_t)i * C + st->hot[(int64_t)u * C + m]];
  }
  int64_t rp = st->rowsum[t] - x;
  int64_t cp = st->colsum[i] - x;
  int64_t inner = (int64_t)J->B * nb + (int64_t)J->A * (2 * rp - 1) +
                  (int64_t)J->A * (2 * cp - 1);
  return (1 - 2 * x) * inner;
}

/* Dense dE of flipping x_k: (1 - 2x_k)(S_kk + sum_{l != k} S_kl x_l). */
static int64_t or_delta_dense(const or_job *J, const or_state *st, int64_t k) {
  int64_t n = J->n;
  int64_t h = J->S[k * n + k];
  for (int64_t m = 0; m < st->hot_var_n; ++m) {
    int64_t l = st->hot_var[m];
    if (l != k) h += J->S[k * n + l];
  }
  return (1 - 2 * (int64_t)st->x[k]) * h;
}

static void or_set(const or_job *J, or_state *st, int64_t k, uint8_t v) {
  if (st->x[k] == v) return;
  st->x[k] = v;
  int32_t dv = v ? 1 : -1;
  if (J->C > 0) {
    int32_t t = (int32_t)(k / J->C), i = (int32_t)(k % J->C);
    st->rowsum[t] += dv;
    st->colsum[i] += dv;
    if (J->structured) {
      if (v) or_hot_add(st, J->C, t, i); else or_hot_remove(st, J->C, t, i);
    }
  }
  if (!J->structured) {
    if (v) {
      st->hot_pos[k] = st->hot_var_n;
      st->hot_var[st->hot_var_n++] = k;
    } else {
      int64_t p = st->hot_pos[k];
      int64_t last = st->hot_var[--st->hot_var_n];
      st->hot_var[p] = last;
      st->hot_pos[last] = p;
      st->hot_pos[k] = -1;
    }
  }
}

static int or_feasible(const or_job *J, const or_state *st) {
  if (J->C <= 0) return 1;
  for (int32_t t = 0; t < J->C; ++t) if (st->rowsum[t] != 1) return 0;
  for (int32_t i = 0; i < J->C; ++i) if (st->colsum[i] != 1) return 0;
  return 1;
}

static int64_t or_energy_of(const or_job *J, const uint8_t *x) {
  if (J->structured) return or_energy_terms(J->C, J->d, J->A, J->B, x, 0, 0, 0);
  return or_energy_dense(J->n, J->S, J->c0, x);
}

static void or_run_replica(const or_job *J, int32_t rr, or_state *st) {
  int64_t n = J->n;
  int32_t r = J->rep_index[rr];
  int32_t C = J->C;
  memset(st->x, 0, (size_t)n);
  if (C > 0) {
    memset(st->rowsum, 0, sizeof(int32_t) * C);
    memset(st->colsum, 0, sizeof(int32_t) * C);
    memset(st->hot_n, 0, sizeof(int32_t) * C);
  }
  if (!J->structured) {
    st->hot_var_n = 0;
    for (int64_t k = 0; k < n; ++k) st->hot_pos[k] = -1;
  }
  /* initial state: zero or the given one, then the clamp / frozen values */
  for (int64_t k = 0; k < n; ++k) {
    uint8_t v = J->init_states ? (J->init_states[(int64_t)rr * n + k] != 0) : 0;
    if (or_is_frozen(J, k)) v = or_frozen_value(J, k);
    or_set(J, st, k, v);
  }
  int64_t E = or_energy_of(J, st->x);
  int64_t best = OR_E_NONE;
  int64_t accepts = 0;
  for (int32_t s = J->sweep_begin; s < J->sweep_end; ++s) {
    const uint32_t *thr = J->thr[s - J->sweep_begin];
    int32_t len = J->thr_len[s - J->sweep_begin];
    for (int64_t k = 0; k < n; ++k) {
      if (or_is_frozen(J, k)) continue;
      int64_t de = J->structured
                       ? or_delta_structured(J, st, (int32_t)(k / C), (int32_t)(k % C))
                       : or_delta_dense(J, st, k);
      if (or_accept(de, thr, len, J->seed, k, s, r)) {
        or_set(J, st, k, (uint8_t)(1 - st->x[k]));
        E += de;
        ++accepts;
      }
    }
    if (or_feasible(J, st) && E < best) best = E;
  }
  memcpy(J->states_out + (int64_t)rr * n, st->x, (size_t)n);
  J->energy_out[rr] = E;
  J->best_out[rr] = best;
  if (J->accepts_out) J->accepts_out[rr] = accepts;
}

typedef struct {
  const or_job *J;
  int32_t first, step;
  int status;
} or_worker;

static void *or_worker_main(void *arg) {
  or_worker *w = (or_worker *)arg;
  const or_job *J = w->J;
  int64_t n = J->n;
  int32_t C = J->C > 0 ? J->C : 1;
  or_state st;
  memset(&st, 0, sizeof st);
  st.x = (uint8_t *)malloc((size_t)n);
  st.rowsum = (int32_t *)malloc(sizeof(int32_t) * C);
  st.colsum = (int32_t *)malloc(sizeof(int32_t) * C);
  st.hot_n = (int32_t *)malloc(sizeof(int32_t) * C);
  st.hot = (int32_t *)malloc(sizeof(int32_t) * (size_t)C * C);
  if (!J->structured) {
    st.hot_var = (int64_t *)malloc(sizeof(int64_t) * n);
    st.hot_pos = (int64_t *)malloc(sizeof(int64_t) * n);
  }
  if (!st.x || !st.rowsum || !st.colsum || !st.hot_n || !st.hot ||
      (!J->structured && (!st.hot_var || !st.hot_pos))) {
    w->status = -2;
  } else {
    for (int32_t rr = w->first; rr < J->n_rep; rr += w->step) or_run_replica(J, rr, &st);
    w->status = 0;
  }
  free(st.x); free(st.rowsum); free(st.colsum); free(st.hot_n); free(st.hot);
  free(st.hot_var); free(st.hot_pos);
  return 0;
}

static int or_run_job(or_job *J, int32_t n_threads) {
  int32_t ns = J->sweep_end - J->sweep_begin;
  if (ns < 0 || J->sweep_begin < 0 || J->sweep_end > J->n_sweeps) return -1;
  J->thr = (uint32_t **)calloc((size_t)(ns > 0 ? ns : 1), sizeof(uint32_t *));
  J->thr_len = (int32_t *)calloc((size_t)(ns > 0 ? ns : 1), sizeof(int32_t));
  int rc = 0;
  for (int32_t s = 0; s < ns && rc == 0; ++s) {
    double T = or_temperature(J->n_sweeps, J->T0, J->T1, J->sweep_begin + s);
    int32_t len = or_thresholds(T, 0, 0);
    J->thr_len[s] = len;
    J->thr[s] = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)len);
    if (!J->thr[s]) rc = -2; else or_thresholds(T, J->thr[s], len);
  }
  if (rc == 0) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > J->n_rep) n_threads = J->n_rep > 0 ? J->n_rep : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    or_worker *ws = (or_worker *)malloc(sizeof(or_worker) * n_threads);
    for (int32_t i = 0; i < n_threads; ++i) {
      ws[i].J = J; ws[i].first = i; ws[i].step = n_threads; ws[i].status = 0;
      pthread_create(&th[i], 0, or_worker_main, &ws[i]);
    }
    for (int32_t i = 0; i < n_threads; ++i) {
      pthread_join(th[i], 0);
      if (ws[i].status) rc = ws[i].status;
    }
    free(th); free(ws);
  }
  for (int32_t s = 0; s < ns; ++s) free(J->thr[s]);
  free(J->thr); free(J->thr_len);
  return rc;
}

/* Anneal the path QUBO in its structured form (Eqs. 3-6, readings R1-R8).
 * Returns 0, -1 on bad arguments, -2 on allocation failure.                  */
int32_t or_anneal_structured(int32_t C, const int32_t *d, int32_t A, int32_t B,
                             int32_t start_cell, int32_t n_sweeps, double T0,
                             double T1, int32_t sweep_begin, int32_t sweep_end,
                             uint64_t seed, int32_t n_rep, const int32_t *rep_index,
                             const uint8_t *init_states, uint8_t *states_out,
                             int64_t *energy_out, int64_t *best_out,
                             int64_t *accepts_out, int32_t n_threads) {
  if (C < 1 || start_cell < 0 || start_cell >= C) return -1;
  or_job J;
  memset(&J, 0, sizeof J);
  J.structured = 1; J.n = (int64_t)C * C; J.C = C; J.A = A; J.B = B;
  J.start_cell = start_cell; J.d = d;
  J.n_sweeps = n_sweeps; J.T0 = T0; J.T1 = T1;
  J.sweep_begin = sweep_begin; J.sweep_end = sweep_end; J.seed = seed;
  J.n_rep = n_rep; J.rep_index = rep_index; J.init_states = init_states;
  J.states_out = states_out; J.energy_out = energy_out; J.best_out = best_out;
  J.accepts_out = accepts_out;
  return or_run_job(&J, n_threads);
}

/* Anneal a generic QUBO given as a dense symmetric S (n x n) and c0.  C > 0
 * (with C*C == n) marks the path structure, used only by the feasibility test
 * of the best energy.                                                         */
int32_t or_anneal_dense(int64_t n, const int32_t *S, int64_t c0, const uint8_t *frozen,
                        const uint8_t *frozen_val, int32_t C, int32_t n_sweeps,
                        double T0, double T1, int32_t sweep_begin, int32_t sweep_end,
                        uint64_t seed, int32_t n_rep, const int32_t *rep_index,
                        const uint8_t *init_states, uint8_t *states_out,
                        int64_t *energy_out, int64_t *best_out, int64_t *accepts_out,
                        int32_t n_threads) {
  if (n < 1 || (C > 0 && (int64_t)C * C != n)) return -1;
  or_job J;
  memset(&J, 0, sizeof J);
  J.structured = 0; J.n = n; J.C = C; J.S = S; J.c0 = c0;
  J.frozen = frozen; J.frozen_val = frozen_val;
  J.n_sweeps = n_sweeps; J.T0 = T0; J.T1 = T1;
  J.sweep_begin = sweep_begin; J.sweep_end = sweep_end; J.seed = seed;
  J.n_rep = n_rep; J.rep_index = rep_index; J.init_states = init_states;
  J.states_out = states_out; J.energy_out = energy_out; J.best_out = best_out;
  J.accepts_out = accepts_out;
  return or_run_job(&J, n_threads);
}

/* Section III-D / Algorithm 1 last step: read the flight path off a state.
 * path[t] = the cell flown at step t; the length is the sum of d over
 * consecutive steps.  Returns 0, or 1 if some row or column sum is not 1.    */
int32_t or_decode(int32_t C, const int32_t *d, const uint8_t *x, int32_t *path,
                  int64_t *length) {
  for (int32_t i = 0; i < C; ++i) {
    int32_t s = 0;
    for (int32_t t = 0; t < C; ++t) s += x[(int64_t)t * C + i];
    if (s != 1) return 1;
  }
  for (int32_t t = 0; t < C; ++t) {
    int32_t s = 0, at = -1;
    for (int32_t i = 0; i < C; ++i)
      if (x[(int64_t)t * C + i]) { ++s; at = i; }
    if (s != 1) return 1;
    path[t] = at;
  }
  int64_t L = 0;
  for (int32_t t = 0; t + 1 < C; ++t) L += d[(int64_t)path[t] * C + path[t + 1]];
  *length = L;
  return 0;
}

/* dE of flipping variable k of state x, through the same formulas the sweep
 * uses, with the sums and hot lists built from x.  structured != 0: the path
 * form (C, d, A, B); otherwise the dense form (n, S).  For the tests that pin
 * dE against E(flip) - E.                                                    */
int64_t or_delta_at(int32_t structured, int32_t C, const int32_t *d, int32_t A,
                    int32_t B, int64_t n, const int32_t *S, const uint8_t *x,
                    int64_t k) {
  or_job J;
  memset(&J, 0, sizeof J);
  J.structured = structured;
  J.C = structured ? C : 0;
  J.n = structured ? (int64_t)C * C : n;
  J.d = d; J.A = A; J.B = B; J.S = S;
  or_state st;
  memset(&st, 0, sizeof st);
  int32_t Cs = J.C > 0 ? J.C : 1;
  st.x = (uint8_t *)calloc((size_t)J.n, 1);
  st.rowsum = (int32_t *)calloc((size_t)Cs, sizeof(int32_t));
  st.colsum = (int32_t *)calloc((size_t)Cs, sizeof(int32_t));
  st.hot_n = (int32_t *)calloc((size_t)Cs, sizeof(int32_t));
  st.hot = (int32_t *)calloc((size_t)Cs * Cs, sizeof(int32_t));
  st.hot_var = (int64_t *)calloc((size_t)J.n, sizeof(int64_t));
  st.hot_pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)J.n);
  for (int64_t m = 0; m < J.n; ++m) st.hot_pos[m] = -1;
  for (int64_t m = 0; m < J.n; ++m) or_set(&J, &st, m, (uint8_t)(x[m] != 0));
  int64_t de = structured ? or_delta_structured(&J, &st, (int32_t)(k / C), (int32_t)(k % C))
                          : or_delta_dense(&J, &st, k);
  free(st.x); free(st.rowsum); free(st.colsum); free(st.hot_n); free(st.hot);
  free(st.hot_var); free(st.hot_pos);
  return de;
}
