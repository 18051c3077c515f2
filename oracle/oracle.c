/*
 * oracle.c — plain CPU oracle for García & Markov, "High-performance Energy
 * Minimization in Spin-glasses" (arXiv:0912.3912).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the GPU library, which shares no code
 * with this file.  Single-threaded, unoptimised, written to be checked by eye
 * against the paper:
 *   energy ............ Sec. II Eq. 1, Sec. VI Eq. 6
 *   lower bound ....... Sec. III Eq. 2
 *   gains / descent ... Sec. IV (gain of a move; random starts; restarts)
 *   FM-style passes ... Sec. IV Fig. 3 with the heap of Fig. 4
 *   branch and bound .. Sec. III (Eqs. 2-4, Lemmas 1-2)
 * plus textbook tools: Gray-code enumeration, a row-by-row transfer-matrix
 * minimisation for grids, greedy graph colouring, and Philox4x32-10 (Salmon,
 * Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 as published (SC'11): 10 rounds of two 32x32->64 multiplies
 * with constants 0xD2511F53 and 0xCD9E8D57, Weyl key bumps 0x9E3779B9 and
 * 0xBB67AE85 between rounds.                                                 */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Random start (Sec. IV: a uniformly random configuration): spin i is +1 iff
 * bit (i mod 128) of Philox(key = seed halves, counter = (i/128, r, k, b)) is 1. */
void orc_random_start(int32_t n, uint64_t seed, uint32_t b, uint32_t r, uint32_t k, int8_t *s) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (int32_t w = 0; w * 128 < n; ++w) {
    uint32_t ctr[4] = {(uint32_t)w, r, k, b}, out[4];
    orc_philox4x32_10(ctr, key, out);
    for (int t = 0; t < 128 && w * 128 + t < n; ++t) {
      uint32_t bit = (out[t / 32] >> (t % 32)) & 1u;
      s[w * 128 + t] = bit ? 1 : -1;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Compensated (Neumaier) FP64 summation, so the oracle's energies carry an
 * error far below the 1e-6 relative bar even on million-spin instances.       */
typedef struct { double s, c; } ksum;
static void ks_add(ksum *k, double x) {
  double t = k->s + x;
  if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
  else k->c += (x - t) + k->s;
  k->s = t;
}
static double ks_get(const ksum *k) { return k->s + k->c; }

/* Neighbour iteration over either a CSR row or a dense row (j != i).          */
#define FOR_NBR(in, i, J_VAR, W_VAR, BODY)                                       \
  do {                                                                           \
    if ((in)->J_dense) {                                                         \
      for (int32_t J_VAR = 0; J_VAR < (in)->n; ++J_VAR) {                        \
        if (J_VAR == (i)) continue;                                              \
        double W_VAR = (in)->J_dense[(int64_t)(i) * (in)->n + J_VAR];            \
        BODY                                                                     \
      }                                                                          \
    } else {                                                                     \
      for (int64_t kk_ = (in)->row_ptr[i]; kk_ < (in)->row_ptr[(i) + 1]; ++kk_) { \
        int32_t J_VAR = (in)->col[kk_];                                          \
        double W_VAR = (in)->J[kk_];                                             \
        BODY                                                                     \
      }                                                                          \
    }                                                                            \
  } while (0)

static double hyper_prod(const orc_instance *in, int32_t e, const int8_t *s, int32_t skip) {
  double p = 1.0;
  for (int64_t q = in->hyper_ptr[e]; q < in->hyper_ptr[e + 1]; ++q) {
    int32_t m = in->hyper_members[q];
    if (m != skip) p *= (double)s[m];
  }
  return p;
}

/* Energy, Eq. 1 extended by the hyper-couplings of Eq. 6: every unordered pair
 * once (j > i), every hyper-edge once, every field once.                      */
double orc_energy(const orc_instance *in, const int8_t *s) {
  ksum acc = {0.0, 0.0};
  for (int32_t i = 0; i < in->n; ++i) {
    FOR_NBR(in, i, j, w, {
      if (j > i) ks_add(&acc, -w * (double)s[i] * (double)s[j]);
    });
    if (in->h) ks_add(&acc, -in->h[i] * (double)s[i]);
  }
  for (int32_t e = 0; e < in->n_hyper; ++e)
    ks_add(&acc, -in->hyper_J[e] * hyper_prod(in, e, s, -1));
  return ks_get(&acc);
}

int64_t orc_energy_int(const orc_instance *in, const int8_t *s) {
  int64_t E = 0;
  for (int32_t i = 0; i < in->n; ++i) {
    FOR_NBR(in, i, j, w, {
      if (j > i) E -= (int64_t)w * s[i] * s[j];
    });
    if (in->h) E -= (int64_t)in->h[i] * s[i];
  }
  for (int32_t e = 0; e < in->n_hyper; ++e)
    E -= (int64_t)in->hyper_J[e] * (int64_t)hyper_prod(in, e, s, -1);
  return E;
}

/* Local field f_i = h_i + sum_j J_ij s_j + sum_{e ∋ i} J_e prod_{k∈e\i} s_k,
 * so that flipping spin i changes E by 2 s_i f_i (Sec. IV, gain = -2 s_i f_i). */
void orc_local_fields(const orc_instance *in, const int8_t *s, double *f) {
  for (int32_t i = 0; i < in->n; ++i) {
    double acc = in->h ? in->h[i] : 0.0;
    FOR_NBR(in, i, j, w, { acc += w * (double)s[j]; });
    f[i] = acc;
  }
  for (int32_t e = 0; e < in->n_hyper; ++e)
    for (int64_t q = in->hyper_ptr[e]; q < in->hyper_ptr[e + 1]; ++q) {
      int32_t m = in->hyper_members[q];
      f[m] += in->hyper_J[e] * hyper_prod(in, e, s, m);
    }
}

/* Eq. 2: no configuration can do better than satisfying every term.          */
double orc_lower_bound(const orc_instance *in) {
  ksum acc = {0.0, 0.0};
  for (int32_t i = 0; i < in->n; ++i) {
    FOR_NBR(in, i, j, w, {
      if (j > i) ks_add(&acc, -fabs(w));
    });
    if (in->h) ks_add(&acc, -fabs(in->h[i]));
  }
  for (int32_t e = 0; e < in->n_hyper; ++e) ks_add(&acc, -fabs(in->hyper_J[e]));
  return ks_get(&acc);
}

/* ------------------------------------------------------------------------ */
/* Hyper-edge incidence: for each spin, the edges containing it, ascending.   */
typedef struct { int64_t *ptr; int32_t *edge; } incidence;

static int build_incidence(const orc_instance *in, incidence *inc) {
  int32_t n = in->n;
  inc->ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t total = in->n_hyper ? in->hyper_ptr[in->n_hyper] : 0;
  inc->edge = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  if (!inc->ptr || !inc->edge) return -1;
  for (int64_t q = 0; q < total; ++q) inc->ptr[in->hyper_members[q] + 1]++;
  for (int32_t i = 0; i < n; ++i) inc->ptr[i + 1] += inc->ptr[i];
  int64_t *fill = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  if (!fill) return -1;
  for (int32_t i = 0; i < n; ++i) fill[i] = inc->ptr[i];
  for (int32_t e = 0; e < in->n_hyper; ++e)
    for (int64_t q = in->hyper_ptr[e]; q < in->hyper_ptr[e + 1]; ++q)
      inc->edge[fill[in->hyper_members[q]]++] = e;
  free(fill);
  return 0;
}
static void free_incidence(incidence *inc) { free(inc->ptr); free(inc->edge); }

/* Greedy colouring of the conflict graph (CSR edges plus every pair inside a
 * hyper-edge), spins in index order, each taking the smallest colour no
 * earlier conflicting spin holds.  Returns the number of colours.            */
int32_t orc_greedy_colouring(const orc_instance *in, int32_t *colour) {
  int32_t n = in->n, ncol = 0;
  incidence inc;
  if (build_incidence(in, &inc)) return -1;
  char *used = (char *)calloc((size_t)n + 2, 1);
  for (int32_t i = 0; i < n; ++i) colour[i] = -1;
  for (int32_t i = 0; i < n; ++i) {
    memset(used, 0, (size_t)n + 2);
    FOR_NBR(in, i, j, w, {
      (void)w;
      if (colour[j] >= 0) used[colour[j]] = 1;
    });
    for (int64_t t = inc.ptr[i]; t < inc.ptr[i + 1]; ++t) {
      int32_t e = inc.edge[t];
      for (int64_t q = in->hyper_ptr[e]; q < in->hyper_ptr[e + 1]; ++q) {
        int32_t m = in->hyper_members[q];
        if (m != i && colour[m] >= 0) used[colour[m]] = 1;
      }
    }
    int32_t c = 0;
    while (used[c]) ++c;
    colour[i] = c;
    if (c + 1 > ncol) ncol = c + 1;
  }
  free(used);
  free_incidence(&inc);
  return ncol;
}

/* 1 iff no two conflicting spins share a colour and all colours are >= 0.    */
int32_t orc_colouring_valid(const orc_instance *in, const int32_t *colour) {
  for (int32_t i = 0; i < in->n; ++i) {
    if (colour[i] < 0) return 0;
    int bad = 0;
    FOR_NBR(in, i, j, w, {
      if (w != 0.0 || !in->J_dense)
        if (colour[j] == colour[i]) bad = 1;
    });
    if (bad) return 0;
  }
  for (int32_t e = 0; e < in->n_hyper; ++e)
    for (int64_t a = in->hyper_ptr[e]; a < in->hyper_ptr[e + 1]; ++a)
      for (int64_t c = a + 1; c < in->hyper_ptr[e + 1]; ++c)
        if (colour[in->hyper_members[a]] == colour[in->hyper_members[c]]) return 0;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Greedy single-spin-flip descent with restarts: the improving moves of the
 * paper's passes (Sec. IV: a move with positive gain lowers the energy), taken
 * spin by spin until no spin has a positive gain, restarted from independent
 * random starts and keeping the best result (Sec. IV, last paragraph before
 * Fig. 3).  Visit order: colour classes ascending and spins ascending inside a
 * class (a class is an independent set, so this equals deciding a whole class
 * at once), or plain index order for the sequential schedule.
 *
 * Modes: ORC_MODE_INT   exact integer fields recomputed at each visit;
 *        ORC_MODE_F64   FP64 fields recomputed at each visit;
 *        ORC_MODE_F32   the library's documented FP32 field semantics:
 *                       incremental updates at each visit from the neighbours
 *                       that flipped since this spin's previous visit (CSR
 *                       order, then hyper-edges ascending), and a from-scratch
 *                       FP64 recomputation rounded to FP32 at descent sweeps
 *                       d with d == 0 or d % refresh_every == 0.
 * stats5 accumulates {visits, flips, converged descents, descents, sweeps}.
 * orc_descent_from runs replicas first_replica .. first_replica + replicas - 1
 * (their random starts use those replica indices) and writes row r of the
 * outputs for replica first_replica + r; orc_descent starts at replica 0.    */
int32_t orc_descent_from(const orc_instance *in, uint64_t seed, uint32_t b, int32_t first_replica,
                         int32_t replicas, const orc_params *p, int8_t *out_spins, double *out_E,
                         int32_t *out_minima, uint64_t *stats5);

int32_t orc_descent(const orc_instance *in, uint64_t seed, uint32_t b, int32_t replicas,
                    const orc_params *p, int8_t *out_spins, double *out_E,
                    int32_t *out_minima, uint64_t *stats5) {
  return orc_descent_from(in, seed, b, 0, replicas, p, out_spins, out_E, out_minima, stats5);
}

int32_t orc_descent_from(const orc_instance *in, uint64_t seed, uint32_t b, int32_t first_replica,
                         int32_t replicas, const orc_params *p, int8_t *out_spins, double *out_E,
                         int32_t *out_minima, uint64_t *stats5) {
  int32_t n = in->n;
  if (n <= 0 || replicas <= 0 || first_replica < 0 || p->max_sweeps < 1 || p->restarts < 1) return -1;
  int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *colour = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int8_t *s = (int8_t *)malloc((size_t)n);
  int8_t *best = (int8_t *)malloc((size_t)n);
  float *f32 = (float *)malloc((size_t)n * sizeof(float));
  int64_t *vt = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *ft = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  incidence inc;
  if (!order || !colour || !s || !best || !f32 || !vt || !ft || build_incidence(in, &inc)) return -2;

  if (p->schedule == ORC_SCHED_SEQUENTIAL) {
    for (int32_t i = 0; i < n; ++i) order[i] = i;
  } else {
    if (in->colour) {
      memcpy(colour, in->colour, (size_t)n * sizeof(int32_t));
    } else if (orc_greedy_colouring(in, colour) < 0) {
      return -2;
    }
    if (!orc_colouring_valid(in, colour)) return -3;
    int32_t ncol = 0, pos = 0;
    for (int32_t i = 0; i < n; ++i) if (colour[i] + 1 > ncol) ncol = colour[i] + 1;
    for (int32_t c = 0; c < ncol; ++c)
      for (int32_t i = 0; i < n; ++i)
        if (colour[i] == c) order[pos++] = i;
  }

  for (int32_t r = 0; r < replicas; ++r) {
    int64_t total = 0;
    int have_best = 0, have_last = 0;
    double bestE = 0.0, lastE = 0.0;
    int32_t minima = 0;
    for (int32_t k = 0; k < p->restarts; ++k) {
      if (p->sweep_budget > 0 && total >= p->sweep_budget) break;
      orc_random_start(n, seed, b, (uint32_t)(first_replica + r), (uint32_t)k, s);
      stats5[3] += 1;
      for (int32_t i = 0; i < n; ++i) { vt[i] = -1; ft[i] = -2; }
      int64_t t = 0;
      int32_t d = 0;
      int converged = 0;
      for (;;) {
        if (p->sweep_budget > 0 && total >= p->sweep_budget) break;
        int refresh = (d == 0) || (p->refresh_every > 0 && d % p->refresh_every == 0);
        int64_t flips = 0;
        for (int32_t q = 0; q < n; ++q) {
          int32_t j = order[q];
          int flip;
          if (p->mode == ORC_MODE_INT) {
            int64_t fi = in->h ? (int64_t)in->h[j] : 0;
            FOR_NBR(in, j, i, w, { fi += (int64_t)w * s[i]; });
            for (int64_t u = inc.ptr[j]; u < inc.ptr[j + 1]; ++u) {
              int32_t e = inc.edge[u];
              fi += (int64_t)in->hyper_J[e] * (int64_t)hyper_prod(in, e, s, j);
            }
            flip = (int64_t)s[j] * fi < 0;
          } else if (p->mode == ORC_MODE_F64) {
            double fd = in->h ? in->h[j] : 0.0;
            FOR_NBR(in, j, i, w, { fd += w * (double)s[i]; });
            for (int64_t u = inc.ptr[j]; u < inc.ptr[j + 1]; ++u) {
              int32_t e = inc.edge[u];
              fd += in->hyper_J[e] * hyper_prod(in, e, s, j);
            }
            flip = (double)s[j] * fd < 0.0;
          } else {
            if (refresh) {
              double fd = in->h ? in->h[j] : 0.0;
              FOR_NBR(in, j, i, w, { fd += w * (double)s[i]; });
              for (int64_t u = inc.ptr[j]; u < inc.ptr[j + 1]; ++u) {
                int32_t e = inc.edge[u];
                fd += in->hyper_J[e] * hyper_prod(in, e, s, j);
              }
              f32[j] = (float)fd;
            } else {
              float fj = f32[j];
              FOR_NBR(in, j, i, w, {
                if (ft[i] > vt[j]) fj = fj + (float)(2.0 * w) * (float)s[i];
              });
              for (int64_t u = inc.ptr[j]; u < inc.ptr[j + 1]; ++u) {
                int32_t e = inc.edge[u];
                int parity = 0;
                for (int64_t q2 = in->hyper_ptr[e]; q2 < in->hyper_ptr[e + 1]; ++q2) {
                  int32_t m = in->hyper_members[q2];
                  if (m != j && ft[m] > vt[j]) parity ^= 1;
                }
                if (parity) fj = fj + (float)(2.0 * in->hyper_J[e]) * (float)hyper_prod(in, e, s, j);
              }
              f32[j] = fj;
            }
            flip = (float)s[j] * f32[j] < 0.0f;
          }
          vt[j] = t;
          if (flip) {
            s[j] = (int8_t)-s[j];
            ft[j] = t;
            ++flips;
          }
          ++t;
        }
        stats5[0] += (uint64_t)n;
        stats5[1] += (uint64_t)flips;
        stats5[4] += 1;
        ++d;
        ++total;
        if (flips == 0) { converged = 1; break; }
        if (d >= p->max_sweeps) break;
      }
      double E = orc_energy(in, s);
      if (converged) {
        ++minima;
        stats5[2] += 1;
        if (!have_best || E < bestE) {
          bestE = E;
          memcpy(best, s, (size_t)n);
          have_best = 1;
        }
      }
      lastE = E;
      have_last = 1;
      if (!have_best) memcpy(out_spins + (int64_t)r * n, s, (size_t)n);
    }
    if (have_best) {
      memcpy(out_spins + (int64_t)r * n, best, (size_t)n);
      out_E[r] = bestE;
    } else {
      out_E[r] = have_last ? lastE : 0.0;
    }
    if (out_minima) out_minima[r] = minima;
  }
  free(order); free(colour); free(s); free(best); free(f32); free(vt); free(ft);
  free_incidence(&inc);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Pass-based local search with hill-climbing (Sec. IV, Fig. 3), gains held in
 * a binary max-heap with a spin->slot index (Fig. 4).  Readings where the text
 * is silent: ties in gain go to the lowest spin index; a prefix is recorded
 * when the running energy drops strictly below the best seen in the pass (so
 * the earliest best prefix is kept); a new pass runs while the previous pass
 * lowered the energy strictly (for FP32 couplings, by more than 1e-9 relative,
 * so FP64 rounding of the running energy cannot fake an improvement; integer
 * and FP64 instances, whose energies both implementations form as the same
 * sequence of FP64 operations, take the strict rule as stated).
 * Starts from *s, leaves the result in *s and returns its energy.            */
typedef struct { int32_t *heap, *pos; double *key; int32_t size; } gheap;

static int gh_before(const gheap *H, int32_t a, int32_t b) {
  if (H->key[a] != H->key[b]) return H->key[a] > H->key[b];
  return a < b;
}
static void gh_swap(gheap *H, int32_t x, int32_t y) {
  int32_t a = H->heap[x], b = H->heap[y];
  H->heap[x] = b; H->heap[y] = a;
  H->pos[b] = x; H->pos[a] = y;
}
static void gh_up(gheap *H, int32_t x) {
  while (x > 0) {
    int32_t parent = (x - 1) / 2;
    if (!gh_before(H, H->heap[x], H->heap[parent])) break;
    gh_swap(H, x, parent);
    x = parent;
  }
}
static void gh_down(gheap *H, int32_t x) {
  for (;;) {
    int32_t l = 2 * x + 1, r = l + 1, m = x;
    if (l < H->size && gh_before(H, H->heap[l], H->heap[m])) m = l;
    if (r < H->size && gh_before(H, H->heap[r], H->heap[m])) m = r;
    if (m == x) break;
    gh_swap(H, x, m);
    x = m;
  }
}
static int32_t gh_pop(gheap *H) {
  int32_t top = H->heap[0];
  gh_swap(H, 0, H->size - 1);
  H->size--;
  H->pos[top] = -1;
  if (H->size > 0) gh_down(H, 0);
  return top;
}
static void gh_update(gheap *H, int32_t spin, double key) {
  if (H->pos[spin] < 0) return; /* locked */
  double old = H->key[spin];
  H->key[spin] = key;
  if (key > old || (key == old)) gh_up(H, H->pos[spin]);
  gh_down(H, H->pos[spin]);
}

double orc_fm_search(const orc_instance *in, int8_t *s, int32_t *passes) {
  int32_t n = in->n;
  incidence inc;
  if (build_incidence(in, &inc)) return NAN;
  double *f = (double *)malloc((size_t)n * sizeof(double));
  int32_t *moves = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  gheap H;
  H.heap = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  H.pos = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  H.key = (double *)malloc((size_t)n * sizeof(double));
  double Estar = orc_energy(in, s);
  int32_t npass = 0;
  for (;;) {
    ++npass;
    orc_local_fields(in, s, f); /* COMPUTE_GAINS: gain_i = -2 s_i f_i */
    H.size = n;
    for (int32_t i = 0; i < n; ++i) {
      H.heap[i] = i;
      H.pos[i] = i;
      H.key[i] = -2.0 * (double)s[i] * f[i];
    }
    for (int32_t x = n / 2 - 1; x >= 0; --x) gh_down(&H, x);
    double Ecur = Estar, Ebest = Estar;
    int32_t best_prefix = 0;
    for (int32_t step = 0; step < n; ++step) {
      int32_t i = gh_pop(&H);           /* SELECT_BEST_MOVE + LOCK_SPIN */
      Ecur -= H.key[i];                 /* APPLY_MOVE */
      s[i] = (int8_t)-s[i];
      moves[step] = i;
      FOR_NBR(in, i, j, w, {            /* UPDATE_GAINS of neighbours */
        f[j] += 2.0 * w * (double)s[i];
        gh_update(&H, j, -2.0 * (double)s[j] * f[j]);
      });
      for (int64_t u = inc.ptr[i]; u < inc.ptr[i + 1]; ++u) {
        int32_t e = inc.edge[u];
        for (int64_t q = in->hyper_ptr[e]; q < in->hyper_ptr[e + 1]; ++q) {
          int32_t m = in->hyper_members[q];
          if (m == i) continue;
          f[m] += 2.0 * in->hyper_J[e] * hyper_prod(in, e, s, m);
          gh_update(&H, m, -2.0 * (double)s[m] * f[m]);
        }
      }
      if (Ecur < Ebest) { Ebest = Ecur; best_prefix = step + 1; }
    }
    /* roll back to the best prefix of this pass (SP* := best-seen SP) */
    for (int32_t step = n - 1; step >= best_prefix; --step) s[moves[step]] = (int8_t)-s[moves[step]];
    double Enew = orc_energy(in, s);
    double margin = (in->is_int || in->is_f64) ? 0.0 : 1e-9 * (1.0 + fabs(Estar));
    if (Enew < Estar - margin) {
      Estar = Enew;
    } else {
      /* no strict improvement: this pass's start SP* is the result */
      for (int32_t step = best_prefix - 1; step >= 0; --step) s[moves[step]] = (int8_t)-s[moves[step]];
      break;
    }
  }
  free(f); free(moves); free(H.heap); free(H.pos); free(H.key);
  free_incidence(&inc);
  if (passes) *passes = npass;
  return orc_energy(in, s);
}

/* ------------------------------------------------------------------------ */
/* Exhaustive search in Gray-code order (textbook): one spin flips per step, so
 * the energy moves by 2 s_i f_i and only the flipped spin's neighbours' fields
 * change.  Returns the ground-state energy (recomputed from scratch for the
 * argmin), the argmin (first in Gray order), and for integer instances the
 * number of ground states.                                                   */
double orc_bruteforce(const orc_instance *in, int8_t *argmin, int64_t *n_ground) {
  int32_t n = in->n;
  if (n < 1 || n > 40) return NAN;
  incidence inc;
  if (build_incidence(in, &inc)) return NAN;
  int8_t *s = (int8_t *)malloc((size_t)n);
  double *f = (double *)malloc((size_t)n * sizeof(double));
  for (int32_t i = 0; i < n; ++i) s[i] = -1;
  orc_local_fields(in, s, f);
  double E = orc_energy(in, s), Emin = E;
  uint64_t tmin = 0, count = 1, steps = (uint64_t)1 << n;
  for (uint64_t t = 1; t < steps; ++t) {
    int32_t i = __builtin_ctzll(t);
    E += 2.0 * (double)s[i] * f[i];
    s[i] = (int8_t)-s[i];
    FOR_NBR(in, i, j, w, { f[j] += 2.0 * w * (double)s[i]; });
    for (int64_t u = inc.ptr[i]; u < inc.ptr[i + 1]; ++u) {
      int32_t e = inc.edge[u];
      for (int64_t q = in->hyper_ptr[e]; q < in->hyper_ptr[e + 1]; ++q) {
        int32_t m = in->hyper_members[q];
        if (m != i) f[m] += 2.0 * in->hyper_J[e] * hyper_prod(in, e, s, m);
      }
    }
    if (in->is_int) {
      if (E < Emin) { Emin = E; tmin = t; count = 1; }
      else if (E == Emin) ++count;
    } else if (E < Emin) {
      Emin = E; tmin = t;
    }
  }
  uint64_t g = tmin ^ (tmin >> 1);
  for (int32_t i = 0; i < n; ++i) argmin[i] = ((g >> i) & 1u) ? 1 : -1;
  free(s); free(f);
  free_incidence(&inc);
  if (n_ground) *n_ground = in->is_int ? (int64_t)count : -1;
  return orc_energy(in, argmin);
}

/* ------------------------------------------------------------------------ */
/* Branch and bound (Sec. III).  Spins are assigned in index order.  The bound
 * starts at Eq. 2 and, when a spin is assigned, every term that becomes fully
 * assigned moves from its best case -|w| to its actual value: +2|w| if it is
 * unsatisfied, 0 otherwise (Eqs. 3-4 with the sign of the printed Eq. 3 read
 * as "increase by twice the bond's magnitude"; a hyper-edge counts once all its
 * members are assigned).  Pruning: the bound reaching the incumbent, which
 * starts at a linear-time greedy solution; and dominance (Lemmas 1-2) applied
 * to single spins: if a spin whose neighbours are all assigned would lower the
 * energy by flipping, every completion is beaten by the flipped one.          */
typedef struct {
  const orc_instance *in;
  incidence inc;
  int32_t n;
  int8_t *s;
  int8_t *best;
  double inc_E, eps;
  int64_t nodes, limit;
  int aborted;
  /* per spin: CSR terms, fields and hyper-edges that close when it is assigned */
  int32_t *complete_at;        /* step at which spin's neighbourhood is fully assigned */
  int64_t *cptr; int32_t *clist; /* spins completing at each step                      */
  int32_t *hyper_last;         /* largest member of each hyper-edge                    */
} bnb_ctx;

static double bnb_increment(bnb_ctx *C, int32_t i) {
  const orc_instance *in = C->in;
  double inc = 0.0;
  FOR_NBR(in, i, j, w, {
    if (j < i && w * (double)C->s[i] * (double)C->s[j] < 0.0) inc += 2.0 * fabs(w);
  });
  if (in->h && in->h[i] * (double)C->s[i] < 0.0) inc += 2.0 * fabs(in->h[i]);
  for (int64_t u = C->inc.ptr[i]; u < C->inc.ptr[i + 1]; ++u) {
    int32_t e = C->inc.edge[u];
    if (C->hyper_last[e] == i && in->hyper_J[e] * hyper_prod(in, e, C->s, -1) < 0.0)
      inc += 2.0 * fabs(in->hyper_J[e]);
  }
  return inc;
}

static int bnb_dominated(bnb_ctx *C, int32_t step) {
  const orc_instance *in = C->in;
  for (int64_t t = C->cptr[step]; t < C->cptr[step + 1]; ++t) {
    int32_t m = C->clist[t];
    double fm = in->h ? in->h[m] : 0.0;
    FOR_NBR(in, m, j, w, { fm += w * (double)C->s[j]; });
    for (int64_t u = C->inc.ptr[m]; u < C->inc.ptr[m + 1]; ++u) {
      int32_t e = C->inc.edge[u];
      fm += in->hyper_J[e] * hyper_prod(in, e, C->s, m);
    }
    if ((double)C->s[m] * fm < -C->eps) return 1;
  }
  return 0;
}

static void bnb_rec(bnb_ctx *C, int32_t i, double lb) {
  if (C->aborted) return;
  if (++C->nodes > C->limit) { C->aborted = 1; return; }
  if (i == C->n) {
    if (lb < C->inc_E - C->eps) {
      C->inc_E = lb;
      memcpy(C->best, C->s, (size_t)C->n);
    }
    return;
  }
  double inc_v[2];
  int8_t vals[2] = {1, -1};
  for (int a = 0; a < 2; ++a) { C->s[i] = vals[a]; inc_v[a] = bnb_increment(C, i); }
  int first = inc_v[1] < inc_v[0] ? 1 : 0;
  for (int a = 0; a < 2; ++a) {
    int v = a == 0 ? first : 1 - first;
    C->s[i] = vals[v];
    double nlb = lb + inc_v[v];
    if (nlb >= C->inc_E + C->eps) continue;       /* bound pruning        */
    if (bnb_dominated(C, i)) continue;             /* Lemma 2 on one spin  */
    bnb_rec(C, i + 1, nlb);
    if (C->aborted) return;
  }
  C->s[i] = 0;
}

int32_t orc_bnb(const orc_instance *in, int64_t node_limit, double *E_out, int8_t *argmin,
                int64_t *nodes_out) {
  bnb_ctx C;
  memset(&C, 0, sizeof C);
  int32_t n = in->n;
  C.in = in;
  C.n = n;
  C.limit = node_limit;
  if (build_incidence(in, &C.inc)) return -1;
  C.s = (int8_t *)calloc((size_t)n, 1);
  C.best = (int8_t *)malloc((size_t)n);
  C.complete_at = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  C.cptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  C.clist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  C.hyper_last = (int32_t *)malloc((size_t)(in->n_hyper > 0 ? in->n_hyper : 1) * sizeof(int32_t));
  for (int32_t e = 0; e < in->n_hyper; ++e) {
    int32_t mx = -1;
    for (int64_t q = in->hyper_ptr[e]; q < in->hyper_ptr[e + 1]; ++q)
      if (in->hyper_members[q] > mx) mx = in->hyper_members[q];
    C.hyper_last[e] = mx;
  }
  for (int32_t m = 0; m < n; ++m) {
    int32_t mx = m;
    FOR_NBR(in, m, j, w, { (void)w; if (j > mx) mx = j; });
    for (int64_t u = C.inc.ptr[m]; u < C.inc.ptr[m + 1]; ++u) {
      int32_t e = C.inc.edge[u];
      if (C.hyper_last[e] > mx) mx = C.hyper_last[e];
    }
    C.complete_at[m] = mx;
    C.cptr[mx + 1]++;
  }
  for (int32_t i = 0; i < n; ++i) C.cptr[i + 1] += C.cptr[i];
  {
    int64_t *fill = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    for (int32_t i = 0; i < n; ++i) fill[i] = C.cptr[i];
    for (int32_t m = 0; m < n; ++m) C.clist[fill[C.complete_at[m]]++] = m;
    free(fill);
  }
  double lb0 = orc_lower_bound(in);
  C.eps = in->is_int ? 0.0 : 1e-9 * (1.0 + fabs(lb0));

  /* Linear-time greedy incumbent: each spin in index order takes the value with
   * the smaller bound increment, then single-flip descent to a local minimum. */
  {
    int8_t *g = C.s;
    for (int32_t i = 0; i < n; ++i) {
      g[i] = 1;
      double a = bnb_increment(&C, i);
      g[i] = -1;
      double b = bnb_increment(&C, i);
      g[i] = (b < a) ? -1 : 1;
    }
    double *f = (double *)malloc((size_t)n * sizeof(double));
    int changed = 1;
    while (changed) {
      changed = 0;
      for (int32_t i = 0; i < n; ++i) {
        orc_local_fields(in, g, f);
        if ((double)g[i] * f[i] < -C.eps) { g[i] = (int8_t)-g[i]; changed = 1; }
      }
    }
    free(f);
    memcpy(C.best, g, (size_t)n);
    C.inc_E = orc_energy(in, g);
    memset(C.s, 0, (size_t)n);
  }
  bnb_rec(&C, 0, lb0);
  int32_t done = C.aborted ? 0 : 1;
  if (E_out) *E_out = orc_energy(in, C.best);
  if (argmin) memcpy(argmin, C.best, (size_t)n);
  if (nodes_out) *nodes_out = C.nodes;
  free(C.s); free(C.best); free(C.complete_at); free(C.cptr); free(C.clist); free(C.hyper_last);
  free_incidence(&C.inc);
  return done;
}

/* ------------------------------------------------------------------------ */
/* Exact ground-state energy of a grid instance by row-by-row dynamic
 * programming over row configurations (the min-plus transfer-matrix method).
 * Spin (r, c) has index r*cols + c.  Every CSR edge must join horizontal or
 * vertical grid neighbours (with wrap-around where periodic); no hyper-edges.
 * Periodic rows are handled by fixing the first row's configuration.         */
static double lookup_J(const orc_instance *in, int32_t i, int32_t j, int *found) {
  for (int64_t k = in->row_ptr[i]; k < in->row_ptr[i + 1]; ++k)
    if (in->col[k] == j) { *found = 1; return in->J[k]; }
  *found = 0;
  return 0.0;
}

double orc_transfer_matrix(const orc_instance *in, int32_t rows, int32_t cols,
                           int32_t periodic_rows, int32_t periodic_cols, int32_t *ok) {
  *ok = 0;
  if (in->J_dense || in->n_hyper > 0 || rows * cols != in->n || cols < 1 || cols > 12) return NAN;
  if ((periodic_cols && cols < 3) || (periodic_rows && rows < 3)) return NAN;
  if (periodic_rows && cols > 8) return NAN;
  int32_t n = in->n;
  double *Jh = (double *)calloc((size_t)n, sizeof(double));
  double *Jv = (double *)calloc((size_t)n, sizeof(double));
  int64_t grid_edges = 0;
  for (int32_t r = 0; r < rows; ++r)
    for (int32_t c = 0; c < cols; ++c) {
      int32_t i = r * cols + c, found;
      if (c + 1 < cols || periodic_cols) {
        Jh[i] = lookup_J(in, i, r * cols + (c + 1) % cols, &found);
        grid_edges += found;
      }
      if (r + 1 < rows || periodic_rows) {
        Jv[i] = lookup_J(in, i, ((r + 1) % rows) * cols + c, &found);
        grid_edges += found;
      }
    }
  if (2 * grid_edges != in->row_ptr[n]) { free(Jh); free(Jv); return NAN; }
  int32_t S = 1 << cols;
  double *rowc = (double *)malloc((size_t)S * sizeof(double));
  double *D = (double *)malloc((size_t)S * sizeof(double));
  double *Dn = (double *)malloc((size_t)S * sizeof(double));
#define SPIN(x, c) ((((x) >> (c)) & 1) ? 1.0 : -1.0)
  double best_total = INFINITY;
  int32_t n_first = periodic_rows ? S : 1;
  for (int32_t x0 = 0; x0 < n_first; ++x0) {
    for (int32_t r = 0; r < rows; ++r) {
      for (int32_t x = 0; x < S; ++x) {
        double e = 0.0;
        for (int32_t c = 0; c < cols; ++c) {
          int32_t i = r * cols + c;
          if (c + 1 < cols || periodic_cols) e -= Jh[i] * SPIN(x, c) * SPIN(x, (c + 1) % cols);
          if (in->h) e -= in->h[i] * SPIN(x, c);
        }
        rowc[x] = e;
      }
      if (r == 0) {
        for (int32_t x = 0; x < S; ++x)
          D[x] = (!periodic_rows || x == x0) ? rowc[x] : INFINITY;
        continue;
      }
      for (int32_t y = 0; y < S; ++y) {
        double m = INFINITY;
        for (int32_t x = 0; x < S; ++x) {
          if (D[x] == INFINITY) continue;
          double tcost = 0.0;
          for (int32_t c = 0; c < cols; ++c)
            tcost -= Jv[(r - 1) * cols + c] * SPIN(x, c) * SPIN(y, c);
          if (D[x] + tcost < m) m = D[x] + tcost;
        }
        Dn[y] = m + rowc[y];
      }
      memcpy(D, Dn, (size_t)S * sizeof(double));
    }
    for (int32_t y = 0; y < S; ++y) {
      double tot = D[y];
      if (periodic_rows) {
        if (tot == INFINITY) continue;
        for (int32_t c = 0; c < cols; ++c)
          tot -= Jv[(rows - 1) * cols + c] * SPIN(y, c) * SPIN(x0, c);
      }
      if (tot < best_total) best_total = tot;
    }
  }
#undef SPIN
  free(Jh); free(Jv); free(rowc); free(D); free(Dn);
  *ok = 1;
  return best_total;
}
