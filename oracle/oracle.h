/*
 * oracle.h — plain, slow, single-threaded CPU oracle for the local-search
 * method of García & Markov (arXiv:0912.3912).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or helper with the GPU library and never calls it.
 *
 * Every function follows a definition from the paper (cited per function) or a
 * textbook/published method named beside it.  Arithmetic is FP64 (or exact
 * integers) unless a function's mode asks for the FP32 mirror of the
 * library's documented float semantics.
 */
#ifndef ISING_ORACLE_H
#define ISING_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* An instance as the oracle sees it.  Couplings are passed as doubles (int8 and
 * float inputs convert exactly).  Either the CSR triple or J_dense is set.     */
typedef struct {
  int32_t n;
  const int64_t *row_ptr; /* [n+1] or NULL when J_dense is used */
  const int32_t *col;
  const double *J;
  const double *J_dense;  /* [n*n] row-major or NULL             */
  const double *h;        /* [n] or NULL                          */
  int32_t n_hyper;
  const int64_t *hyper_ptr;
  const int32_t *hyper_members;
  const double *hyper_J;
  const int32_t *colour;  /* [n] or NULL                          */
  int32_t is_int;         /* all couplings/fields integer-valued  */
  int32_t is_f64;         /* given as FP64 values (the library's ISING_F64):
                             passes stop at the first pass without strict
                             improvement, as for integer instances           */
} orc_instance;

enum { ORC_MODE_INT = 0, ORC_MODE_F64 = 1, ORC_MODE_F32 = 2 };
enum { ORC_SCHED_COLOUR = 0, ORC_SCHED_SEQUENTIAL = 1 };

typedef struct {
  int32_t max_sweeps, restarts, sweep_budget, refresh_every, schedule, mode;
} orc_params;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_random_start(int32_t n, uint64_t seed, uint32_t b, uint32_t r, uint32_t k, int8_t *s);

double orc_energy(const orc_instance *in, const int8_t *s);
int64_t orc_energy_int(const orc_instance *in, const int8_t *s);
void orc_local_fields(const orc_instance *in, const int8_t *s, double *f);
double orc_lower_bound(const orc_instance *in);

int32_t orc_greedy_colouring(const orc_instance *in, int32_t *colour);
int32_t orc_colouring_valid(const orc_instance *in, const int32_t *colour);

int32_t orc_descent(const orc_instance *in, uint64_t seed, uint32_t b, int32_t replicas,
                    const orc_params *p, int8_t *out_spins, double *out_E,
                    int32_t *out_minima, uint64_t *stats5);
int32_t orc_descent_from(const orc_instance *in, uint64_t seed, uint32_t b, int32_t first_replica,
                         int32_t replicas, const orc_params *p, int8_t *out_spins, double *out_E,
                         int32_t *out_minima, uint64_t *stats5);

double orc_fm_search(const orc_instance *in, int8_t *s, int32_t *passes);

double orc_bruteforce(const orc_instance *in, int8_t *argmin, int64_t *n_ground);
int32_t orc_bnb(const orc_instance *in, int64_t node_limit, double *E_out, int8_t *argmin,
                int64_t *nodes_out);
double orc_transfer_matrix(const orc_instance *in, int32_t rows, int32_t cols,
                           int32_t periodic_rows, int32_t periodic_cols, int32_t *ok);

#ifdef __cplusplus
}
#endif
#endif
