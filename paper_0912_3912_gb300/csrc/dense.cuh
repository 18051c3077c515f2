// dense.cuh — per-replica search state shared by the dense-instance kernels
// (dense.cu, dense_tc.cu, dense_push.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace isg {

// One replica of a dense search.  A round is one descent of every replica that
// is not finished: `round` marks the replicas taking part in the current one.
struct DenseRep {
  int32_t active;   // descent in progress
  int32_t conv;     // the descent just ended in a 1-flip minimum
  int32_t total;    // sweeps over all descents (the sweep budget counts these)
  int32_t minima;   // converged descents
  int32_t d;        // sweeps of the current descent
  int32_t k;        // restart index of the current descent
  int32_t flips;    // flips of the sweep in progress (block comparator)
  int32_t round;    // takes part in the current round
  double best;      // lowest energy of a converged descent
  double E;         // energy of the current state, as the search computes it
};

// Replicas of a dense instance that leave the tensor-core sweeps still
// descending are continued by dense_push_run: one CTA per replica, fields in
// registers, one coupling-row update per flip.
//   J [n][n] FP32, h [n] FP32 (zeros allowed), F [R][n] fields (h included),
//   S [Rp][n] BF16 spins (rows of the replicas it finishes are rewritten);
//   n <= 16384, a multiple of 4 (padded; n_eval = the instance's own spins,
//   for the work counters).
cudaError_t dense_push_run(int n, int n_eval, int R, int max_sweeps, int budget, const float *J, const float *h,
                           const float *F, __nv_bfloat16 *S, DenseRep *rep, int32_t *counter,
                           unsigned long long *stats, int sm_count, cudaStream_t s);

// A 2-D BF16 tensor map (row-major, `inner` elements per row, `outer` rows)
// for TMA tile loads of box_inner x box_outer with 128-byte swizzling.
cudaError_t tc_encode_2d(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                         uint32_t box_outer);

// Exact energies (Eq. 1, each pair once, up to the quantisation of J to 32-bit
// fixed point) of R returned dense-instance states on tensor cores
// (dense_energy.cu).  dense_planes_build writes the four BF16 digit planes of
// J [np][np] (np a multiple of 128) to P [4][np][np] and their band copies to
// U [4][np][128], and the scale exponent to *F (synchronises the stream).
// dense_energy_run: spins int8 [R][n]; h [np] FP32 (zero padded); S BF16
// scratch [Rp][np], pint / ph scratch [np/128][Rp] with Rp = R rounded up to
// 128; E FP64 [R] out; error set to ISING_ERR_TIMEOUT when a bounded wait
// gives up.  Adds its kernel launches to *launches.
cudaError_t dense_planes_build(const float *J, int np, __nv_bfloat16 *P, __nv_bfloat16 *U, int *F, int sm_count,
                               cudaStream_t s);
cudaError_t dense_energy_run(const int8_t *spins, int n, int np, int R, const float *h, const __nv_bfloat16 *P,
                             const __nv_bfloat16 *U, int F, __nv_bfloat16 *S, long long *pint, double *ph,
                             double *E, int32_t *error, int sm_count, int *launches, cudaStream_t s);

}  // namespace isg
