// dense.cuh — per-replica search state shared by the dense-instance kernels
// (dense.cu, dense_tc.cu, dense_push.cu).
#pragma once

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
//   n <= 4096, a multiple of 4 (padded; n_eval = the instance's own spins,
//   for the work counters).
cudaError_t dense_push_run(int n, int n_eval, int R, int max_sweeps, int budget, const float *J, const float *h,
                           const float *F, __nv_bfloat16 *S, DenseRep *rep, int32_t *counter,
                           unsigned long long *stats, int sm_count, cudaStream_t s);

}  // namespace isg
