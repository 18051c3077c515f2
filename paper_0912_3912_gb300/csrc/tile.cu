// tile.cu — persistent tile kernels: one CTA works on one (instance,
// 32-replica group) tile at a time, pulled from a work queue, with the
// instance's spins bit-packed in shared memory (bit r of word i = replica r of
// spin i is +1).
//
// Method (García & Markov, Sec. IV): single-spin moves taken when their gain
// -2 s_i f_i is positive, whole sweeps repeated until no move is taken (a 1-flip
// local minimum), independent random starts, the best result kept.  Colour
// classes are independent sets, so all spins of a class decide at once.
//
// Three evaluators share the sweep/restart machinery:
//   MODE 0  integer couplings, one warp per spin, lane = replica, exact int32
//           fields recomputed from the neighbours' bits at each visit;
//   MODE 1  FP32 couplings, one warp per spin, lane = replica, FP32 fields kept
//           per (spin, replica) and updated at each visit from the neighbours
//           that flipped since the previous visit (the paper's incremental gain
//           update), with an FP64 from-scratch refresh at descent sweeps
//           d % refresh == 0 (always d == 0);
//   MODE 2  multi-spin coding for J in {-1,+1}, h in {-1,0,+1}: one thread per
//           spin evaluates all 32 replicas with bitwise logic (unsatisfied-bond
//           masks counted in a bit-sliced adder, compared with the per-field
//           thresholds).
// Replicas of a tile run their descents in lockstep rounds: descent k of every
// lane starts together; a lane whose descent ended waits (masked) until the
// round ends.  Each replica's own sequence of states is exactly the one its
// C-ABI semantics define.
#include <cfloat>

#include "device_common.cuh"

namespace isg {

namespace {

// Energy of replica lane r of the tile (Eq. 1 + Eq. 6), FP64 (exact for
// integer couplings), summed over the whole block in a fixed order.
template <bool FLOAT>
__device__ double tile_lane_energy(const DevGraph &G, const InstDesc &I, const uint32_t *sw, int r,
                                   double *redd, long long *redi) {
  const int n = I.n;
  if (FLOAT) {
    const float *Jf = reinterpret_cast<const float *>(G.J);
    const float *hf = reinterpret_cast<const float *>(G.h);
    const float *hJ = reinterpret_cast<const float *>(G.hJ);
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int64_t gi = I.spin_off + i;
      const double si = ((sw[i] >> r) & 1u) ? 1.0 : -1.0;
      double e = (double)__ldg(hf + gi) * si;
      for (uint32_t k = __ldg(G.row + gi), ke = __ldg(G.row + gi + 1); k < ke; ++k) {
        const int j = __ldg(G.col + k);
        if (j > i) e += (double)__ldg(Jf + k) * si * (((sw[j] >> r) & 1u) ? 1.0 : -1.0);
      }
      acc -= e;
    }
    for (int e = threadIdx.x; e < I.n_hyper; e += blockDim.x) {
      const int64_t ge = I.hyper_off + e;
      uint32_t neg = 0;
      for (uint32_t q = __ldg(G.hptr + ge), qe = __ldg(G.hptr + ge + 1); q < qe; ++q)
        neg ^= ~(sw[__ldg(G.hmem + q)] >> r) & 1u;
      const double p = neg ? -1.0 : 1.0;
      acc -= (double)__ldg(hJ + ge) * p;
    }
    return block_sum(acc, redd);
  } else {
    const int8_t *Ji = reinterpret_cast<const int8_t *>(G.J);
    const int8_t *hi = reinterpret_cast<const int8_t *>(G.h);
    const int8_t *hJ = reinterpret_cast<const int8_t *>(G.hJ);
    long long acc = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int64_t gi = I.spin_off + i;
      const uint32_t bi = (sw[i] >> r) & 1u;
      int e = bi ? (int)__ldg(hi + gi) : -(int)__ldg(hi + gi);
      for (uint32_t k = __ldg(G.row + gi), ke = __ldg(G.row + gi + 1); k < ke; ++k) {
        const int j = __ldg(G.col + k);
        if (j > i) {
          const int w = __ldg(Ji + k);
          e += ((((sw[j] >> r) & 1u) ^ bi) ? -w : w);
        }
      }
      acc -= e;
    }
    for (int e = threadIdx.x; e < I.n_hyper; e += blockDim.x) {
      const int64_t ge = I.hyper_off + e;
      uint32_t neg = 0;
      for (uint32_t q = __ldg(G.hptr + ge), qe = __ldg(G.hptr + ge + 1); q < qe; ++q)
        neg ^= ~(sw[__ldg(G.hmem + q)] >> r) & 1u;
      const int w = __ldg(hJ + ge);
      acc -= neg ? -w : w;
    }
    return (double)block_sum(acc, redi);
  }
}

// u >= t for a bit-sliced 4-bit count (c0 least significant), t a per-thread value.
__device__ __forceinline__ uint32_t sliced_ge(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              int t) {
  if (t <= 0) return 0xffffffffu;
  if (t > 15) return 0u;
  uint32_t gt = 0, eq = 0xffffffffu;
  const uint32_t c[4] = {c0, c1, c2, c3};
#pragma unroll
  for (int p = 3; p >= 0; --p) {
    const uint32_t tb = ((t >> p) & 1) ? 0xffffffffu : 0u;
    gt |= eq & c[p] & ~tb;
    eq &= ~(c[p] ^ tb);
  }
  return gt | eq;
}

}  // namespace

template <int MODE>
__global__ void __launch_bounds__(kTileThreads, 1) tile_kernel(const TileArgs *__restrict__ Aptr) {
  extern __shared__ uint32_t smem[];
  __shared__ int s_tile;
  __shared__ uint32_t s_any, s_active, s_conv, s_upd;
  __shared__ int32_t s_total[32], s_minima[32];
  __shared__ double s_best[32];
  __shared__ double s_redd[32];
  __shared__ long long s_redi[32];

  const TileArgs &A = *Aptr;
  const DevGraph G = A.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int nmax = A.nmax;
  uint32_t *sw = smem;
  uint32_t *fm = smem + nmax;
  uint32_t *bw = A.bw + (size_t)blockIdx.x * nmax;
  float *F = A.F ? A.F + (size_t)blockIdx.x * nmax * 32 : nullptr;
  unsigned long long my_flips = 0, my_evals = 0, my_sweeps = 0, my_minima = 0, my_desc = 0;

  for (;;) {
    if (tid == 0) s_tile = atomicAdd(A.queue, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= A.n_tiles) break;
    const int b = A.tiles[t].x, g = A.tiles[t].y;
    const InstDesc I = G.inst[b];
    const int n = I.n;
    const int rem = A.R - 32 * g;
    const uint32_t lane_valid = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    const uint64_t seed = A.seeds[b];
    const int ncls = A.sequential ? n : I.ncls;
    if (tid < 32) {
      s_total[tid] = 0;
      s_minima[tid] = 0;
      s_best[tid] = DBL_MAX;
    }
    __syncthreads();

    for (int k = 0;; ++k) {
      if (tid == 0) {
        uint32_t start = 0;
        if (k < A.restarts)
          for (int r = 0; r < 32; ++r)
            if (((lane_valid >> r) & 1u) && (A.budget <= 0 || s_total[r] < A.budget)) start |= 1u << r;
        s_active = start;
        my_desc += __popc(start);
      }
      __syncthreads();
      uint32_t active = s_active;
      if (!active) break;

      // Random starts for the lanes beginning descent k (Sec. IV); a warp
      // transposes 32 replicas x 128 spins with ballots.
      for (int w = warp; w * 128 < n; w += nwarps) {
        const uint4 x = start_bits(seed, (uint32_t)w, (uint32_t)(32 * g + lane), (uint32_t)k, (uint32_t)b);
        for (int q = 0; q < 4; ++q) {
          const uint32_t xw = word_of(x, q);
          for (int u = 0; u < 32; ++u) {
            const int i = w * 128 + q * 32 + u;
            if (i >= n) break;
            const uint32_t m = __ballot_sync(0xffffffffu, (xw >> u) & 1u);
            if (lane == 0) {
              sw[i] = (sw[i] & ~active) | (m & active);
              if (MODE == 1) fm[i] &= ~active;
            }
          }
        }
      }
      __syncthreads();

      for (int d = 0; active; ++d) {
        const bool refresh = (d == 0) || (A.refresh > 0 && d % A.refresh == 0);
        if (tid == 0) s_any = 0;
        uint32_t anyf = 0;
        for (int c = 0; c < ncls; ++c) {
          int c0, c1;
          if (A.sequential) {
            c0 = c;
            c1 = c + 1;
          } else {
            c0 = __ldg(G.cls + I.cls_off + c);
            c1 = __ldg(G.cls + I.cls_off + c + 1);
          }
          if (MODE == 2) {
            const int8_t *Ji = reinterpret_cast<const int8_t *>(G.J);
            const int8_t *hi = reinterpret_cast<const int8_t *>(G.h);
            for (int v = c0 + tid; v < c1; v += blockDim.x) {
              const int j = A.sequential ? v : __ldg(G.order + I.spin_off + v);
              const int64_t gj = I.spin_off + j;
              const uint32_t wj = sw[j];
              uint32_t c0b = 0, c1b = 0, c2b = 0, c3b = 0;
              const uint32_t k0 = __ldg(G.row + gj), k1 = __ldg(G.row + gj + 1);
              for (uint32_t kk = k0; kk < k1; ++kk) {
                const int i = __ldg(G.col + kk);
                const uint32_t neg = __ldg(Ji + kk) < 0 ? 0xffffffffu : 0u;
                uint32_t x = wj ^ sw[i] ^ neg;  // unsatisfied bond
                uint32_t cy = c0b & x;
                c0b ^= x;
                x = cy;
                cy = c1b & x;
                c1b ^= x;
                x = cy;
                cy = c2b & x;
                c2b ^= x;
                c3b ^= cy;
              }
              const int deg = (int)(k1 - k0);
              const int hv = __ldg(hi + gj);
              // flip iff 2u > deg + h s  (dE = 2 s f < 0 with |J| = 1)
              uint32_t flip;
              if (hv == 0) {
                flip = sliced_ge(c0b, c1b, c2b, c3b, deg / 2 + 1);
              } else {
                const uint32_t plus = hv > 0 ? wj : ~wj;  // lanes with h s = +1
                const int tp = (deg + 1) / 2 + 1;
                const int tm = deg >= 1 ? (deg - 1) / 2 + 1 : 0;
                flip = (sliced_ge(c0b, c1b, c2b, c3b, tp) & plus) |
                       (sliced_ge(c0b, c1b, c2b, c3b, tm) & ~plus);
              }
              flip &= active;
              sw[j] = wj ^ flip;
              anyf |= flip;
              my_flips += __popc(flip);
            }
          } else {
            for (int v = c0 + warp; v < c1; v += nwarps) {
              const int j = A.sequential ? v : __ldg(G.order + I.spin_off + v);
              const int64_t gj = I.spin_off + j;
              const uint32_t wj = sw[j];
              const bool up = (wj >> lane) & 1u;
              const uint32_t k0 = __ldg(G.row + gj), k1 = __ldg(G.row + gj + 1);
              const uint32_t e0 = __ldg(G.inc_ptr + gj), e1 = __ldg(G.inc_ptr + gj + 1);
              bool flip;
              if (MODE == 0) {
                const int8_t *Ji = reinterpret_cast<const int8_t *>(G.J);
                const int8_t *hJ = reinterpret_cast<const int8_t *>(G.hJ);
                int f = __ldg(reinterpret_cast<const int8_t *>(G.h) + gj);
                for (uint32_t kk = k0; kk < k1; ++kk) {
                  const int i = __ldg(G.col + kk);
                  const int w = __ldg(Ji + kk);
                  f += ((sw[i] >> lane) & 1u) ? w : -w;
                }
                for (uint32_t q = e0; q < e1; ++q) {
                  const int e = __ldg(G.inc_edge + q);
                  uint32_t neg = 0;
                  for (uint32_t m = __ldg(G.hptr + e), me = __ldg(G.hptr + e + 1); m < me; ++m) {
                    const int mm = __ldg(G.hmem + m);
                    if (mm != j) neg ^= ~(sw[mm] >> lane) & 1u;
                  }
                  const int w = __ldg(hJ + e);
                  f += neg ? -w : w;
                }
                flip = up ? (f < 0) : (f > 0);
              } else {
                const float *Jf = reinterpret_cast<const float *>(G.J);
                const float *hJ = reinterpret_cast<const float *>(G.hJ);
                float f;
                if (refresh) {
                  double acc = (double)__ldg(reinterpret_cast<const float *>(G.h) + gj);
                  for (uint32_t kk = k0; kk < k1; ++kk) {
                    const int i = __ldg(G.col + kk);
                    const double w = (double)__ldg(Jf + kk);
                    acc = __dadd_rn(acc, ((sw[i] >> lane) & 1u) ? w : -w);
                  }
                  for (uint32_t q = e0; q < e1; ++q) {
                    const int e = __ldg(G.inc_edge + q);
                    uint32_t neg = 0;
                    for (uint32_t m = __ldg(G.hptr + e), me = __ldg(G.hptr + e + 1); m < me; ++m) {
                      const int mm = __ldg(G.hmem + m);
                      if (mm != j) neg ^= ~(sw[mm] >> lane) & 1u;
                    }
                    const double w = (double)__ldg(hJ + e);
                    acc = __dadd_rn(acc, neg ? -w : w);
                  }
                  f = __double2float_rn(acc);
                } else {
                  f = F[(size_t)j * 32 + lane];
                  for (uint32_t kk = k0; kk < k1; ++kk) {
                    const int i = __ldg(G.col + kk);
                    if ((fm[i] >> lane) & 1u) {
                      const float w2 = 2.0f * __ldg(Jf + kk);
                      f = __fadd_rn(f, ((sw[i] >> lane) & 1u) ? w2 : -w2);
                    }
                  }
                  for (uint32_t q = e0; q < e1; ++q) {
                    const int e = __ldg(G.inc_edge + q);
                    uint32_t neg = 0, par = 0;
                    for (uint32_t m = __ldg(G.hptr + e), me = __ldg(G.hptr + e + 1); m < me; ++m) {
                      const int mm = __ldg(G.hmem + m);
                      if (mm != j) {
                        neg ^= ~(sw[mm] >> lane) & 1u;
                        par ^= (fm[mm] >> lane) & 1u;
                      }
                    }
                    if (par) {
                      const float w2 = 2.0f * __ldg(hJ + e);
                      f = __fadd_rn(f, neg ? -w2 : w2);
                    }
                  }
                }
                F[(size_t)j * 32 + lane] = f;
                flip = up ? (f < 0.0f) : (f > 0.0f);
              }
              flip = flip && ((active >> lane) & 1u);
              const uint32_t m = __ballot_sync(0xffffffffu, flip);
              if (lane == 0) {
                sw[j] = wj ^ m;
                if (MODE == 1) fm[j] = m;
              }
              anyf |= m;
              my_flips += flip ? 1 : 0;
            }
          }
          __syncthreads();
        }
        // end of sweep: which lanes flipped at all?
        anyf = __reduce_or_sync(0xffffffffu, anyf);
        if (lane == 0 && anyf) atomicOr(&s_any, anyf);
        __syncthreads();
        if (tid == 0) {
          const uint32_t any = s_any;
          uint32_t ended = 0;
          for (int r = 0; r < 32; ++r)
            if ((active >> r) & 1u) s_total[r] += 1;
          const uint32_t conv = active & ~any;
          ended |= conv;
          if (d + 1 >= A.max_sweeps) ended |= active;
          if (A.budget > 0)
            for (int r = 0; r < 32; ++r)
              if (((active >> r) & 1u) && s_total[r] >= A.budget) ended |= 1u << r;
          my_sweeps += __popc(active);
          my_evals += (unsigned long long)__popc(active) * (unsigned long long)n;
          my_minima += __popc(conv);
          s_conv = conv;
          s_upd = 0;
          s_active = active & ~ended;
        }
        __syncthreads();
        uint32_t conv = s_conv;
        while (conv) {
          const int r = __ffs(conv) - 1;
          conv &= conv - 1;
          const double E = tile_lane_energy<MODE == 1>(G, I, sw, r, s_redd, s_redi);
          if (tid == 0) {
            s_minima[r] += 1;
            if (E < s_best[r]) {
              s_best[r] = E;
              s_upd |= 1u << r;
            }
          }
        }
        __syncthreads();
        const uint32_t upd = s_upd;
        if (upd)
          for (int i = tid; i < n; i += blockDim.x) bw[i] = (bw[i] & ~upd) | (sw[i] & upd);
        active = s_active;
        __syncthreads();
      }
    }

    // Result per lane: best converged state, else the final state of its last descent.
    uint32_t has_best = 0;
    for (int r = 0; r < 32; ++r)
      if (s_minima[r] > 0) has_best |= 1u << r;
    uint32_t need = lane_valid & ~has_best;
    while (need) {
      const int r = __ffs(need) - 1;
      need &= need - 1;
      const double E = tile_lane_energy<MODE == 1>(G, I, sw, r, s_redd, s_redi);
      if (tid == 0) s_best[r] = E;
    }
    __syncthreads();
    const int64_t out_base = (int64_t)A.R * I.spin_off + (int64_t)(32 * g) * n;
    for (int i = tid; i < n; i += blockDim.x) {
      const uint32_t wv = (bw[i] & has_best) | (sw[i] & ~has_best);
      for (int r = 0; r < 32; ++r)
        if ((lane_valid >> r) & 1u) A.spins[out_base + (int64_t)r * n + i] = ((wv >> r) & 1u) ? 1 : -1;
    }
    if (tid < 32 && ((lane_valid >> tid) & 1u)) {
      const int64_t o = (int64_t)b * A.R + 32 * g + tid;
      A.energy[o] = s_best[tid];
      if (A.energy_i32) A.energy_i32[o] = (int32_t)s_best[tid];
      if (A.minima) A.minima[o] = s_minima[tid];
    }
    __syncthreads();
  }

  // work counters
  my_flips = block_sum<unsigned long long>(my_flips, reinterpret_cast<unsigned long long *>(s_redi));
  if (tid == 0) {
    atomicAdd(A.stats + 0, my_evals);
    atomicAdd(A.stats + 1, my_flips);
    atomicAdd(A.stats + 2, my_minima);
    atomicAdd(A.stats + 3, my_desc);
    atomicAdd(A.stats + 4, my_sweeps);
  }
}

size_t tile_smem_bytes(int mode, int nmax) {
  return (size_t)(mode == 2 ? 1 : 2) * (size_t)nmax * sizeof(uint32_t);
}

int tile_max_ctas_per_sm(int mode, size_t smem) {
  int blocks = 0;
  cudaError_t e;
  if (mode == 0) {
    e = cudaFuncSetAttribute(tile_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, tile_kernel<0>, kTileThreads, smem);
  } else if (mode == 1) {
    e = cudaFuncSetAttribute(tile_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, tile_kernel<1>, kTileThreads, smem);
  } else {
    e = cudaFuncSetAttribute(tile_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, tile_kernel<2>, kTileThreads, smem);
  }
  return e == cudaSuccess ? blocks : 0;
}

cudaError_t launch_tile(ising_handle *h, int mode, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (mode == 0) {
    e = cudaFuncSetAttribute(tile_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) tile_kernel<0><<<grid, kTileThreads, smem, s>>>(h->d_tile_args);
  } else if (mode == 1) {
    e = cudaFuncSetAttribute(tile_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) tile_kernel<1><<<grid, kTileThreads, smem, s>>>(h->d_tile_args);
  } else {
    e = cudaFuncSetAttribute(tile_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) tile_kernel<2><<<grid, kTileThreads, smem, s>>>(h->d_tile_args);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace isg
