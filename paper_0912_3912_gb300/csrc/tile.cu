// tile.cu — persistent tile kernels: one CTA (256 threads; four per SM, two for
// the lattice mode) works on one (instance, 32-replica group) tile at a time,
// pulled from a work queue largest first, with the instance's spins bit-packed
// in shared memory (bit r of word i = replica r of spin i is +1).
//
// Method (García & Markov, Sec. IV): single-spin moves taken when their gain
// -2 s_i f_i is positive, whole sweeps repeated until no move is taken (a 1-flip
// local minimum), independent random starts, the best result kept.  Colour
// classes are independent sets, so all spins of a class decide at once.
//
// Four evaluators share the sweep/restart machinery:
//   MODE 0  integer couplings, one warp per spin, lane = replica, exact int32
//           fields recomputed from the neighbours' bits at each visit;
//   MODE 1  FP32 couplings, one warp per spin, lane = replica, FP32 fields kept
//           per (spin, replica) and updated at each visit from the neighbours
//           that flipped since the previous visit (the paper's incremental gain
//           update), with a from-scratch refresh at descent sweeps
//           d % refresh == 0 (always d == 0): the FP64 sum rounded to FP32,
//           formed exactly in fixed point when that is exact (runit >= 0);
//           fields of instances that fit stay in shared memory;
//   MODE 2  multi-spin coding for J in {-1,+1}, h in {-1,0,+1}: one thread per
//           spin evaluates all 32 replicas with bitwise logic (unsatisfied-bond
//           masks counted in a bit-sliced adder, compared with the per-field
//           thresholds);
//   MODE 3  the same on periodic 2-d/3-d lattices, with neighbours computed
//           from the lattice geometry and the field folded into the count.
// Replicas of a tile run their descents in lockstep rounds: descent k of every
// lane starts together; a lane whose descent ended waits (masked) until the
// round ends.  Each replica's own sequence of states is exactly the one its
// C-ABI semantics define.
#include <cfloat>

#include <algorithm>

#include "device_common.cuh"

namespace isg {

namespace {

// Energies of all 32 replica lanes of the tile at once (Eq. 1 + Eq. 6): one
// warp per spin, lane = replica.  Integer couplings sum exactly in int64;
// FP32 couplings sum exactly in 64-bit fixed point when the instance allows it
// (InstDesc::ebase >= 0; one final rounding to FP64), else in FP64 with warps
// added in ascending order.  Each pair is counted at its smaller index, each
// hyper-edge once.  Every path is deterministic; the result goes to E[32].
template <bool FLOAT>
__device__ void tile_energy_lanes(const DevGraph &G, const InstDesc &I, const uint32_t *sw, double *red,
                                  double *E) {
  const int n = I.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ub = I.ebase;
  const bool fx = FLOAT && ub >= 0;
  double accd = 0.0;
  long long acci = 0;
  unsigned long long accl = 0;
  // the warp's spins i = warp + k nw, 32 at a time: lane k reads spin k's row
  // bounds and field in one pass, then the spins are taken in order
  for (int ib = warp; ib < n; ib += 32 * nw) {
    const int il = ib + lane * nw;
    uint32_t k0l = 0, k1l = 0, hvl = 0;
    if (il < n) {
      const int64_t g = I.spin_off + il;
      k0l = __ldg(G.row + g);
      k1l = __ldg(G.row + g + 1);
      hvl = FLOAT ? __float_as_uint(__ldg(reinterpret_cast<const float *>(G.h) + g))
                  : (uint32_t)(int32_t)__ldg(reinterpret_cast<const int8_t *>(G.h) + g);
    }
    const int cnt = min(32, (n - ib + nw - 1) / nw);
    for (int src = 0; src < cnt; ++src) {
      const int i = ib + src * nw;
      const uint32_t bi = (sw[i] >> lane) & 1u;
      const uint32_t k0 = __shfl_sync(0xffffffffu, k0l, src), k1 = __shfl_sync(0xffffffffu, k1l, src);
      const uint32_t hraw = __shfl_sync(0xffffffffu, hvl, src);
      if (FLOAT) {
        const float *Jf = reinterpret_cast<const float *>(G.J);
        const float hv = __uint_as_float(hraw);
        if (fx) {
          const int64_t th = xr_term(hv, ub);
          xe_add(acci, accl, bi ? -th : th);
          for (uint32_t k = k0; k < k1; ++k) {
            const int j = __ldg(G.col + k);
            if (j > i) {
              const int64_t t = xr_term(__ldg(Jf + k), ub);
              xe_add(acci, accl, (((sw[j] >> lane) & 1u) ^ bi) ? t : -t);
            }
          }
        } else {
          double e = bi ? (double)hv : -(double)hv;
          for (uint32_t k = k0; k < k1; ++k) {
            const int j = __ldg(G.col + k);
            if (j > i) {
              const double w = (double)__ldg(Jf + k);
              e += (((sw[j] >> lane) & 1u) ^ bi) ? -w : w;
            }
          }
          accd -= e;
        }
      } else {
        const int8_t *Ji = reinterpret_cast<const int8_t *>(G.J);
        const int hv = (int)hraw;
        int e = bi ? hv : -hv;
        for (uint32_t k = k0; k < k1; ++k) {
          const int j = __ldg(G.col + k);
          if (j > i) {
            const int w = __ldg(Ji + k);
            e += (((sw[j] >> lane) & 1u) ^ bi) ? -w : w;
          }
        }
        acci -= e;
      }
    }
  }
  for (int e = warp; e < I.n_hyper; e += nw) {
    const int64_t ge = I.hyper_off + e;
    uint32_t neg = 0;
    for (uint32_t q = __ldg(G.hptr + ge), qe = __ldg(G.hptr + ge + 1); q < qe; ++q)
      neg ^= ~(sw[__ldg(G.hmem + q)] >> lane) & 1u;
    if (FLOAT) {
      const float w = __ldg(reinterpret_cast<const float *>(G.hJ) + ge);
      if (fx) {
        const int64_t t = xr_term(w, ub);
        xe_add(acci, accl, neg ? t : -t);
      } else {
        accd -= neg ? -(double)w : (double)w;
      }
    } else {
      const int w = __ldg(reinterpret_cast<const int8_t *>(G.hJ) + ge);
      acci -= neg ? -w : w;
    }
  }
  long long *ri = reinterpret_cast<long long *>(red);
  __syncthreads();
  if (FLOAT && !fx) red[warp * 32 + lane] = accd;
  else ri[warp * 32 + lane] = acci;
  __syncthreads();
  long long hi = 0;
  if (warp == 0) {
    if (FLOAT && !fx) {
      double a = red[lane];
      for (int w = 1; w < nw; ++w) a += red[w * 32 + lane];
      E[lane] = a;
    } else {
      for (int w = 0; w < nw; ++w) hi += ri[w * 32 + lane];
      if (!FLOAT) E[lane] = (double)hi;
    }
  }
  if (fx) {
    __syncthreads();
    reinterpret_cast<unsigned long long *>(red)[warp * 32 + lane] = accl;
    __syncthreads();
    if (warp == 0) {
      unsigned long long lo = 0;
      for (int w = 0; w < nw; ++w) lo += reinterpret_cast<unsigned long long *>(red)[w * 32 + lane];
      E[lane] = xe_value(hi, lo, ub);
    }
  }
  __syncthreads();
}

// Energies of all 32 lanes for a +/-1 periodic lattice with |h| <= 1 (the
// multi-spin coded lattice path): E = 2 U - (n d + #{h != 0}), U = the lane's
// number of unsatisfied bonds and fields.  Each thread adds, per site, the
// unsatisfied masks of its forward bonds (+x, +y, +z) and of its field into a
// bit-sliced per-lane counter; a butterfly of bit-sliced adds totals the
// counters over the warp, and warps are added in shared memory.  Exact integers.
__device__ void tile_energy_lattice(const DevGraph &G, const InstDesc &I, const uint32_t *sw, int *cnt,
                                    double *E) {
  constexpr int Q = 14;  // counter depth: up to 2^14 - 1 per lane and thread
  const int n = I.n, L = I.lat_L, D = I.lat_d, lane = threadIdx.x & 31;
  const int stride[3] = {1, L, L * L};
  uint32_t acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) acc[q] = 0u;
  int nz = 0;
  if (threadIdx.x < 32) cnt[threadIdx.x] = 0;
  if (threadIdx.x == 32) cnt[32] = 0;
  __syncthreads();
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    const int j = __ldg(G.order + I.spin_off + v);
    const uint32_t info = __ldg(G.latinfo + I.spin_off + v);
    const int hv = __ldg(reinterpret_cast<const int8_t *>(G.h) + I.spin_off + j);
    const uint32_t wj = sw[j];
    uint32_t f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      f[a] = 0u;
      if (a < D) {
        const int d = 2 * a;  // forward direction along axis a
        const int nb = j + stride[a] - (((info >> d) & 1u) ? L * stride[a] : 0);
        f[a] = wj ^ sw[nb] ^ (((info >> (8 + d)) & 1u) ? 0xffffffffu : 0u);
      }
    }
    const uint32_t uf = hv == 0 ? 0u : (hv > 0 ? ~wj : wj);
    nz += hv != 0;
    // compress the four masks into weights 1, 2, 4 and add them to the counter
    const uint32_t s1 = f[0] ^ f[1] ^ f[2], c1 = (f[0] & f[1]) | (f[0] & f[2]) | (f[1] & f[2]);
    const uint32_t s2 = s1 ^ uf, c2 = s1 & uf;
    const uint32_t t1 = c1 ^ c2, t2 = c1 & c2;
    uint32_t cy = acc[0] & s2;
    acc[0] ^= s2;
    const uint32_t x1 = acc[1] ^ t1 ^ cy;
    cy = (acc[1] & t1) | (acc[1] & cy) | (t1 & cy);
    acc[1] = x1;
    const uint32_t x2 = acc[2] ^ t2 ^ cy;
    cy = (acc[2] & t2) | (acc[2] & cy) | (t2 & cy);
    acc[2] = x2;
#pragma unroll
    for (int q = 3; q < Q; ++q) {
      const uint32_t c = acc[q] & cy;
      acc[q] ^= cy;
      cy = c;
    }
  }
  const long long mine = warp_sliced_total<Q>(acc, lane);  // lane r: replica r's warp total
  nz = warp_sum(nz);
  atomicAdd(&cnt[lane], (int)mine);
  if (lane == 0) atomicAdd(&cnt[32], nz);
  __syncthreads();
  if (threadIdx.x < 32) E[threadIdx.x] = 2.0 * (double)cnt[threadIdx.x] - (double)n * D - (double)cnt[32];
  __syncthreads();
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
__global__ void __launch_bounds__(kTileThreads, MODE == 3 ? 2 : 4) tile_kernel(const TileArgs *__restrict__ Aptr) {
  extern __shared__ uint32_t smem[];
  __shared__ int s_tile;
  __shared__ uint32_t s_any, s_active, s_convround, s_upd;
  __shared__ int32_t s_total[32], s_minima[32];
  __shared__ double s_best[32], s_E[32];
  __shared__ double s_red[(kTileThreads / 32) * 32];
  __shared__ int s_cnt[33];

  const TileArgs &A = *Aptr;
  const DevGraph G = A.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int nmax = A.nmax;
  uint32_t *sw = smem;
  uint32_t *fm = smem + nmax;
  // pending bits: spin i's bit is set when a neighbour flipped (in any lane)
  // since i's last visit; a spin without it keeps its field and stays stable
  uint32_t *pb = smem + (MODE >= 2 ? 1 : 2) * nmax;
  uint32_t *bw = A.bw + (size_t)blockIdx.x * nmax;
  float *F = A.F ? A.F + (size_t)blockIdx.x * nmax * 32 : nullptr;
  // FP32 fields of instances up to A.fsm_cap spins stay in shared memory
  float *Fs = reinterpret_cast<float *>(smem + (((MODE >= 2 ? 1 : 2) * nmax + (nmax + 31) / 32 + 3) & ~3));
  // Work counters: thread 0's sweep-level counts go straight to shared memory;
  // every thread counts its flips and evaluated pairs of the current sweep in
  // 32 bits and adds the warp's total at the end of each sweep.
  //   s_work: 0 flip_evals, 1 flips, 2 minima, 3 descents, 4 sweeps, 5 evaluated
  __shared__ unsigned long long s_work[6];
  if (tid < 6) s_work[tid] = 0;
  uint32_t my_flips = 0, my_eval = 0;

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
    float *Fc = (MODE == 1 && n <= A.fsm_cap) ? Fs : F;
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
        s_convround = 0;
        s_work[3] += __popc(start);
      }
      __syncthreads();
      uint32_t active = s_active;
      if (!active) break;

      // Random starts for the lanes beginning descent k (Sec. IV); a warp
      // transposes 32 replicas x 128 spins with shuffle exchanges.
      for (int w = warp; w * 128 < n; w += nwarps) {
        const uint4 x = start_bits(seed, (uint32_t)w, (uint32_t)(32 * g + lane), (uint32_t)k, (uint32_t)b);
        for (int q = 0; q < 4; ++q) {
          const uint32_t xw = word_of(x, q);
          const uint32_t mine = warp_transpose32(xw, lane);  // lane u: site u's word
          const int i = w * 128 + q * 32 + lane;
          if (i < n) {
            sw[i] = (sw[i] & ~active) | (mine & active);
            if (MODE == 1) fm[i] &= ~active;
          }
        }
      }
      __syncthreads();

      for (int d = 0; active; ++d) {
        const bool refresh = (d == 0) || (A.refresh > 0 && d % A.refresh == 0);
        const bool fresh = MODE == 1 ? refresh : d == 0;  // every spin is evaluated
        auto pending = [&](int j) -> bool { return fresh || ((pb[j >> 5] >> (j & 31)) & 1u); };
        auto clear_pending = [&](int j) {
          if ((pb[j >> 5] >> (j & 31)) & 1u) atomicAnd(&pb[j >> 5], ~(1u << (j & 31)));
        };
        auto mark = [&](int i) { atomicOr(&pb[i >> 5], 1u << (i & 31)); };
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
          if (MODE == 3) {
            // +/-1 periodic lattice, |h| <= 1: the field counts as one more
            // bond, so every site flips when at least deg/2 + 1 of its bonds and
            // field are unsatisfied (3-d: majority of three carries; 2-d: >= 3).
            const int L = I.lat_L, D = I.lat_d;
            const int stride[3] = {1, L, L * L};
            for (int v = c0 + tid; v < c1; v += blockDim.x) {
              const int j = __ldg(G.order + I.spin_off + v);
              if (!pending(j)) continue;
              clear_pending(j);
              my_eval += __popc(active);
              const uint32_t info = __ldg(G.latinfo + I.spin_off + v);
              const int hv = __ldg(reinterpret_cast<const int8_t *>(G.h) + I.spin_off + j);
              const uint32_t wj = sw[j];
              uint32_t x[6];
#pragma unroll
              for (int d = 0; d < 6; ++d) {
                x[d] = 0u;
                if (d < 2 * D) {
                  const int a = d >> 1, st = stride[a];
                  int nb = (d & 1) ? j - st : j + st;
                  if ((info >> d) & 1u) nb += (d & 1) ? L * st : -L * st;
                  x[d] = wj ^ sw[nb] ^ (((info >> (8 + d)) & 1u) ? 0xffffffffu : 0u);
                }
              }
              const uint32_t uf = hv == 0 ? 0u : (hv > 0 ? ~wj : wj);
              uint32_t flip;
              const uint32_t s1 = x[0] ^ x[1] ^ x[2], c1 = (x[0] & x[1]) | (x[0] & x[2]) | (x[1] & x[2]);
              if (D == 3) {
                const uint32_t s2 = x[3] ^ x[4] ^ x[5], c2 = (x[3] & x[4]) | (x[3] & x[5]) | (x[4] & x[5]);
                const uint32_t c3 = (s1 & s2) | (s1 & uf) | (s2 & uf);
                flip = (c1 & c2) | (c1 & c3) | (c2 & c3);  // count >= 4
              } else {
                const uint32_t s2 = x[3] ^ uf ^ s1, c2 = (x[3] & uf) | (x[3] & s1) | (uf & s1);
                flip = (c1 & c2) | ((c1 | c2) & s2);  // count >= 3
              }
              flip &= active;
              if (flip)
                for (int d = 0; d < 2 * D; ++d) {
                  const int a = d >> 1, st = stride[a];
                  int nb = (d & 1) ? j - st : j + st;
                  if ((info >> d) & 1u) nb += (d & 1) ? L * st : -L * st;
                  mark(nb);
                }
              sw[j] = wj ^ flip;
              anyf |= flip;
              my_flips += __popc(flip);
            }
          } else if (MODE == 2) {
            const int8_t *Ji = reinterpret_cast<const int8_t *>(G.J);
            const int8_t *hi = reinterpret_cast<const int8_t *>(G.h);
            for (int v = c0 + tid; v < c1; v += blockDim.x) {
              const int j = A.sequential ? v : __ldg(G.order + I.spin_off + v);
              if (!pending(j)) continue;
              clear_pending(j);
              my_eval += __popc(active);
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
              if (flip)
                for (uint32_t kk = k0; kk < k1; ++kk) mark(__ldg(G.col + kk));
              sw[j] = wj ^ flip;
              anyf |= flip;
              my_flips += __popc(flip);
            }
          } else {
            // The warp's positions v = c0 + warp + k nwarps, 32 at a time: lane k
            // reads position k's spin and pending bit (one round trip for the 32),
            // a position with nothing pending is settled at once (its visit flips
            // nothing), and the others are visited in order.
            for (int vb = c0 + warp; vb < c1; vb += 32 * nwarps) {
              const int vl = vb + lane * nwarps;
              const bool inr = vl < c1;
              const int jl = inr ? (A.sequential ? vl : __ldg(G.order + I.spin_off + vl)) : 0;
              const bool pl = inr && pending(jl);
              if (MODE == 1 && inr && !pl && fm[jl]) fm[jl] = 0u;
              // a pending position's row and hyper-edge bounds, read with the batch
              uint32_t k0l = 0, k1l = 0, e0l = 0, e1l = 0;
              if (pl) {
                const int64_t g = I.spin_off + jl;
                k0l = __ldg(G.row + g);
                k1l = __ldg(G.row + g + 1);
                e0l = __ldg(G.inc_ptr + g);
                e1l = __ldg(G.inc_ptr + g + 1);
              }
              uint32_t todo = __ballot_sync(0xffffffffu, pl);
              while (todo) {
              const int src = __ffs(todo) - 1;
              todo &= todo - 1u;
              const int j = __shfl_sync(0xffffffffu, jl, src);
              const int64_t gj = I.spin_off + j;
              const uint32_t wj = sw[j];
              const bool up = (wj >> lane) & 1u;
              const uint32_t k0 = __shfl_sync(0xffffffffu, k0l, src), k1 = __shfl_sync(0xffffffffu, k1l, src);
              const uint32_t e0 = __shfl_sync(0xffffffffu, e0l, src), e1 = __shfl_sync(0xffffffffu, e1l, src);
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
                  const int2 oth = __ldg(G.inc_oth + q);
                  uint32_t neg = 0;
                  if (oth.x >= 0) {
                    neg = (~(sw[oth.x] >> lane) & 1u) ^ (~(sw[oth.y] >> lane) & 1u);
                  } else {
                    for (uint32_t m = __ldg(G.hptr + e), me = __ldg(G.hptr + e + 1); m < me; ++m) {
                      const int mm = __ldg(G.hmem + m);
                      if (mm != j) neg ^= ~(sw[mm] >> lane) & 1u;
                    }
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
                  // from scratch: the FP64 sum rounded to FP32, formed exactly in
                  // fixed point with the spin's precomputed unit when that is exact
                  const float hj = __ldg(reinterpret_cast<const float *>(G.h) + gj);
                  const int u = __ldg(G.runit + gj);
                  if (u >= 0) {
                    int64_t acc = xr_term(hj, u);
                    for (uint32_t kk = k0; kk < k1; ++kk) {
                      const int64_t t = xr_term(__ldg(Jf + kk), u);
                      acc += ((sw[__ldg(G.col + kk)] >> lane) & 1u) ? t : -t;
                    }
                    for (uint32_t q = e0; q < e1; ++q) {
                      const int e = __ldg(G.inc_edge + q);
                      const int2 oth = __ldg(G.inc_oth + q);
                      uint32_t neg = 0;
                      if (oth.x >= 0) {
                        neg = (~(sw[oth.x] >> lane) & 1u) ^ (~(sw[oth.y] >> lane) & 1u);
                      } else {
                        for (uint32_t m = __ldg(G.hptr + e), me = __ldg(G.hptr + e + 1); m < me; ++m) {
                          const int mm = __ldg(G.hmem + m);
                          if (mm != j) neg ^= ~(sw[mm] >> lane) & 1u;
                        }
                      }
                      const int64_t t = xr_term(__ldg(hJ + e), u);
                      acc += neg ? -t : t;
                    }
                    f = xr_round(acc, u);
                  } else {
                    double acc = (double)hj;
                    for (uint32_t kk = k0; kk < k1; ++kk) {
                      const int i = __ldg(G.col + kk);
                      const double w = (double)__ldg(Jf + kk);
                      acc = __dadd_rn(acc, ((sw[i] >> lane) & 1u) ? w : -w);
                    }
                    for (uint32_t q = e0; q < e1; ++q) {
                      const int e = __ldg(G.inc_edge + q);
                      const int2 oth = __ldg(G.inc_oth + q);
                      uint32_t neg = 0;
                      if (oth.x >= 0) {
                        neg = (~(sw[oth.x] >> lane) & 1u) ^ (~(sw[oth.y] >> lane) & 1u);
                      } else {
                        for (uint32_t m = __ldg(G.hptr + e), me = __ldg(G.hptr + e + 1); m < me; ++m) {
                          const int mm = __ldg(G.hmem + m);
                          if (mm != j) neg ^= ~(sw[mm] >> lane) & 1u;
                        }
                      }
                      const double w = (double)__ldg(hJ + e);
                      acc = __dadd_rn(acc, neg ? -w : w);
                    }
                    f = __double2float_rn(acc);
                  }
                } else {
                  // Pull the flips of the neighbours since this spin's previous
                  // visit (CSR order, then hyper-edges ascending), one pass; with
                  // none for this lane, field and decision are unchanged.
                  f = Fc[(size_t)j * 32 + lane];
                  bool dirty = false;
                  // the first kPre entries of the row fetched together (one round
                  // trip instead of one per entry), then applied in CSR order
                  constexpr int kPre = 6;
                  const int dg = (int)(k1 - k0);
                  int ci[kPre];
                  float cw[kPre];
#pragma unroll
                  for (int q = 0; q < kPre; ++q)
                    if (q < dg) {
                      ci[q] = __ldg(G.col + k0 + q);
                      cw[q] = __ldg(Jf + k0 + q);
                    }
#pragma unroll
                  for (int q = 0; q < kPre; ++q)
                    if (q < dg) {
                      const int i = ci[q];
                      if ((fm[i] >> lane) & 1u) {
                        const float w2 = 2.0f * cw[q];
                        f = __fadd_rn(f, ((sw[i] >> lane) & 1u) ? w2 : -w2);
                        dirty = true;
                      }
                    }
                  for (uint32_t kk = k0 + kPre; kk < k1; ++kk) {
                    const int i = __ldg(G.col + kk);
                    if ((fm[i] >> lane) & 1u) {
                      const float w2 = 2.0f * __ldg(Jf + kk);
                      f = __fadd_rn(f, ((sw[i] >> lane) & 1u) ? w2 : -w2);
                      dirty = true;
                    }
                  }
                  for (uint32_t q = e0; q < e1; ++q) {
                    const int e = __ldg(G.inc_edge + q);
                    const int2 oth = __ldg(G.inc_oth + q);  // a 3-member edge's other two, with the id
                    uint32_t neg = 0, par = 0;
                    if (oth.x >= 0) {
                      neg = (~(sw[oth.x] >> lane) & 1u) ^ (~(sw[oth.y] >> lane) & 1u);
                      par = ((fm[oth.x] >> lane) & 1u) ^ ((fm[oth.y] >> lane) & 1u);
                    } else {
                      for (uint32_t m = __ldg(G.hptr + e), me = __ldg(G.hptr + e + 1); m < me; ++m) {
                        const int mm = __ldg(G.hmem + m);
                        if (mm != j) {
                          neg ^= ~(sw[mm] >> lane) & 1u;
                          par ^= (fm[mm] >> lane) & 1u;
                        }
                      }
                    }
                    if (par) {
                      const float w2 = 2.0f * __ldg(hJ + e);
                      f = __fadd_rn(f, neg ? -w2 : w2);
                      dirty = true;
                    }
                  }
                  if (!dirty) {
                    flip = false;
                    goto decided;
                  }
                }
                Fc[(size_t)j * 32 + lane] = f;
                flip = up ? (f < 0.0f) : (f > 0.0f);
              decided:;
              }
              flip = flip && ((active >> lane) & 1u);
              const uint32_t m = __ballot_sync(0xffffffffu, flip);
              if (lane == 0) {
                my_eval += __popc(active);
                clear_pending(j);
                sw[j] = wj ^ m;
                if (MODE == 1) fm[j] = m;
              }
              if (m) {
                // the neighbours' pending marks, one lane per row entry / member
                for (uint32_t kk = k0 + lane; kk < k1; kk += 32) mark(__ldg(G.col + kk));
                for (uint32_t q = e0; q < e1; ++q) {
                  const int2 oth = __ldg(G.inc_oth + q);
                  if (oth.x >= 0) {
                    if (lane < 2) mark(lane == 0 ? oth.x : oth.y);
                    continue;
                  }
                  const int e = __ldg(G.inc_edge + q);
                  for (uint32_t mm = __ldg(G.hptr + e) + lane, me = __ldg(G.hptr + e + 1); mm < me; mm += 32) {
                    const int o = __ldg(G.hmem + mm);
                    if (o != j) mark(o);
                  }
                }
              }
              anyf |= m;
              my_flips += flip ? 1 : 0;
              }
            }
          }
          __syncthreads();
        }
        // end of sweep: which lanes flipped at all?
        anyf = __reduce_or_sync(0xffffffffu, anyf);
        if (lane == 0 && anyf) atomicOr(&s_any, anyf);
        {
          const uint32_t wf = __reduce_add_sync(0xffffffffu, my_flips);
          const uint32_t we = __reduce_add_sync(0xffffffffu, my_eval);
          if (lane == 0 && wf) atomicAdd(&s_work[1], (unsigned long long)wf);
          if (lane == 0 && we) atomicAdd(&s_work[5], (unsigned long long)we);
          my_flips = my_eval = 0;
        }
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
          s_work[4] += __popc(active);
          s_work[0] += (unsigned long long)__popc(active) * (unsigned long long)n;
          s_work[2] += __popc(conv);
          s_convround |= conv;
          s_active = active & ~ended;
        }
        __syncthreads();
        active = s_active;
        if (!active) {
          // Round over: converged lanes have been frozen since their last sweep,
          // so all of them are scored in one lane-parallel pass.
          const uint32_t cr = s_convround;
          if (cr) {
            if (MODE == 3) tile_energy_lattice(G, I, sw, s_cnt, s_E);
            else tile_energy_lanes<MODE == 1>(G, I, sw, s_red, s_E);
            if (tid == 0) {
              uint32_t upd = 0;
              for (int r = 0; r < 32; ++r)
                if ((cr >> r) & 1u) {
                  s_minima[r] += 1;
                  if (s_E[r] < s_best[r]) {
                    s_best[r] = s_E[r];
                    upd |= 1u << r;
                  }
                }
              s_upd = upd;
            }
            __syncthreads();
            const uint32_t upd = s_upd;
            if (upd)
              for (int i = tid; i < n; i += blockDim.x) bw[i] = (bw[i] & ~upd) | (sw[i] & upd);
          }
        }
        __syncthreads();
      }
    }

    // Result per lane: best converged state, else the final state of its last descent.
    uint32_t has_best = 0;
    for (int r = 0; r < 32; ++r)
      if (s_minima[r] > 0) has_best |= 1u << r;
    if (lane_valid & ~has_best) {
      if (MODE == 3) tile_energy_lattice(G, I, sw, s_cnt, s_E);
      else tile_energy_lanes<MODE == 1>(G, I, sw, s_red, s_E);
      if (tid < 32 && !((has_best >> tid) & 1u)) s_best[tid] = s_E[tid];
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
  __syncthreads();
  if (tid < 6 && s_work[tid]) atomicAdd(A.stats + tid, s_work[tid]);
}

size_t tile_smem_bytes(int mode, int nmax) {
  return (size_t)(mode >= 2 ? 1 : 2) * (size_t)nmax * sizeof(uint32_t) + (size_t)((nmax + 31) / 32) * sizeof(uint32_t);
}

// Spins whose FP32 fields (32 lanes) fit in shared memory next to the tile's
// words, within `budget` bytes of dynamic shared memory.
int tile_fsm_cap(int nmax, size_t budget) {
  const size_t base = (tile_smem_bytes(1, nmax) + 15) / 16 * 16;
  if (budget <= base) return 0;
  const size_t cap = (budget - base) / (32 * sizeof(float));
  return (int)std::min<size_t>(cap, (size_t)nmax);
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
  } else if (mode == 2) {
    e = cudaFuncSetAttribute(tile_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, tile_kernel<2>, kTileThreads, smem);
  } else {
    e = cudaFuncSetAttribute(tile_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, tile_kernel<3>, kTileThreads, smem);
  }
  return e == cudaSuccess ? blocks : 0;
}

// Launch only: the shared-memory attribute was set by tile_max_ctas_per_sm, so
// this is a plain stream operation and can be captured into a graph.
cudaError_t launch_tile(ising_handle *h, int mode, int grid, size_t smem, cudaStream_t s) {
  if (mode == 0) tile_kernel<0><<<grid, kTileThreads, smem, s>>>(h->d_tile_args);
  else if (mode == 1) tile_kernel<1><<<grid, kTileThreads, smem, s>>>(h->d_tile_args);
  else if (mode == 2) tile_kernel<2><<<grid, kTileThreads, smem, s>>>(h->d_tile_args);
  else tile_kernel<3><<<grid, kTileThreads, smem, s>>>(h->d_tile_args);
  return cudaGetLastError();
}

}  // namespace isg
