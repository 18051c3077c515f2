// fm.cu — the paper's pass-based local search with hill climbing (Sec. IV,
// Fig. 3) for instances of up to 4096 spins.
//
// One warp per search, as many per CTA as shared memory allows (fields in
// FP64, the pass's move list, lock bits and spins of each warp's instance).
// From each random start (Philox, the counter layout of ising_local_search)
// the search runs passes.  A pass computes every spin's gain -2 s_i f_i
// (FP64), then n times: takes the largest gain among the spins not yet moved
// in this pass (ties to the lowest index), applies that move even when the gain
// is negative (hill climbing), locks the spin, updates its neighbours' fields,
// and records the prefix whose running energy is strictly the lowest so far
// (the earliest such prefix).  The pass is then rolled back to that prefix; a
// new pass follows while the pass lowered the energy strictly (for float
// couplings by more than 1e-9 relative, so FP64 rounding cannot fake an
// improvement), else the pass's start is the result.  The paper keeps the
// gains in a heap (Fig. 4); here the warp takes the maximum by shuffles at each
// move (gains compared as order-preserving integers), which selects the same spin.
//
// The arithmetic follows the definition in this order: fields are FP64 sums
// of h_i, then the CSR row in stored order, then the incident hyper-edges in
// ascending edge order; a move of spin i adds 2 J_ij s_i to the fields of its
// CSR neighbours in row order and then each incident hyper-edge's term to its
// other members.  Integer couplings are exact throughout.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <map>
#include <vector>

#include "device_common.cuh"

namespace isg {

namespace {

constexpr int kFT = 256;           // threads per CTA
constexpr int kFW = kFT / 32;
constexpr int kFmMaxSpins = 4096;

struct FmArgs {
  DevGraph g;
  int32_t n_items, R, restarts, max_passes, is_float;
  const int2 *items;          // (instance, replica), largest instances first
  const uint64_t *seeds;      // [instances]
  int32_t *queue;
  int8_t *spins;              // [instance block: R x n] results
  double *energy;             // [instance][replica]
  int32_t *passes;            // [instance][replica] or null
  unsigned long long *stats;
};

__device__ __forceinline__ double coupling(const DevGraph &G, bool fl, int64_t k) {
  return fl ? (double)__ldg(reinterpret_cast<const float *>(G.J) + k)
            : (double)__ldg(reinterpret_cast<const int8_t *>(G.J) + k);
}
__device__ __forceinline__ double field_h(const DevGraph &G, bool fl, int64_t gi) {
  return fl ? (double)__ldg(reinterpret_cast<const float *>(G.h) + gi)
            : (double)__ldg(reinterpret_cast<const int8_t *>(G.h) + gi);
}
__device__ __forceinline__ double coupling_e(const DevGraph &G, bool fl, int64_t e) {
  return fl ? (double)__ldg(reinterpret_cast<const float *>(G.hJ) + e)
            : (double)__ldg(reinterpret_cast<const int8_t *>(G.hJ) + e);
}
// product of the spins of hyper-edge e except `skip` (-1: all)
__device__ __forceinline__ double hyper_prod(const DevGraph &G, int64_t e, const int8_t *s, int skip) {
  double p = 1.0;
  for (uint32_t q = __ldg(G.hptr + e), qe = __ldg(G.hptr + e + 1); q < qe; ++q) {
    const int m = __ldg(G.hmem + q);
    if (m != skip) p *= (double)s[m];
  }
  return p;
}

// Order-preserving integer image of the gain -2 s f (FP64, never NaN): larger
// gain, larger key; +0 and -0 map to the same key, as they compare equal.
// Integer compares keep the per-move maximum off the FP64 pipe.
__device__ __forceinline__ unsigned long long gain_key(double f, int8_t s) {
  unsigned long long b = (unsigned long long)__double_as_longlong(f);
  if (s > 0) b ^= 0x8000000000000000ull;  // the gain has the sign of -s f
  if ((b << 1) == 0ull) b = 0ull;          // -0 -> +0
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// E (Eq. 1 extended by Eq. 6) by one warp: pairs once (j > i), fields,
// hyper-edges; lane partial sums, then the warp sum (a fixed order)
__device__ double fm_energy(const DevGraph &G, const InstDesc &I, bool fl, const int8_t *s, int lane) {
  double acc = 0.0;
  for (int i = lane; i < I.n; i += 32) {
    const int64_t gi = I.spin_off + i;
    const double si = (double)s[i];
    for (uint32_t k = __ldg(G.row + gi), ke = __ldg(G.row + gi + 1); k < ke; ++k) {
      const int j = __ldg(G.col + k);
      if (j > i) acc -= coupling(G, fl, k) * si * (double)s[j];
    }
    acc -= field_h(G, fl, gi) * si;
  }
  for (int e = lane; e < I.n_hyper; e += 32) {
    const int64_t ge = I.hyper_off + e;
    acc -= coupling_e(G, fl, ge) * hyper_prod(G, ge, s, -1);
  }
  return warp_sum(acc);
}

// bytes of shared memory one warp needs for an instance of n spins
__host__ __device__ constexpr size_t fm_warp_bytes(int n) {
  return (size_t)n * 8 + (size_t)n * 4 + (size_t)((n + 31) / 32) * 4 + (size_t)n * 2 + 16;
}

// One warp per (instance, replica): no CTA barriers on the per-move path.
__global__ void __launch_bounds__(kFT) fm_kernel(FmArgs A, int nmax) {
  extern __shared__ __align__(16) uint8_t fm_smem[];
  const DevGraph &G = A.g;
  const bool fl = A.is_float != 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t *base = fm_smem + (size_t)warp * ((fm_warp_bytes(nmax) + 15) & ~(size_t)15);
  unsigned long long c_moves = 0, c_passes = 0, c_starts = 0;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(A.queue, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= A.n_items) break;
    const int b = A.items[it].x, r = A.items[it].y;
    const InstDesc I = G.inst[b];
    const int n = I.n;
    const int64_t so = I.spin_off;
    double *f = reinterpret_cast<double *>(base);                          // [n] fields
    int32_t *moves = reinterpret_cast<int32_t *>(f + n);                  // [n] moves of the pass
    uint32_t *lock = reinterpret_cast<uint32_t *>(moves + n);             // [n/32] moved in this pass
    int8_t *s = reinterpret_cast<int8_t *>(lock + (n + 31) / 32);         // [n] spins
    int8_t *sb = s + n;                                                   // [n] best over the starts
    const uint64_t seed = A.seeds[b];
    double E_all = DBL_MAX;  // lane 0's copy is used
    int total_passes = 0;
    for (int k = 0; k < A.restarts; ++k) {
      for (int i = lane; i < n; i += 32) {
        const uint4 x = start_bits(seed, (uint32_t)(i >> 7), (uint32_t)r, (uint32_t)k, (uint32_t)b);
        s[i] = ((word_of(x, (i & 127) >> 5) >> (i & 31)) & 1u) ? 1 : -1;
      }
      __syncwarp();
      double Estar = fm_energy(G, I, fl, s, lane);  // the same value in every lane
      int passes = 0;
      for (;;) {
        ++passes;
        // fields: h, the CSR row in order, then the hyper-edges in ascending order
        for (int i = lane; i < n; i += 32) {
          const int64_t gi = so + i;
          double acc = field_h(G, fl, gi);
          for (uint32_t kk = __ldg(G.row + gi), ke = __ldg(G.row + gi + 1); kk < ke; ++kk)
            acc += coupling(G, fl, kk) * (double)s[__ldg(G.col + kk)];
          for (uint32_t u = __ldg(G.inc_ptr + gi), ue = __ldg(G.inc_ptr + gi + 1); u < ue; ++u) {
            const int64_t e = __ldg(G.inc_edge + u);
            acc += coupling_e(G, fl, e) * hyper_prod(G, e, s, i);
          }
          f[i] = acc;
        }
        for (int w = lane; w < (n + 31) / 32; w += 32) lock[w] = 0u;
        __syncwarp();
        double Ecur = Estar, Ebest = Estar;  // lane 0's copies are used
        int best_prefix = 0;
        for (int step = 0; step < n; ++step) {
          // the largest gain among unlocked spins, ties to the lowest index
          unsigned long long bk = 0ull;
          int bi = 0x7fffffff;
          for (int i = lane; i < n; i += 32) {
            if ((lock[i >> 5] >> lane) & 1u) continue;  // i & 31 == lane
            const unsigned long long key = gain_key(f[i], s[i]);
            if (bi == 0x7fffffff || key > bk) {  // ascending i: the first of equal keys stays
              bk = key;
              bi = i;
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oi != 0x7fffffff && (bi == 0x7fffffff || ok > bk || (ok == bk && oi < bi))) {
              bk = ok;
              bi = oi;
            }
          }
          const int i = bi;  // every lane holds the same winner
          if (lane == 0) {
            const double gain = -2.0 * (double)s[i] * f[i];
            Ecur -= gain;  // apply the move
            if (Ecur < Ebest) {
              Ebest = Ecur;
              best_prefix = step + 1;
            }
            moves[step] = i;
            lock[i >> 5] |= 1u << (i & 31);
            s[i] = (int8_t)-s[i];
          }
          __syncwarp();
          // neighbours' fields: the CSR row (distinct columns, one lane each),
          // then the hyper-edges in order (one lane: shared members possible)
          const double si2 = 2.0 * (double)s[i];
          const int64_t gi = so + i;
          for (uint32_t kk = __ldg(G.row + gi) + lane, ke = __ldg(G.row + gi + 1); kk < ke; kk += 32)
            f[__ldg(G.col + kk)] += coupling(G, fl, kk) * si2;
          const uint32_t u0 = __ldg(G.inc_ptr + gi), u1 = __ldg(G.inc_ptr + gi + 1);
          if (u0 < u1) {
            __syncwarp();
            if (lane == 0)
              for (uint32_t u = u0; u < u1; ++u) {
                const int64_t e = __ldg(G.inc_edge + u);
                const double w2 = 2.0 * coupling_e(G, fl, e);
                for (uint32_t q = __ldg(G.hptr + e), qe = __ldg(G.hptr + e + 1); q < qe; ++q) {
                  const int m = __ldg(G.hmem + q);
                  if (m != i) f[m] += w2 * hyper_prod(G, e, s, m);
                }
              }
          }
          __syncwarp();
        }
        // roll back to the best prefix (each spin moved once: distinct entries)
        const int bp = __shfl_sync(0xffffffffu, best_prefix, 0);
        for (int st = bp + lane; st < n; st += 32) s[moves[st]] = (int8_t)-s[moves[st]];
        __syncwarp();
        const double Enew = fm_energy(G, I, fl, s, lane);
        const double margin = fl ? 1e-9 * (1.0 + fabs(Estar)) : 0.0;
        c_moves += (unsigned long long)n;
        if (Enew < Estar - margin && (A.max_passes <= 0 || passes < A.max_passes)) {
          Estar = Enew;
          continue;
        }
        if (Enew < Estar - margin) {
          Estar = Enew;  // pass cap reached after an improving pass: keep it
        } else {
          for (int st = lane; st < bp; st += 32) s[moves[st]] = (int8_t)-s[moves[st]];
          __syncwarp();
        }
        break;
      }
      total_passes += passes;
      c_passes += (unsigned long long)passes;
      c_starts += 1;
      // keep the best start (strictly lower energy; ties keep the earlier)
      if (Estar < E_all) {
        E_all = Estar;
        for (int i = lane; i < n; i += 32) sb[i] = s[i];
      }
      __syncwarp();
    }
    int8_t *out = A.spins + (int64_t)A.R * so + (int64_t)r * n;
    for (int i = lane; i < n; i += 32) out[i] = sb[i];
    if (lane == 0) {
      A.energy[(int64_t)b * A.R + r] = E_all;
      if (A.passes) A.passes[(int64_t)b * A.R + r] = total_passes;
    }
    __syncwarp();
  }
  if (lane == 0 && c_starts) {
    atomicAdd(A.stats + 0, c_moves);   // gains evaluated at a move: every spin once per pass
    atomicAdd(A.stats + 1, c_moves);   // moves applied (hill climbing included)
    atomicAdd(A.stats + 3, c_starts);  // starts
    atomicAdd(A.stats + 4, c_passes);  // passes
  }
}

// device (instance, replica) lists per handle, kept across calls
std::map<const ising_handle *, std::pair<int2 *, int64_t>> &fm_items() {
  static std::map<const ising_handle *, std::pair<int2 *, int64_t>> m;
  return m;
}

}  // namespace

int fm_max_spins() { return kFmMaxSpins; }

// One launch over every (instance, replica).  seeds: device [instances].
cudaError_t launch_fm(ising_handle *h, int32_t R, int32_t restarts, int32_t max_passes, int8_t *spins, double *E,
                      int32_t *passes, cudaStream_t s) {
  const int64_t n_items = (int64_t)h->n_inst * R;
  if (n_items > 0x7fffffff) return cudaErrorInvalidValue;
  auto &slot = fm_items()[h];
  cudaError_t e;
  if (slot.second < n_items) {
    cudaFree(slot.first);
    slot.first = nullptr;
    slot.second = 0;
    if ((e = cudaMalloc(&slot.first, (size_t)n_items * sizeof(int2))) != cudaSuccess) return e;
    slot.second = n_items;
  }
  std::vector<int32_t> ord(h->n_inst);
  for (int32_t b = 0; b < h->n_inst; ++b) ord[b] = b;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return h->inst[a].n > h->inst[c].n; });
  std::vector<int2> items;
  items.reserve((size_t)n_items);
  for (int32_t b : ord)
    for (int32_t r = 0; r < R; ++r) items.push_back(make_int2(b, r));
  if ((e = cudaMemcpyAsync(slot.first, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(h->d_queue, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
  FmArgs A;
  A.g = h->graph();
  A.n_items = (int32_t)n_items;
  A.R = R;
  A.restarts = restarts;
  A.max_passes = max_passes;
  A.is_float = h->dtype == ISING_F32 ? 1 : 0;
  A.items = slot.first;
  A.seeds = h->d_seeds;
  A.queue = h->d_queue;
  A.spins = spins;
  A.energy = E;
  A.passes = passes;
  A.stats = h->d_stats;
  const int nmax = h->nmax;
  // warps per CTA (one replica each) as shared memory allows
  const size_t per_warp = (fm_warp_bytes(nmax) + 15) & ~(size_t)15;
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  const int warps = (int)std::max<size_t>(1, std::min<size_t>(kFW, (size_t)smem_optin / per_warp));
  const size_t smem = per_warp * warps;
  if ((e = cudaFuncSetAttribute(fm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fm_kernel, warps * 32, smem)) != cudaSuccess)
    return e;
  const int64_t ctas_needed = (n_items + warps - 1) / warps;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)h->sm_count * std::max(per_sm, 1), ctas_needed));
  fm_kernel<<<grid, warps * 32, smem, s>>>(A, nmax);
  h->launches += 1;
  return cudaGetLastError();
}

void fm_free(ising_handle *h) {
  auto &m = fm_items();
  auto it = m.find(h);
  if (it == m.end()) return;
  cudaFree(it->second.first);
  m.erase(it);
}

}  // namespace isg
