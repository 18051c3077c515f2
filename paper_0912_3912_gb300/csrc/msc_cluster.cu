// msc_cluster.cu — multi-spin-coded descent on periodic lattices with one
// thread-block cluster per (instance, 32-replica group).
//
// Same method and semantics as the multi-spin-coded tile kernel (García &
// Markov, Sec. IV: improving single-spin moves by colour class, a sweep without
// flips ends a descent, Philox restarts, best state kept), but the lattice is
// split over the P CTAs of a cluster: CTA q holds the spin words of sites
// [q n/P, (q+1) n/P) (z-slabs of the lattice) in its shared memory and reads
// the few neighbours owned by other CTAs through distributed shared memory.
// Colour classes are separated by cluster barriers, so one lattice uses P SMs
// instead of one.  All per-lane bookkeeping (sweep counts, convergence, best
// energies) is replicated identically in every CTA of the cluster, so the
// cluster's control flow stays uniform and every barrier is matched.
#include <cfloat>

#include "device_common.cuh"
#include "tc.cuh"

namespace isg {

namespace {

constexpr int kCT = 512;

__device__ __forceinline__ void dsmem_or(uint32_t addr, uint32_t v) {
  asm volatile("atom.shared::cluster.or.b32 _, [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

template <int D>
__global__ void __launch_bounds__(kCT, 1) msc_cluster_kernel(const TileArgs *__restrict__ Aptr, int P, int shift) {
  extern __shared__ uint32_t smem[];
  __shared__ uint32_t s_any_local, s_active, s_convround, s_upd, s_start;
  __shared__ int32_t s_total[32], s_minima[32];
  __shared__ double s_best[32], s_E[32];
  __shared__ int32_t s_cnt[33];
  __shared__ int32_t s_rng[2][2];

  const TileArgs &A = *Aptr;
  const DevGraph G = A.g;
  const uint32_t rank = tc::cluster_rank();
  const int tile = blockIdx.x / P;
  const int tid = threadIdx.x, lane = tid & 31;
  const int b = A.tiles[tile].x, g = A.tiles[tile].y;
  const InstDesc I = G.inst[b];
  const int n = I.n, L = I.lat_L;
  const int csz = n / P;             // sites per CTA (a power of two, multiple of 128)
  shift = 31 - __clz(csz);
  const int lo = (int)rank * csz;
  uint32_t *sw = smem;               // words of sites lo .. lo + csz - 1
  uint32_t *pb = smem + csz;         // pending bits of the same sites
  uint32_t *bw = A.bw + (size_t)tile * A.nmax;
  const int rem = A.R - 32 * g;
  const uint32_t lane_valid = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
  const uint64_t seed = A.seeds[b];
  const int stride[3] = {1, L, L * L};
  const int64_t so = I.spin_off;
  unsigned long long my_flips = 0, my_evals = 0, my_sweeps = 0, my_minima = 0, my_desc = 0;

  auto word = [&](int j) -> uint32_t {
    const uint32_t owner = (uint32_t)j >> shift;
    if (owner == rank) return sw[j - lo];
    return tc::ld_cluster_u32(tc::map_shared(sw + (j - ((int)owner << shift)), owner));
  };
  auto mark = [&](int j) {
    const uint32_t owner = (uint32_t)j >> shift;
    const int o = j - ((int)owner << shift);
    if (owner == rank) atomicOr(&pb[o >> 5], 1u << (o & 31));
    else dsmem_or(tc::map_shared(pb + (o >> 5), owner), 1u << (o & 31));
  };
  auto nbr = [&](int j, uint32_t info, int d) -> int {
    const int st = stride[d >> 1];
    int nb = (d & 1) ? j - st : j + st;
    if ((info >> d) & 1u) nb += (d & 1) ? L * st : -L * st;
    return nb;
  };

  // my part of each colour class: positions whose site lies in [lo, lo + csz)
  if (tid < 2) {
    const int c = tid;
    int a = __ldg(G.cls + I.cls_off + c), e = __ldg(G.cls + I.cls_off + c + 1);
    int l1 = a, h1 = e;
    while (l1 < h1) {
      const int mid = (l1 + h1) >> 1;
      if (__ldg(G.order + so + mid) < lo) l1 = mid + 1;
      else h1 = mid;
    }
    int l2 = l1, h2 = e;
    while (l2 < h2) {
      const int mid = (l2 + h2) >> 1;
      if (__ldg(G.order + so + mid) < lo + csz) l2 = mid + 1;
      else h2 = mid;
    }
    s_rng[c][0] = l1;
    s_rng[c][1] = l2;
  }
  if (tid < 32) {
    s_total[tid] = 0;
    s_minima[tid] = 0;
    s_best[tid] = DBL_MAX;
  }
  __syncthreads();

  // lane-parallel energies of the cluster's lattice: every CTA counts its own
  // sites, the counts are summed over the cluster in rank order
  auto energies = [&]() {
    constexpr int Q = 14;
    uint32_t acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = 0u;
    int nz = 0;
    if (tid < 33) s_cnt[tid] = 0;
    __syncthreads();
    for (int c = 0; c < 2; ++c)
    for (int v = s_rng[c][0] + tid; v < s_rng[c][1]; v += blockDim.x) {
      const int j = __ldg(G.order + so + v);
      const uint32_t info = __ldg(G.latinfo + so + v);
      const uint32_t wj = sw[j - lo];
      const int hv = __ldg(reinterpret_cast<const int8_t *>(G.h) + so + j);
      uint32_t f[3] = {0u, 0u, 0u};
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (a < D)  // forward bond along axis a (direction 2a), counted once per bond
          f[a] = wj ^ word(nbr(j, info, 2 * a)) ^ (((info >> (8 + 2 * a)) & 1u) ? 0xffffffffu : 0u);
      const uint32_t uf = hv == 0 ? 0u : (hv > 0 ? ~wj : wj);
      nz += hv != 0;
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
    long long mine = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q)
      for (int r = 0; r < 32; ++r) {
        const int c = __popc(__ballot_sync(0xffffffffu, (acc[q] >> r) & 1u));
        if (lane == r) mine += (long long)c << q;
      }
    nz = warp_sum(nz);
    atomicAdd(&s_cnt[lane], (int)mine);
    if (lane == 0) atomicAdd(&s_cnt[32], nz);
    __syncthreads();
    tc::cluster_sync();
    if (tid < 32) {
      long long u = 0, z = 0;
      for (int c = 0; c < P; ++c) {
        u += (int)tc::ld_cluster_u32(tc::map_shared(&s_cnt[tid], (uint32_t)c));
        z += (int)tc::ld_cluster_u32(tc::map_shared(&s_cnt[32], (uint32_t)c));
      }
      s_E[tid] = 2.0 * (double)u - (double)n * D - (double)z;
    }
    tc::cluster_sync();  // counts read everywhere before they are reset
  };

  for (int k = 0;; ++k) {
    if (tid == 0) {
      uint32_t start = 0;
      if (k < A.restarts)
        for (int r = 0; r < 32; ++r)
          if (((lane_valid >> r) & 1u) && (A.budget <= 0 || s_total[r] < A.budget)) start |= 1u << r;
      s_active = start;
      s_convround = 0;
      if (rank == 0) my_desc += __popc(start);
    }
    __syncthreads();
    uint32_t active = s_active;
    if (!active) break;  // identical in every CTA of the cluster
    // random starts of my sites (Philox, counter layout of the C ABI)
    for (int w = (lo >> 7) + (tid >> 5); w < ((lo + csz) >> 7); w += blockDim.x >> 5) {
      const uint4 x = start_bits(seed, (uint32_t)w, (uint32_t)(32 * g + lane), (uint32_t)k, (uint32_t)b);
      for (int q = 0; q < 4; ++q) {
        const uint32_t xw = word_of(x, q);
        uint32_t mine = 0;
        for (int u = 0; u < 32; ++u) {
          const uint32_t m = __ballot_sync(0xffffffffu, (xw >> u) & 1u);
          if (lane == u) mine = m;
        }
        const int o = w * 128 + q * 32 + lane - lo;
        sw[o] = (sw[o] & ~active) | (mine & active);
      }
    }
    tc::cluster_sync();

    for (int d = 0; active; ++d) {
      const bool fresh = d == 0;
      if (tid == 0) s_any_local = 0;
      uint32_t anyf = 0;
      for (int c = 0; c < 2; ++c) {
        const int v0 = s_rng[c][0], v1 = s_rng[c][1];
        for (int v = v0 + tid; v < v1; v += blockDim.x) {
          const int j = __ldg(G.order + so + v), o = j - lo;
          const bool pend = (pb[o >> 5] >> (o & 31)) & 1u;
          if (!fresh && !pend) continue;  // no neighbour flipped since the last visit
          if (pend) atomicAnd(&pb[o >> 5], ~(1u << (o & 31)));
          const uint32_t info = __ldg(G.latinfo + so + v);
          const int hv = __ldg(reinterpret_cast<const int8_t *>(G.h) + so + j);
          const uint32_t wj = sw[o];
          uint32_t x[6];
#pragma unroll
          for (int dd = 0; dd < 6; ++dd) {
            x[dd] = 0u;
            if (dd < 2 * D) x[dd] = wj ^ word(nbr(j, info, dd)) ^ (((info >> (8 + dd)) & 1u) ? 0xffffffffu : 0u);
          }
          const uint32_t uf = hv == 0 ? 0u : (hv > 0 ? ~wj : wj);
          const uint32_t s1 = x[0] ^ x[1] ^ x[2], c1 = (x[0] & x[1]) | (x[0] & x[2]) | (x[1] & x[2]);
          uint32_t flip;
          if (D == 3) {
            const uint32_t s2 = x[3] ^ x[4] ^ x[5], c2 = (x[3] & x[4]) | (x[3] & x[5]) | (x[4] & x[5]);
            const uint32_t c3 = (s1 & s2) | (s1 & uf) | (s2 & uf);
            flip = (c1 & c2) | (c1 & c3) | (c2 & c3);
          } else {
            const uint32_t s2 = x[3] ^ uf ^ s1, c2 = (x[3] & uf) | (x[3] & s1) | (uf & s1);
            flip = (c1 & c2) | ((c1 | c2) & s2);
          }
          flip &= active;
          if (flip) {
            sw[o] = wj ^ flip;
            for (int dd = 0; dd < 2 * D; ++dd) mark(nbr(j, info, dd));
            anyf |= flip;
            my_flips += __popc(flip);
          }
        }
        tc::cluster_sync();  // class done in every CTA; its flips and marks visible
      }
      anyf = __reduce_or_sync(0xffffffffu, anyf);
      if (lane == 0 && anyf) atomicOr(&s_any_local, anyf);
      __syncthreads();
      tc::cluster_sync();
      if (tid == 0) {
        uint32_t any = 0;
        for (int c = 0; c < P; ++c) any |= tc::ld_cluster_u32(tc::map_shared(&s_any_local, (uint32_t)c));
        uint32_t ended = 0;
        for (int r = 0; r < 32; ++r)
          if ((active >> r) & 1u) s_total[r] += 1;
        const uint32_t conv = active & ~any;
        ended |= conv;
        if (d + 1 >= A.max_sweeps) ended |= active;
        if (A.budget > 0)
          for (int r = 0; r < 32; ++r)
            if (((active >> r) & 1u) && s_total[r] >= A.budget) ended |= 1u << r;
        if (rank == 0) {
          my_sweeps += __popc(active);
          my_evals += (unsigned long long)__popc(active) * (unsigned long long)n;
          my_minima += __popc(conv);
        }
        s_convround |= conv;
        s_active = active & ~ended;
      }
      tc::cluster_sync();  // s_any_local read everywhere before the next reset
      active = s_active;
      if (!active) {
        const uint32_t cr = s_convround;
        if (cr) {
          energies();
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
            for (int o = tid; o < csz; o += blockDim.x) bw[lo + o] = (bw[lo + o] & ~upd) | (sw[o] & upd);
        }
      }
      __syncthreads();
    }
  }

  // results: best converged state per lane, else the final state of its last descent
  uint32_t has_best = 0;
  for (int r = 0; r < 32; ++r)
    if (s_minima[r] > 0) has_best |= 1u << r;
  if (lane_valid & ~has_best) {
    energies();
    if (tid < 32 && !((has_best >> tid) & 1u)) s_best[tid] = s_E[tid];
  }
  __syncthreads();
  const int64_t out_base = (int64_t)A.R * I.spin_off + (int64_t)(32 * g) * n;
  for (int o = tid; o < csz; o += blockDim.x) {
    const uint32_t wv = (bw[lo + o] & has_best) | (sw[o] & ~has_best);
    for (int r = 0; r < 32; ++r)
      if ((lane_valid >> r) & 1u) A.spins[out_base + (int64_t)r * n + lo + o] = ((wv >> r) & 1u) ? 1 : -1;
  }
  if (rank == 0 && tid < 32 && ((lane_valid >> tid) & 1u)) {
    const int64_t o = (int64_t)b * A.R + 32 * g + tid;
    A.energy[o] = s_best[tid];
    if (A.energy_i32) A.energy_i32[o] = (int32_t)s_best[tid];
    if (A.minima) A.minima[o] = s_minima[tid];
  }
  __syncthreads();
  if (tid == 0) {
    atomicAdd(A.stats + 0, my_evals);
    atomicAdd(A.stats + 2, my_minima);
    atomicAdd(A.stats + 3, my_desc);
    atomicAdd(A.stats + 4, my_sweeps);
  }
  __shared__ unsigned long long s_fl[kCT / 32];
  my_flips = block_sum(my_flips, s_fl);
  if (tid == 0) atomicAdd(A.stats + 1, my_flips);
  tc::cluster_sync();  // no CTA leaves while peers may still read its shared memory
}

}  // namespace

size_t msc_cluster_smem(int csz) { return (size_t)csz * 4 + (size_t)(csz / 32) * 4; }

cudaError_t launch_msc_cluster(ising_handle *h, int n_tiles, int P, int csz_max, int D, cudaStream_t s) {
  const size_t smem = msc_cluster_smem(csz_max);
  const int shift = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_tiles * P);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (D == 3) {
    e = cudaFuncSetAttribute(msc_cluster_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, msc_cluster_kernel<3>, (const TileArgs *)h->d_tile_args, P, shift);
  } else {
    e = cudaFuncSetAttribute(msc_cluster_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, msc_cluster_kernel<2>, (const TileArgs *)h->d_tile_args, P, shift);
  }
  return e;
}

}  // namespace isg
