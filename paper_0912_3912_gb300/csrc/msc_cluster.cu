// msc_cluster.cu — multi-spin-coded descent on periodic lattices with one
// thread-block cluster per (instance, 32-replica group).
//
// Same method and semantics as the multi-spin-coded tile kernel (García &
// Markov, Sec. IV: improving single-spin moves by colour class, a sweep without
// flips ends a descent, Philox restarts, best state kept), but the lattice is
// split over the P CTAs of a cluster: CTA q holds the spin words of sites
// [q n/P, (q+1) n/P) (whole z-slabs, or y-slabs in 2D) in its shared memory and
// reads the neighbour words owned by other CTAs through distributed shared
// memory.  The two checkerboard classes are separated by cluster barriers, so
// one lattice uses P SMs instead of one.
//
// Work layout: a warp visits a chunk of 64 consecutive sites per step, lane t
// taking the t-th site of the current class in the chunk (each row segment of
// even length holds equally many sites of both parities), so all 32 lanes do
// useful work and site indices, neighbours and wrap-around follow from the
// coordinates.  Coupling signs and the field of every site are one byte in
// shared memory.  Pending flags per (class, chunk) say whether some site of the
// class in the chunk has a neighbour that flipped since its last visit; a chunk
// without one is stable and skipped (only the first sweep of a descent visits
// everything).  All per-lane bookkeeping (sweep counts, convergence, best
// energies) is replicated identically in every CTA of the cluster, so the
// cluster's control flow stays uniform and every barrier is matched.
#include <cfloat>

#include "device_common.cuh"
#include "tc.cuh"

namespace isg {

namespace {

// CTAs of 512 threads, one per SM (two per SM at 64 registers, in clusters of
// 8, measured slower on the 32^3 lattice)
constexpr int kCT = 512;

template <int D>
__global__ void __launch_bounds__(kCT, 1) msc_cluster_kernel(const TileArgs *__restrict__ Aptr, int P) {
  extern __shared__ uint32_t smem[];
  __shared__ uint32_t s_any[2], s_active, s_convround, s_upd;
  __shared__ int32_t s_total[32], s_minima[32];
  __shared__ double s_best[32], s_E[32];
  __shared__ int32_t s_cnt[33];
  __shared__ int32_t s_rng[2][2];

  const TileArgs &A = *Aptr;
  const DevGraph G = A.g;
  const uint32_t rank = tc::cluster_rank();
  const int tile = blockIdx.x / P;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int b = A.tiles[tile].x, g = A.tiles[tile].y;
  const InstDesc I = G.inst[b];
  const int n = I.n, L = I.lat_L, lgL = 31 - __clz(L);
  const int csz = n / P;  // sites per CTA: a power of two, a multiple of 64 and of L^(D-1)
  const int lgc = 31 - __clz(csz);
  const int nch = csz >> 6;  // 64-site chunks per CTA
  const int lo = (int)rank * csz;
  uint32_t *sw = smem;                                          // words of sites lo .. lo + csz - 1
  uint32_t *pend = smem + csz;                                  // [2][nch] pending flags
  uint8_t *tab = reinterpret_cast<uint8_t *>(smem + csz + 2 * nch);  // [csz]: neg bits 0..5, h != 0, h > 0
  uint32_t *bw = smem + csz + 2 * nch + csz / 4;                      // [csz]: best words of my sites
  const int rem = A.R - 32 * g;
  const uint32_t lane_valid = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
  const uint64_t seed = A.seeds[b];
  const int64_t so = I.spin_off;
  const int lgp = min(lgL, 6) - 1;  // log2 of the class sites per row segment of a chunk
  unsigned long long my_flips = 0, my_evals = 0, my_sweeps = 0, my_minima = 0, my_desc = 0;
  unsigned long long my_eval = 0;  // (site, replica) pairs of the chunks visited (skipped chunks excluded)

  // word of site j (any CTA of the cluster).  Only neighbours along the slab
  // axis (z in 3D, y in 2D) can lie in another CTA, and a warp's sites share
  // that axis coordinate, so the branch is uniform.
  auto word = [&](int j) -> uint32_t {
    const uint32_t owner = (uint32_t)j >> lgc;
    if (owner == rank) return sw[j - lo];
    return tc::ld_cluster_u32(tc::map_shared(sw + (j & (csz - 1)), owner));
  };
  auto mark = [&](int j, int cls) {
    const uint32_t owner = (uint32_t)j >> lgc;
    uint32_t *f = pend + cls * nch + ((j & (csz - 1)) >> 6);
    if (owner == rank) *f = 1u;
    else tc::st_cluster_u32(tc::map_shared(f, owner), 1u);
  };
  // neighbour of site j in direction d (+x, -x, +y, -y, +z, -z), periodic:
  // step the axis coordinate inside its bit field (L is a power of two)
  auto nbr = [&](int j, int d) -> int {
    const int sh = (d >> 1) * lgL, m = (L - 1) << sh;
    const int t = (d & 1) ? j - (1 << sh) : j + (1 << sh);
    return (j & ~m) | (t & m);
  };
  // neighbour word in direction d of a site of mine (local off the slab axis)
  auto nword = [&](int j, int d) -> uint32_t {
    const int nb = nbr(j, d);
    if ((d >> 1) == D - 1) return word(nb);
    return sw[nb - lo];
  };

  // my part of each colour class (positions whose site lies in [lo, lo + csz))
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
  if (tid < 2) s_any[tid] = 0u;
  for (int q = tid; q < 2 * nch; q += blockDim.x) pend[q] = 0u;
  __syncthreads();
  // per-site byte: coupling signs by direction and the field
  for (int c = 0; c < 2; ++c)
    for (int v = s_rng[c][0] + tid; v < s_rng[c][1]; v += blockDim.x) {
      const int j = __ldg(G.order + so + v);
      const uint32_t info = __ldg(G.latinfo + so + v);
      const int hv = __ldg(reinterpret_cast<const int8_t *>(G.h) + so + j);
      tab[j - lo] = (uint8_t)(((info >> 8) & 63u) | (hv != 0 ? 64u : 0u) | (hv > 0 ? 128u : 0u));
    }
  __syncthreads();

  // lane-parallel energies of the cluster's lattice: every CTA counts its own
  // sites (one site per thread, the forward bonds +x, +y, +z and the field),
  // the counts are summed over the cluster in rank order
  auto energies = [&]() {
    constexpr int Q = 10;  // per-thread counts stay below 2^10 (csz / blockDim sites, D + 1 terms each)
    uint32_t acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = 0u;
    int nz = 0;
    if (tid < 33) s_cnt[tid] = 0;
    __syncthreads();
    for (int o = tid; o < csz; o += blockDim.x) {
      const int j = lo + o;
      const uint32_t wj = sw[o], t = tab[o];
      uint32_t f[3] = {0u, 0u, 0u};
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (a < D) f[a] = wj ^ nword(j, 2 * a) ^ (((t >> (2 * a)) & 1u) ? 0xffffffffu : 0u);
      const uint32_t uf = (t & 64u) ? ((t & 128u) ? ~wj : wj) : 0u;
      nz += (t & 64u) ? 1 : 0;
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

  uint32_t sc = 0;  // sweeps so far (all descents): picks the convergence buffer
  for (int k = 0;; ++k) {
    if (warp == 0) {
      const uint32_t start = __ballot_sync(
          0xffffffffu, k < A.restarts && ((lane_valid >> lane) & 1u) && (A.budget <= 0 || s_total[lane] < A.budget));
      if (lane == 0) {
        s_active = start;
        s_convround = 0;
        if (rank == 0) my_desc += __popc(start);
      }
    }
    __syncthreads();
    uint32_t active = s_active;
    if (!active) break;  // identical in every CTA of the cluster
    // random starts of my sites (Philox, counter layout of the C ABI)
    for (int w = (lo >> 7) + warp; w < ((lo + csz) >> 7); w += nwarps) {
      const uint4 x = start_bits(seed, (uint32_t)w, (uint32_t)(32 * g + lane), (uint32_t)k, (uint32_t)b);
      for (int q = 0; q < 4; ++q) {
        const uint32_t xw = word_of(x, q);
        const uint32_t mine = warp_transpose32(xw, lane);  // lane u: site u's word
        const int o = w * 128 + q * 32 + lane - lo;
        sw[o] = (sw[o] & ~active) | (mine & active);
      }
    }
    tc::cluster_sync();

    for (int d = 0; active; ++d, ++sc) {
      const bool fresh = d == 0;
      const int pb = sc & 1;
      uint32_t anyf = 0;
      for (int c = 0; c < 2; ++c) {
        for (int ch = warp; ch < nch; ch += nwarps) {
          uint32_t *pf = pend + c * nch + ch;
          if (!fresh && !*pf) continue;  // no site of the class here has a neighbour that flipped
          __syncwarp();
          if (lane == 0) {
            *pf = 0u;  // marks made in this phase go to the other class
            my_eval += 32ull * (unsigned long long)__popc(active);
          }
          // lane's site: the lane-th site of class c in the chunk
          const int r = lane >> lgp, q = lane & ((1 << lgp) - 1);
          const int rowbase = lo + (ch << 6) + (r << (lgp + 1));
          const int yz = (rowbase >> lgL) + (D == 3 ? (rowbase >> (2 * lgL)) : 0);
          const int j = rowbase + 2 * q + ((yz + c) & 1);
          const uint32_t wj = sw[j - lo], t = tab[j - lo];
          uint32_t x[6];
#pragma unroll
          for (int dd = 0; dd < 6; ++dd) {
            x[dd] = 0u;
            if (dd < 2 * D) x[dd] = wj ^ nword(j, dd) ^ (((t >> dd) & 1u) ? 0xffffffffu : 0u);
          }
          const uint32_t uf = (t & 64u) ? ((t & 128u) ? ~wj : wj) : 0u;
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
            sw[j - lo] = wj ^ flip;
            anyf |= flip;
            my_flips += __popc(flip);
          }
          // Pending flags of the chunks holding the flipped sites' neighbours.
          // Per direction those chunks are at most two, and lanes are ordered
          // so that they are the targets of the lowest and the highest
          // flipping lane (checked exhaustively for every accepted shape).
          const uint32_t fb = __ballot_sync(0xffffffffu, flip != 0u);
          if (fb) {
            const int jl = __shfl_sync(0xffffffffu, j, __ffs(fb) - 1);
            const int jh = __shfl_sync(0xffffffffu, j, 31 - __clz(fb));
            if (lane < 4 * D) {
              const int dd = lane < 2 * D ? lane : lane - 2 * D;
              mark(nbr(lane < 2 * D ? jl : jh, dd), c ^ 1);
            }
          }
        }
        if (c == 1) {
          anyf = __reduce_or_sync(0xffffffffu, anyf);
          if (lane == 0 && anyf) atomicOr(&s_any[pb], anyf);
        }
        tc::cluster_sync();  // class done in every CTA: its flips, marks and flags visible
        // every CTA read the other buffer's flags before this barrier: reset it
        if (c == 0 && tid == 0) s_any[pb ^ 1] = 0u;
      }
      if (warp == 0) {
        // lane = replica; lanes < P read the peers' convergence words
        const uint32_t any = __reduce_or_sync(
            0xffffffffu, lane < P ? tc::ld_cluster_u32(tc::map_shared(&s_any[pb], (uint32_t)lane)) : 0u);
        const bool act = (active >> lane) & 1u;
        int tot = s_total[lane];
        if (act) s_total[lane] = ++tot;
        const uint32_t conv = active & ~any;
        uint32_t ended = conv | __ballot_sync(0xffffffffu, act && A.budget > 0 && tot >= A.budget);
        if (d + 1 >= A.max_sweeps) ended |= active;
        if (lane == 0) {
          if (rank == 0) {
            my_sweeps += __popc(active);
            my_evals += (unsigned long long)__popc(active) * (unsigned long long)n;
            my_minima += __popc(conv);
          }
          s_convround |= conv;
          s_active = active & ~ended;
        }
      }
      __syncthreads();
      active = s_active;
      if (!active) {
        const uint32_t cr = s_convround;
        if (cr) {
          energies();
          if (warp == 0) {
            bool better = false;
            if ((cr >> lane) & 1u) {
              s_minima[lane] += 1;
              better = s_E[lane] < s_best[lane];
              if (better) s_best[lane] = s_E[lane];
            }
            const uint32_t upd = __ballot_sync(0xffffffffu, better);
            if (lane == 0) s_upd = upd;
          }
          __syncthreads();
          const uint32_t upd = s_upd;
          if (upd)
            for (int o = tid; o < csz; o += blockDim.x) bw[o] = (bw[o] & ~upd) | (sw[o] & upd);
        }
        // stale pending flags are harmless: the next descent's first sweep
        // visits every chunk and resets them
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
    const uint32_t wv = (bw[o] & has_best) | (sw[o] & ~has_best);
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
  my_eval = block_sum(my_eval, s_fl);
  if (tid == 0) atomicAdd(A.stats + 5, my_eval);
  tc::cluster_sync();  // no CTA leaves while peers may still read its shared memory
}

}  // namespace

// words, pending flags, per-site bytes, best words
size_t msc_cluster_smem(int csz) { return (size_t)csz * 4 + (size_t)(csz / 64) * 2 * 4 + (size_t)csz + (size_t)csz * 4; }

template <int D>
cudaError_t launch_cfg(cudaLaunchConfig_t &cfg, const TileArgs *args, int P, size_t smem, int *max_active) {
  auto kern = msc_cluster_kernel<D>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (max_active) return cudaOccupancyMaxActiveClusters(max_active, kern, &cfg);
  return cudaLaunchKernelEx(&cfg, kern, args, P);
}

// Launch (max_active == nullptr) or report how many clusters can be resident at once.
cudaError_t msc_cluster_launch_or_query(ising_handle *h, int n_tiles, int P, int csz_max, int D, cudaStream_t s,
                                        int *max_active) {
  const size_t smem = msc_cluster_smem(csz_max);

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
  const TileArgs *args = (const TileArgs *)h->d_tile_args;
  return D == 3 ? launch_cfg<3>(cfg, args, P, smem, max_active) : launch_cfg<2>(cfg, args, P, smem, max_active);
}

cudaError_t launch_msc_cluster(ising_handle *h, int n_tiles, int P, int csz_max, int D, cudaStream_t s) {
  return msc_cluster_launch_or_query(h, n_tiles, P, csz_max, D, s, nullptr);
}

int msc_cluster_max_active(ising_handle *h, int n_tiles, int P, int csz_max, int D) {
  int m = 0;
  if (msc_cluster_launch_or_query(h, n_tiles, P, csz_max, D, nullptr, &m) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return m;
}

}  // namespace isg
