// sweep.cu — large instances (too big for one CTA's shared memory): every
// colour class is one launch over the whole GPU; a sweep is the sequence of
// class launches plus a one-block end-of-sweep launch, with the round-end
// kernels (energy pass, restarts) after every fourth sweep; chunks of sweeps
// are captured once into a CUDA graph (cached) and replayed until every replica
// is done, the host polling a done flag one chunk behind.
//
// Same method and semantics as the tile kernels (García & Markov, Sec. IV:
// improving single-spin moves, repeated sweeps to a 1-flip minimum, random
// restarts, best kept; incremental FP32 field updates for float couplings with
// an exact refresh).  State lives in global memory: spin words sw[g][n] (bit l =
// replica 32g + l), flip masks fm[g][n], pending masks pend[g][n] (lanes with a
// neighbour that flipped since the spin's last visit), best words bw[g][n], FP32 fields
// F[g][position][LPS] stored in colour-class order so a class reads them
// contiguously.  LPS (lanes per spin) = 32, 16 or 8 replicas share one warp
// visit; with LPS < 32 a warp visits 32/LPS spins at once.
//
// Periodic lattices use the compact per-site metadata (DevGraph::meta/Jpos)
// instead of the CSR: 4 bytes of neighbour directions and coupling signs plus
// the couplings in class order, all read contiguously.
#include <cfloat>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <string>

#include "device_common.cuh"

namespace isg {

namespace {

constexpr int kST = 256;  // threads per CTA
// Resident CTAs per SM the visits are compiled for (registers per thread =
// 64K / (kST * this)): the multi-spin-coded visits 8, the lane visits below.
constexpr int kVisitCtasPerSm = 4;  // the FP32/int lane visits: 64 registers per thread

struct GroupState {
  uint32_t lane_valid, active, convround, any, upd, start;
  int32_t k, d, done, round_end, final_pass, pad;
  int32_t total[32], minima[32];
  double best[32], E[32];
};

struct SweepArgs {
  DevGraph g;
  InstDesc I;
  int32_t b, R, G, LPS;
  int32_t max_sweeps, restarts, budget, refresh, sequential, lattice;
  uint64_t seed;
  uint32_t *sw, *fm, *bw;
  uint32_t *pend;  // [g][n]: lanes in which some neighbour flipped since the spin's last visit
  // Parity-coloured lattices with an even side (class position = site >> 1):
  // per (group, class, chunk of 32 class positions) a flag word whose low
  // byte is set when a flip pushed a pending mark into the chunk and whose
  // high byte is set when the chunk's own last visit flipped a spin (so its
  // flip masks are nonzero).  A non-refresh visit skips chunks whose word is
  // zero; null when not applicable.  [g][2][nchunk]
  uint16_t *cflag;
  int32_t nchunk;
  // With cflag set the class positions map to sites arithmetically: class c,
  // position p holds site j = 2p + ((c + y + z) mod 2), y and z the row's
  // coordinates from 2p / L (exact multiply-shift division by L for values
  // below 2^24: q = (x * divL_m) >> divL_k)
  uint64_t divL_m;
  int32_t divL_k;
  float *F;
  GroupState *gs;
  double *partial;  // [grid_e][G][32]: FP64 sums of the CTAs (FP64 energies)
  // [G][32][2]: integer and fixed-point energies, high and low halves, summed
  // by atomic adds (order-free); read and zeroed by the last CTA
  unsigned long long *eacc;
  int32_t grid_e;
  // 1: energies of a lattice group taken site-parallel (lane = site, a loop over
  // the group's LPS replicas) with int64 sums per lane and warp; set when the
  // instance's term width and the sites per warp cannot overflow them
  int32_t en_fast;
  // 1: a multi-spin-coded lattice (J = +/-1, h in {-1, 0, 1}) whose energies are
  // counted bit-sliced (E = 2 U - B, U the unsatisfied bonds and fields)
  int32_t en_count;
  // 1: launch the chunk kernels with programmatic stream serialization
  // (measured faster for the multi-spin-coded visits, slower for the FP32 ones)
  int32_t pdl;
  unsigned int *counter;
  int32_t *all_done;
  unsigned long long *stats;
  int8_t *spins;
  double *energy;
  int32_t *energy_i32;
  int32_t *minima;
};

__device__ __forceinline__ int lat_nbr(int j, uint32_t meta, int k, int L) {
  const int dir = (meta >> (8 + 3 * k)) & 7;
  const int a = dir >> 1;
  const int stride = a == 0 ? 1 : (a == 1 ? L : L * L);
  int off = (dir & 1) ? -stride : stride;
  if ((meta >> k) & 1u) off += (dir & 1) ? L * stride : -L * stride;
  return j + off;
}


// Programmatic dependent launch (multi-spin-coded lattices; SweepArgs::pdl).
// The kernels of a sweep chunk may then be scheduled while their predecessor
// drains: a visit lets its dependants launch once each of its CTAs has done its
// main work (launch_dependents), and every chunk kernel waits, before reading
// anything its predecessor writes, until that grid has completed and its writes
// are visible (wait).  The wait is the hardware's grid dependency, not a spin on
// memory; for a kernel launched without the attribute both return at once.
__device__ __forceinline__ void pdl_prologue() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__global__ void sweep_init(SweepArgs A) {
  const int g = threadIdx.x;
  if (g < A.G) {
    GroupState &S = A.gs[g];
    const int rem = A.R - 32 * g;
    const int lanes = rem >= A.LPS ? A.LPS : rem;
    S.lane_valid = lanes >= 32 ? 0xffffffffu : ((1u << lanes) - 1u);
    S.start = S.lane_valid;
    S.active = S.lane_valid;
    S.convround = S.any = S.upd = 0;
    S.k = 0;
    S.d = 0;
    S.done = 0;
    S.round_end = 0;
    S.final_pass = 0;
    for (int r = 0; r < 32; ++r) {
      S.total[r] = 0;
      S.minima[r] = 0;
      S.best[r] = DBL_MAX;
      S.E[r] = 0.0;
    }
    atomicAdd(A.stats + 3, (unsigned long long)__popc(S.start));
  }
  if (threadIdx.x == 0) {
    *A.counter = 0;
    *A.all_done = 0;
  }
}

// u >= t for a bit-sliced 4-bit count (q0 least significant), t per thread.
__device__ __forceinline__ uint32_t sliced_ge4(uint32_t q0, uint32_t q1, uint32_t q2, uint32_t q3, int t) {
  if (t <= 0) return 0xffffffffu;
  if (t > 15) return 0u;
  uint32_t gt = 0, eq = 0xffffffffu;
  const uint32_t qq[4] = {q0, q1, q2, q3};
#pragma unroll
  for (int p = 3; p >= 0; --p) {
    const uint32_t tb = ((t >> p) & 1) ? 0xffffffffu : 0u;
    gt |= eq & qq[p] & ~tb;
    eq &= ~(qq[p] ^ tb);
  }
  return gt | eq;
}

// End of a sweep: per group, which lanes converged, which descents ended.
// One warp per group, lane l = replica lane l.  (Folding this into the last
// class visit - its last CTA closing the sweep - was measured slower than this
// separate launch.)
__global__ void sweep_end(SweepArgs A) {
  pdl_prologue();
  const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= A.G) return;
  GroupState &S = A.gs[g];
  const uint32_t active = S.active;
  const uint32_t any = S.any;
  __syncwarp();
  if (lane == 0) {
    S.start = 0;
    S.upd = 0;
  }
  if (!active) return;
  const bool mine = (active >> lane) & 1u;
  bool over = false;
  if (mine) {
    const int32_t t = S.total[lane] + 1;
    S.total[lane] = t;
    over = A.budget > 0 && t >= A.budget;
  }
  const uint32_t conv = active & ~any;
  uint32_t ended = __ballot_sync(0xffffffffu, over) | conv;
  const int32_t d = S.d + 1;
  if (d >= A.max_sweeps) ended |= active;
  if (lane == 0) {
    S.any = 0;
    S.d = d;
    atomicAdd(A.stats + 4, (unsigned long long)__popc(active));
    atomicAdd(A.stats + 0, (unsigned long long)__popc(active) * (unsigned long long)A.I.n);
    atomicAdd(A.stats + 2, (unsigned long long)__popc(conv));
    S.convround |= conv;
    S.active = active & ~ended;
    if (!(active & ~ended)) S.round_end = 1;
  }
}

// One colour class of one sweep.  MODE 0 int lanes, 1 FP32 lanes, 2 multi-spin
// coded.  Groups are walked in an outer loop so the per-group state is read once
// per warp and no index needs a division.
template <int MODE, int LPS, bool LAT>
__global__ void __launch_bounds__(kST, (MODE == 2 && LAT) ? 8 : kVisitCtasPerSm) sweep_visit(SweepArgs A, int32_t c) {
  __shared__ uint32_t s_any[32];
  __shared__ unsigned long long s_red[kST / 32];
  __shared__ int s_off[6], s_wrap[6];
  __shared__ unsigned int s_eval;
  const DevGraph &G = A.g;
  const InstDesc &I = A.I;
  const int n = I.n, L = I.lat_L;
  const int64_t so = I.spin_off;
  const int tid = threadIdx.x, lane = threadIdx.x & 31;
  pdl_prologue();
  if (tid < 32) s_any[tid] = 0;
  if (tid == 0) s_eval = 0;
  if (LAT && tid < 6) {
    // direction d: +x, -x, +y, -y, +z, -z; stride and wrap-around correction
    const int a = tid >> 1;
    const int st = a == 0 ? 1 : (a == 1 ? L : L * L);
    s_off[tid] = (tid & 1) ? -st : st;
    s_wrap[tid] = (tid & 1) ? L * st : -L * st;
  }
  __syncthreads();
  int c0, c1;
  if (A.sequential) {
    c0 = c;
    c1 = c + 1;
  } else {
    c0 = __ldg(G.cls + I.cls_off + c);
    c1 = __ldg(G.cls + I.cls_off + c + 1);
  }
  const int cs = c1 - c0;
  // per-thread counts of one launch (each below 2^32: a thread visits at most
  // n / threads positions of LPS replicas)
  uint32_t my_flips = 0;
  uint32_t my_eval = 0;  // (spin, replica) pairs whose gain this visit computed (skipped ones excluded)
  constexpr uint32_t lmask = LPS == 32 ? 0xffffffffu : ((1u << LPS) - 1u);

  if constexpr (MODE == 2) {
    const int8_t *hi = reinterpret_cast<const int8_t *>(G.h);
    const int8_t *Ji = reinterpret_cast<const int8_t *>(G.J);
    const int D = I.lat_d;
    for (int g = 0; g < A.G; ++g) {
      const uint32_t active = A.gs[g].active & lmask;
      if (!active) continue;
      const bool fresh = A.gs[g].d == 0;
      uint32_t *swg = A.sw + (size_t)g * n;
      uint32_t *pendg = A.pend + (size_t)g * n;
      uint32_t anyg = 0;
      for (int t = blockIdx.x * blockDim.x + tid; t < cs; t += gridDim.x * blockDim.x) {
        const int v = c0 + t;
        const int j = A.sequential ? v : __ldg(G.order + so + v);
        // everything indexed by the site itself is read in one round trip
        const uint32_t pj = pendg[j];
        const uint32_t wj = swg[j];
        const int hv = __ldg(hi + so + j);
        const uint32_t info = LAT ? __ldg(G.latinfo + so + v) : 0u;
        if (!fresh && !(pj & active)) continue;  // no neighbour flipped: still stable
        if (pj) pendg[j] = 0u;
        my_eval += __popc(active);
        uint32_t flip;
        if (LAT) {
          // field folded into the count: flip iff >= deg/2 + 1 of bonds+field unsatisfied
          uint32_t x[6];
#pragma unroll
          for (int d = 0; d < 6; ++d) {
            x[d] = 0u;
            if (d < 2 * D) {
              const int nb = j + s_off[d] + (((info >> d) & 1u) ? s_wrap[d] : 0);
              x[d] = wj ^ swg[nb] ^ (((info >> (8 + d)) & 1u) ? 0xffffffffu : 0u);
            }
          }
          const uint32_t uf = hv == 0 ? 0u : (hv > 0 ? ~wj : wj);
          const uint32_t s1 = x[0] ^ x[1] ^ x[2], c1b = (x[0] & x[1]) | (x[0] & x[2]) | (x[1] & x[2]);
          if (D == 3) {
            const uint32_t s2 = x[3] ^ x[4] ^ x[5], c2b = (x[3] & x[4]) | (x[3] & x[5]) | (x[4] & x[5]);
            const uint32_t c3b = (s1 & s2) | (s1 & uf) | (s2 & uf);
            flip = (c1b & c2b) | (c1b & c3b) | (c2b & c3b);
          } else {
            const uint32_t s2 = x[3] ^ uf ^ s1, c2b = (x[3] & uf) | (x[3] & s1) | (uf & s1);
            flip = (c1b & c2b) | ((c1b | c2b) & s2);
          }
        } else {
          uint32_t q0 = 0, q1 = 0, q2 = 0, q3 = 0;
          const uint32_t k0 = __ldg(G.row + so + j), k1 = __ldg(G.row + so + j + 1);
          const int deg = (int)(k1 - k0);
          for (uint32_t kk = k0; kk < k1; ++kk) {
            uint32_t x = wj ^ swg[__ldg(G.col + kk)] ^ (__ldg(Ji + kk) < 0 ? 0xffffffffu : 0u);
            uint32_t cy = q0 & x;
            q0 ^= x;
            x = cy;
            cy = q1 & x;
            q1 ^= x;
            x = cy;
            cy = q2 & x;
            q2 ^= x;
            q3 ^= cy;
          }
          if (hv == 0) {
            flip = sliced_ge4(q0, q1, q2, q3, deg / 2 + 1);
          } else {
            const uint32_t plus = hv > 0 ? wj : ~wj;
            flip = (sliced_ge4(q0, q1, q2, q3, (deg + 1) / 2 + 1) & plus) |
                   (sliced_ge4(q0, q1, q2, q3, deg >= 1 ? (deg - 1) / 2 + 1 : 0) & ~plus);
          }
        }
        flip &= active;
        if (flip) {
          swg[j] = wj ^ flip;
          anyg |= flip;
          my_flips += __popc(flip);
          if (LAT) {
            for (int d = 0; d < 2 * D; ++d)
              atomicOr(&pendg[j + s_off[d] + (((info >> d) & 1u) ? s_wrap[d] : 0)], flip);
          } else {
            for (uint32_t kk = __ldg(G.row + so + j), k1 = __ldg(G.row + so + j + 1); kk < k1; ++kk)
              atomicOr(&pendg[__ldg(G.col + kk)], flip);
          }
        }
      }
      anyg = __reduce_or_sync(0xffffffffu, anyg);
      if (lane == 0 && anyg) atomicOr(&s_any[g], anyg);
    }
  } else {
    // Lane paths.  A warp takes 32 consecutive class positions at a time: one
    // coalesced pass reads their pending masks and ballots the positions that
    // must be evaluated; those are then visited SPW at a time (LPS lanes =
    // replicas each), with all loads of one visit independent of each other.
    constexpr int SPW = 32 / LPS;
    const int sub = lane / LPS, ln = lane % LPS;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int wid = blockIdx.x * (blockDim.x >> 5) + (tid >> 5);
    const float *Jf = reinterpret_cast<const float *>(G.J);
    const float *hJf = reinterpret_cast<const float *>(G.hJ);
    for (int g = 0; g < A.G; ++g) {
      const GroupState &S = A.gs[g];
      const uint32_t active = S.active;
      if (!active) continue;
      const int dd = S.d;
      const bool refresh = (dd == 0) || (A.refresh > 0 && dd % A.refresh == 0);
      uint32_t *swg = A.sw + (size_t)g * n;
      uint32_t *fmg = A.fm + (size_t)g * n;
      uint32_t *pendg = A.pend + (size_t)g * n;
      float *Fg = (MODE == 1) ? A.F + (size_t)g * n * LPS : nullptr;
      const bool fresh = MODE == 1 ? refresh : dd == 0;  // every spin is evaluated
      uint32_t anyg = 0;
      if constexpr (MODE == 1 && LAT) {
        // Periodic lattice, FP32 fields.  Lane = position for every read a
        // visit needs (its word, the neighbour words, their flip masks, the
        // couplings, the field), so a warp step costs one round trip to memory.
        // Refresh sweeps evaluate every (site, replica) pair: SPW sites at a
        // time, LPS lanes each, values taken by shuffle.  Other sweeps evaluate
        // only the pairs with a pending bit: the positions stage their reads and
        // stored fields in shared memory, the pairs are listed, and all 32 lanes
        // work through the list; the flips are then applied per position.
        const int D2 = 2 * I.lat_d;
        const float *Jp0 = reinterpret_cast<const float *>(G.Jpos) + so;
        const float *hf = reinterpret_cast<const float *>(G.h) + so;
        uint16_t *cf_own = A.cflag ? A.cflag + ((size_t)g * 2 + c) * A.nchunk : nullptr;
        uint8_t *cf_oth = A.cflag ? reinterpret_cast<uint8_t *>(A.cflag + ((size_t)g * 2 + (c ^ 1)) * A.nchunk) : nullptr;
        auto nb_of = [&](int jj, uint32_t mm, int kk) -> int {
          const int dir = (mm >> (8 + 3 * kk)) & 7;
          return jj + s_off[dir] + (((mm >> kk) & 1u) ? s_wrap[dir] : 0);
        };
        // site of class position v (parity lattices with flags: no order load)
        auto site_of = [&](int v) -> int {
          if (!cf_own) return __ldg(G.order + so + v);
          const uint32_t p2 = 2u * (uint32_t)(v - c0);
          const uint32_t rho = (uint32_t)(((uint64_t)p2 * A.divL_m) >> A.divL_k);
          const uint32_t z = (uint32_t)(((uint64_t)rho * A.divL_m) >> A.divL_k);
          const uint32_t y = rho - z * (uint32_t)L;
          return (int)(p2 + (((uint32_t)c + y + z) & 1u));
        };
        for (int base = wid * 32; base < cs; base += nwarps * 32) {
          // chunk base >> 5 of this class: nothing pending and no flip masks to
          // clear means nothing to do (the word is read by every lane alike)
          if (cf_own && !refresh && cf_own[base >> 5] == 0) continue;
          const int v1 = c0 + base + lane;
          const bool valid1 = v1 < c1;
          const int j1 = valid1 ? site_of(v1) : 0;
          const uint32_t p1 = valid1 ? pendg[j1] : 0u;
          const uint32_t meta1 = valid1 ? __ldg(G.meta + so + v1) : 0u;
          const uint32_t fm1 = valid1 ? fmg[j1] : 0u;
          const bool need1 = valid1 && (refresh || (p1 & active) != 0u);
          if (valid1 && p1) pendg[j1] = 0u;
          if (valid1 && !need1 && fm1) fmg[j1] = 0u;  // no flips at this visit
          uint32_t todo = __ballot_sync(0xffffffffu, need1);
          if (!todo) {
            if (cf_own && lane == 0) cf_own[base >> 5] = 0;
            continue;
          }
          // replica visits of the positions not skipped (one shared add per warp step)
          if (lane == 0) atomicAdd(&s_eval, (uint32_t)__popc(todo) * (uint32_t)__popc(active));
          if (!refresh) {
            // Site-parallel: the position lane pulls, for each of its pending
            // replicas, the flips of the neighbours since the site's previous
            // visit (CSR order; FP32, round to nearest) into the stored field,
            // four replicas per 16-byte access, and decides the replicas whose
            // field changed.  With no flipped neighbour in a replica the field
            // and the decision are unchanged.
            uint32_t seg = 0u;
            if (need1) {
              const uint32_t pm = p1 & active;
              float *Frow = Fg + (size_t)v1 * LPS;
              // the pending replicas' field groups, fetched with the neighbour
              // reads below (pending includes every replica whose field changes;
              // 16-lane groups only: with 8 lanes the registers run short)
              constexpr int NG = LPS == 16 ? 4 : 1;
              float4 fpre[NG];
              if constexpr (LPS == 16) {
#pragma unroll
                for (int g4 = 0; g4 < NG; ++g4)
                  fpre[g4] = ((pm >> (4 * g4)) & 0xfu) ? *reinterpret_cast<const float4 *>(Frow + 4 * g4)
                                                      : make_float4(0.f, 0.f, 0.f, 0.f);
              }
              const uint32_t wj1 = swg[j1];
              uint32_t wn[6], fn[6];
              float w2[6];
              uint32_t dirtym = 0u;
#pragma unroll
              for (int kk = 0; kk < 6; ++kk) {
                wn[kk] = 0u;
                fn[kk] = 0u;
                w2[kk] = 0.0f;
                if (kk < D2) {
                  const int i = nb_of(j1, meta1, kk);
                  wn[kk] = swg[i];
                  fn[kk] = fmg[i] & pm;
                  w2[kk] = 2.0f * __ldg(Jp0 + (int64_t)kk * G.nsp + v1);
                  dirtym |= fn[kk];
                }
              }
#pragma unroll
              for (int r0 = 0; r0 < LPS; r0 += 4) {
                if (!((dirtym >> r0) & 0xfu)) continue;
                float4 f4;
                if constexpr (LPS == 16) f4 = fpre[r0 / 4];
                else f4 = *reinterpret_cast<const float4 *>(Frow + r0);
                float o[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  const int r = r0 + q;
                  if (!((dirtym >> r) & 1u)) continue;
                  float f = o[q];
#pragma unroll
                  for (int kk = 0; kk < 6; ++kk)
                    if ((fn[kk] >> r) & 1u) f = __fadd_rn(f, ((wn[kk] >> r) & 1u) ? w2[kk] : -w2[kk]);
                  o[q] = f;
                  if (((wj1 >> r) & 1u) ? (f < 0.0f) : (f > 0.0f)) seg |= 1u << r;
                }
                *reinterpret_cast<float4 *>(Frow + r0) = make_float4(o[0], o[1], o[2], o[3]);
              }
              if (seg) {
                swg[j1] = wj1 ^ seg;
                for (int kk = 0; kk < D2; ++kk) {
                  const int nb = nb_of(j1, meta1, kk);
                  atomicOr(&pendg[nb], seg);
                  if (cf_oth) cf_oth[2 * (nb >> 6)] = 1;
                }
              }
              if (seg || fm1) fmg[j1] = seg;
            }
            if (cf_own) {
              const bool fl = __any_sync(0xffffffffu, seg != 0u);
              if (lane == 0) cf_own[base >> 5] = fl ? (uint16_t)0x0100 : (uint16_t)0;
            }
            anyg |= seg;
            my_flips += __popc(seg);
            continue;
          }
          // refresh sweep: every pair of every position, site-parallel.  The
          // position lane forms its site's terms once - fixed-point integers
          // when the sum is exact, else the FP32 values for the FP64 path - and
          // evaluates all LPS replicas of the site from registers, writing the
          // fields four replicas at a time.
          uint32_t segr = 0u;
          if (need1) {
            const uint32_t wj1 = swg[j1];
            const float hj = __ldg(hf + j1);
            float jw[6];
            uint32_t wn[6];
            XRange xr;
            xr_see(xr, hj);
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) {
              jw[kk] = 0.0f;
              wn[kk] = 0u;
              if (kk < D2) {
                wn[kk] = swg[nb_of(j1, meta1, kk)];
                jw[kk] = __ldg(Jp0 + (int64_t)kk * G.nsp + v1);
                xr_see(xr, jw[kk]);
              }
            }
            float *Frow = Fg + (size_t)v1 * LPS;
            uint32_t seg = 0u;
            if (xr_exact(xr)) {
              // from scratch, exactly: f = (h + sum_k J_k) - sum over the
              // neighbours pointing down of 2 J_k, in fixed point with the
              // site's unit, rounded once to FP32
              const int u = xr.emax < 0 ? 24 : xr.emin;
              int64_t base0 = xr_term(hj, u), t2[6];
#pragma unroll
              for (int kk = 0; kk < 6; ++kk) {
                const int64_t t = kk < D2 ? xr_term(jw[kk], u) : 0;
                base0 += t;
                t2[kk] = 2 * t;
              }
#pragma unroll 1
              for (int r0 = 0; r0 < LPS; r0 += 4) {
                float o[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  const int r = r0 + q;
                  int64_t acc = base0;
#pragma unroll
                  for (int kk = 0; kk < 6; ++kk)
                    if (!((wn[kk] >> r) & 1u)) acc -= t2[kk];
                  o[q] = xr_round(acc, u);
                  if (((wj1 >> r) & 1u) ? (o[q] < 0.0f) : (o[q] > 0.0f)) seg |= 1u << r;
                }
                *reinterpret_cast<float4 *>(Frow + r0) = make_float4(o[0], o[1], o[2], o[3]);
              }
            } else {
              // the FP64 sum in the defined order (field, then the row's entries)
#pragma unroll 1
              for (int r0 = 0; r0 < LPS; r0 += 4) {
                float o[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  const int r = r0 + q;
                  double acc = (double)hj;
#pragma unroll
                  for (int kk = 0; kk < 6; ++kk)
                    if (kk < D2) acc = __dadd_rn(acc, ((wn[kk] >> r) & 1u) ? (double)jw[kk] : -(double)jw[kk]);
                  o[q] = __double2float_rn(acc);
                  if (((wj1 >> r) & 1u) ? (o[q] < 0.0f) : (o[q] > 0.0f)) seg |= 1u << r;
                }
                *reinterpret_cast<float4 *>(Frow + r0) = make_float4(o[0], o[1], o[2], o[3]);
              }
            }
            seg &= active;
            segr = seg;
            anyg |= seg;
            // apply: words of this class, pending marks of the other class,
            // flip masks (nothing another lane of this visit reads)
            if (seg) {
              swg[j1] = wj1 ^ seg;
              for (int kk = 0; kk < D2; ++kk) {
                const int nb = nb_of(j1, meta1, kk);
                atomicOr(&pendg[nb], seg);
                if (cf_oth) cf_oth[2 * (nb >> 6)] = 1;
              }
            }
            if (seg || fm1) fmg[j1] = seg;
            my_flips += __popc(seg);
          }
          if (cf_own) {
            const bool fl = __any_sync(0xffffffffu, segr != 0u);
            if (lane == 0) cf_own[base >> 5] = fl ? (uint16_t)0x0100 : (uint16_t)0;
          }
          __syncwarp();  // staging read before the next batch overwrites it
        }
      } else
      for (int base = wid * 32; base < cs; base += nwarps * 32) {
        const int v1 = c0 + base + lane;
        const bool valid1 = v1 < c1;
        const int j1 = valid1 ? (A.sequential ? v1 : __ldg(G.order + so + v1)) : 0;
        const uint32_t p1 = valid1 ? pendg[j1] : 0u;
        const uint32_t meta1 = (LAT && valid1) ? __ldg(G.meta + so + v1) : 0u;
        // Only a spin with a neighbour that flipped since its last visit can
        // change its decision (its field is otherwise unchanged and it was left
        // stable); the pending mask, pushed by flipping neighbours, says which
        // lanes.  The class is an independent set, so nothing pushes into it now.
        const bool need1 = valid1 && (fresh || (p1 & active) != 0u);
        if (valid1 && p1) pendg[j1] = 0u;
        if (MODE == 1 && valid1 && !need1 && !refresh && fmg[j1]) fmg[j1] = 0u;  // no flips at this visit
        uint32_t todo = __ballot_sync(0xffffffffu, need1);
        while (todo) {
          uint32_t t = todo;
          for (int q = 0; q < sub; ++q) t &= t - 1u;
          const int src = t ? __ffs(t) - 1 : 31;
          const bool valid = t != 0u;
          for (int q = 0; q < SPW; ++q) todo &= todo - 1u;
          const int v = __shfl_sync(0xffffffffu, v1, src);
          const int j = __shfl_sync(0xffffffffu, j1, src);
          const uint32_t pj = __shfl_sync(0xffffffffu, p1, src);
          const uint32_t meta = __shfl_sync(0xffffffffu, meta1, src);
          const bool need = valid && (fresh || ((pj >> ln) & 1u));
          const uint32_t wj = valid ? swg[j] : 0u;
          const bool up = (wj >> ln) & 1u;
          bool flip = false;
          if (need && ((active >> ln) & 1u)) my_eval += 1;
          if (need) {
            const uint32_t k0 = LAT ? 0u : __ldg(G.row + so + j);
            const uint32_t k1 = LAT ? (uint32_t)(2 * I.lat_d) : __ldg(G.row + so + j + 1);
            const uint32_t e0 = LAT ? 0u : __ldg(G.inc_ptr + so + j);
            const uint32_t e1 = LAT ? 0u : __ldg(G.inc_ptr + so + j + 1);
            auto nbr = [&](uint32_t kk) -> int {
              if (LAT) {
                const int dir = (meta >> (8 + 3 * kk)) & 7;
                return j + s_off[dir] + (((meta >> kk) & 1u) ? s_wrap[dir] : 0);
              }
              return __ldg(G.col + kk);
            };
            if (MODE == 0) {
              int f = __ldg(reinterpret_cast<const int8_t *>(G.h) + so + j);
              const int8_t *Jp = LAT ? reinterpret_cast<const int8_t *>(G.Jpos) + so + v : nullptr;
              if (LAT) {
                uint32_t sn[6];
                int wv[6];
#pragma unroll
                for (int kk = 0; kk < 6; ++kk)
                  if (kk < (int)k1) {
                    sn[kk] = swg[nbr(kk)];
                    wv[kk] = __ldg(Jp + (int64_t)kk * G.nsp);
                  }
#pragma unroll
                for (int kk = 0; kk < 6; ++kk)
                  if (kk < (int)k1) f += ((sn[kk] >> ln) & 1u) ? wv[kk] : -wv[kk];
              } else {
                for (uint32_t kk = k0; kk < k1; ++kk) {
                  const int w = (int)__ldg(reinterpret_cast<const int8_t *>(G.J) + kk);
                  f += ((swg[nbr(kk)] >> ln) & 1u) ? w : -w;
                }
              }
              if constexpr (!LAT) for (uint32_t q = e0; q < e1; ++q) {  // no hyper-edges on lattices
                const int e = __ldg(G.inc_edge + q);
                uint32_t neg = 0;
                for (uint32_t m = __ldg(G.hptr + e), me = __ldg(G.hptr + e + 1); m < me; ++m) {
                  const int mm = __ldg(G.hmem + m);
                  if (mm != j) neg ^= ~(swg[mm] >> ln) & 1u;
                }
                const int w = __ldg(reinterpret_cast<const int8_t *>(G.hJ) + e);
                f += neg ? -w : w;
              }
              flip = up ? (f < 0) : (f > 0);
            } else {
              const float *Jp = LAT ? reinterpret_cast<const float *>(G.Jpos) + so + v : nullptr;
              float *Fp = Fg + (size_t)v * LPS + ln;
              auto coup = [&](uint32_t kk) -> float {
                return LAT ? __ldg(Jp + (int64_t)kk * G.nsp) : __ldg(Jf + kk);
              };
              float f;
              if (refresh) {
                // from scratch: the FP64 sum rounded to FP32, formed exactly in
                // fixed point with the spin's precomputed unit when that is exact
                // (this path serves CSR instances; lattices take the staged path)
                const float hj = __ldg(reinterpret_cast<const float *>(G.h) + so + j);
                auto hyper_neg = [&](int e) -> uint32_t {
                  uint32_t neg = 0;
                  for (uint32_t m = __ldg(G.hptr + e), me = __ldg(G.hptr + e + 1); m < me; ++m) {
                    const int mm = __ldg(G.hmem + m);
                    if (mm != j) neg ^= ~(swg[mm] >> ln) & 1u;
                  }
                  return neg;
                };
                const int u = __ldg(G.runit + so + j);
                if (u >= 0) {
                  int64_t acc = xr_term(hj, u);
                  for (uint32_t kk = k0; kk < k1; ++kk) {
                    const int64_t tt = xr_term(coup(kk), u);
                    acc += ((swg[nbr(kk)] >> ln) & 1u) ? tt : -tt;
                  }
                  if constexpr (!LAT) for (uint32_t q = e0; q < e1; ++q) {  // no hyper-edges on lattices
                    const int e = __ldg(G.inc_edge + q);
                    const int64_t tt = xr_term(__ldg(hJf + e), u);
                    acc += hyper_neg(e) ? -tt : tt;
                  }
                  f = xr_round(acc, u);
                } else {
                  double acc = (double)hj;
                  for (uint32_t kk = k0; kk < k1; ++kk) {
                    const double w = (double)coup(kk);
                    acc = __dadd_rn(acc, ((swg[nbr(kk)] >> ln) & 1u) ? w : -w);
                  }
                  if constexpr (!LAT) for (uint32_t q = e0; q < e1; ++q) {  // no hyper-edges on lattices
                    const int e = __ldg(G.inc_edge + q);
                    const double w = (double)__ldg(hJf + e);
                    acc = __dadd_rn(acc, hyper_neg(e) ? -w : w);
                  }
                  f = __double2float_rn(acc);
                }
                *Fp = f;
                flip = up ? (f < 0.0f) : (f > 0.0f);
              } else {
                // Pull the flips of the neighbours since this spin's previous
                // visit (CSR order, then hyper-edges ascending).  If none flipped
                // for this lane the field and so the decision are unchanged.
                f = *Fp;
                bool dirty = false;
                if (LAT) {
                  uint32_t fn[6], sn[6];
                  float jw[6];
#pragma unroll
                  for (int kk = 0; kk < 6; ++kk)
                    if (kk < (int)k1) {
                      const int i = nbr(kk);
                      fn[kk] = fmg[i];
                      sn[kk] = swg[i];
                      jw[kk] = coup(kk);
                    }
#pragma unroll
                  for (int kk = 0; kk < 6; ++kk)
                    if (kk < (int)k1 && ((fn[kk] >> ln) & 1u)) {
                      const float w2 = 2.0f * jw[kk];
                      f = __fadd_rn(f, ((sn[kk] >> ln) & 1u) ? w2 : -w2);
                      dirty = true;
                    }
                } else {
                  for (uint32_t kk = k0; kk < k1; ++kk) {
                    const int i = nbr(kk);
                    if ((fmg[i] >> ln) & 1u) {
                      const float w2 = 2.0f * coup(kk);
                      f = __fadd_rn(f, ((swg[i] >> ln) & 1u) ? w2 : -w2);
                      dirty = true;
                    }
                  }
                  if constexpr (!LAT) for (uint32_t q = e0; q < e1; ++q) {  // no hyper-edges on lattices
                    const int e = __ldg(G.inc_edge + q);
                    uint32_t neg = 0, par = 0;
                    for (uint32_t m = __ldg(G.hptr + e), me = __ldg(G.hptr + e + 1); m < me; ++m) {
                      const int mm = __ldg(G.hmem + m);
                      if (mm != j) {
                        const uint32_t x = swg[mm];
                        neg ^= ~(x >> ln) & 1u;
                        par ^= (fmg[mm] >> ln) & 1u;
                      }
                    }
                    if (par) {
                      const float w2 = 2.0f * __ldg(hJf + e);
                      f = __fadd_rn(f, neg ? -w2 : w2);
                      dirty = true;
                    }
                  }
                }
                if (dirty) {
                  *Fp = f;
                  flip = up ? (f < 0.0f) : (f > 0.0f);
                }
              }
            }
            flip = flip && ((active >> ln) & 1u);
          }
          const uint32_t m = __ballot_sync(0xffffffffu, flip);
          const uint32_t seg = (m >> (sub * LPS)) & lmask;
          if (valid && ln == 0) {
            if (seg) {
              swg[j] = wj ^ seg;
              // tell the neighbours (and hyper-edge co-members) which lanes flipped
              if (LAT) {
                for (int kk = 0; kk < 2 * I.lat_d; ++kk) {
                  const int dir = (meta >> (8 + 3 * kk)) & 7;
                  atomicOr(&pendg[j + s_off[dir] + (((meta >> kk) & 1u) ? s_wrap[dir] : 0)], seg);
                }
              } else {
                for (uint32_t kk = __ldg(G.row + so + j), k1 = __ldg(G.row + so + j + 1); kk < k1; ++kk)
                  atomicOr(&pendg[__ldg(G.col + kk)], seg);
                for (uint32_t q = __ldg(G.inc_ptr + so + j), q1 = __ldg(G.inc_ptr + so + j + 1); q < q1; ++q) {
                  const int e = __ldg(G.inc_edge + q);
                  for (uint32_t mm = __ldg(G.hptr + e), me = __ldg(G.hptr + e + 1); mm < me; ++mm) {
                    const int o = __ldg(G.hmem + mm);
                    if (o != j) atomicOr(&pendg[o], seg);
                  }
                }
              }
            }
            if (MODE == 1 && (seg || fmg[j])) fmg[j] = seg;
          }
          anyg |= seg;
          my_flips += flip ? 1 : 0;
        }
      }
      anyg = __reduce_or_sync(0xffffffffu, anyg);
      if (lane == 0 && anyg) atomicOr(&s_any[g], anyg);
    }
  }
  pdl_trigger();
  __syncthreads();
  if (tid < A.G && s_any[tid]) atomicOr(&A.gs[tid].any, s_any[tid]);
  const unsigned long long flips_b = block_sum((unsigned long long)my_flips, s_red);
  if (tid == 0 && flips_b) atomicAdd(A.stats + 1, flips_b);
  const unsigned long long eval_b = block_sum((unsigned long long)my_eval, s_red) + s_eval;
  if (tid == 0 && eval_b) atomicAdd(A.stats + 5, eval_b);
}

// Warp sums of NV per-lane values at once: NV halving exchange steps leave
// each lane one value index, the remaining steps add across the other lanes;
// lane r < NV returns the warp total of v[r], lanes r >= NV return 0.
// 2 NV - 1 shuffles instead of NV * 5.
template <int NV>
__device__ __forceinline__ int64_t warp_sums_to_lanes(int64_t (&v)[NV], int lane) {
  constexpr int LOG = NV == 32 ? 5 : (NV == 16 ? 4 : (NV == 8 ? 3 : (NV == 4 ? 2 : (NV == 2 ? 1 : 0))));
  static_assert((1 << LOG) == NV, "NV must be a power of two <= 32");
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int o = 16 >> s;
    if (s < LOG) {
      const int h = NV >> (s + 1);
      const bool upper = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < NV / 2; ++i)
        if (i < h) {
          const int64_t send = upper ? v[i] : v[i + h];
          const int64_t keep = upper ? v[i + h] : v[i];
          v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    }
  }
  // lane L now holds the total of value index (L >> (5 - LOG)) & (NV - 1)
  const int64_t t = __shfl_sync(0xffffffffu, v[0], (lane << (5 - LOG)) & 31);
  return lane < NV ? t : 0;
}

// Energies of the lanes whose round ended (all lanes of the group at once,
// lane-parallel; exact int64 for integer couplings, exact 64-bit fixed point
// for FP32 couplings when InstDesc::ebase >= 0, else FP64), then - in the last
// CTA to finish - the round's bookkeeping: minima, best energies, the next
// descent's lanes.  Per-CTA partials are added in CTA order (deterministic).
template <bool FLOAT, int LPS, bool LAT>
__global__ void __launch_bounds__(kST, 4) sweep_energy(SweepArgs A) {
  __shared__ double s_red[kST / 32][32];
  __shared__ __align__(8) uint32_t s_stage[LAT ? (kST / 32) * 704 : 1];
  __shared__ bool s_last;
  const DevGraph &G = A.g;
  const InstDesc &I = A.I;
  const int n = I.n, L = I.lat_L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int ub = I.ebase;
  const bool fx = FLOAT && ub >= 0;
  pdl_prologue();
  bool any = false;
  for (int g = 0; g < A.G; ++g) any = any || A.gs[g].round_end || A.gs[g].final_pass;
  if (!any) return;
  constexpr int SPW = 32 / LPS;
  const int sub = lane / LPS, ln = lane % LPS;
  for (int g = 0; g < A.G; ++g) {
    const GroupState &S = A.gs[g];
    double accd = 0.0;
    long long acci = 0;
    unsigned long long accl = 0;
    if (S.round_end || S.final_pass) {
      const uint32_t *swg = A.sw + (size_t)g * n;
      if (LAT && !FLOAT && A.en_count) {
        // Multi-spin-coded lattice, site-parallel in site order: with J = +/-1
        // and h in {-1, 0, 1} every bond and nonzero field term is +1 when
        // unsatisfied and -1 otherwise, so E_r = 2 U_r - B with U_r the
        // unsatisfied terms of replica r and B the number of terms.  Lane = site
        // forms the unsatisfied masks of its forward bonds and field (bit r =
        // replica r) and adds them into bit-sliced per-lane counters; one
        // butterfly per warp then gives lane r the warp's U_r.
        constexpr int Q = 8;  // per-lane counts stay below 2^8 (host-checked: 4 terms x sites per lane)
        uint32_t cnt[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) cnt[q] = 0u;
        int nterms = 0;
        const int dl = I.lat_d;
        const int64_t so = I.spin_off;
        const int8_t *Jf8 = reinterpret_cast<const int8_t *>(G.Jfwd);
        const int8_t *h8 = reinterpret_cast<const int8_t *>(G.h);
        auto add_bit = [&](uint32_t m) {
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const uint32_t c = cnt[q] & m;
            cnt[q] ^= m;
            m = c;
          }
        };
        for (int base = (blockIdx.x * nw + warp) * 32; base < n; base += gridDim.x * nw * 32) {
          const int j = base + lane;
          if (j >= n) continue;
          int q1, q2;
          if (A.divL_m) {
            q1 = (int)(((uint64_t)j * A.divL_m) >> A.divL_k);
            q2 = (int)(((uint64_t)q1 * A.divL_m) >> A.divL_k);
          } else {
            q1 = j / L;
            q2 = q1 / L;
          }
          const int x = j - q1 * L, y = q1 - q2 * L;  // (z = q2)
          int nb[3];
          nb[0] = x == L - 1 ? j - (L - 1) : j + 1;
          nb[1] = y == L - 1 ? j - (L - 1) * L : j + L;
          nb[2] = q2 == L - 1 ? j - (L - 1) * L * L : j + L * L;
          const uint32_t wj = swg[j];
          uint32_t u[3];
          int neg[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            u[a] = 0u;
            neg[a] = 0;
            if (a < dl) {
              u[a] = swg[nb[a]];
              neg[a] = __ldg(Jf8 + (int64_t)a * G.nsp + so + j) < 0;
            }
          }
          const int hv = __ldg(h8 + so + j);
          // unsatisfied: J s s' < 0, i.e. (spins differ) xor (J < 0); -h s > 0
#pragma unroll
          for (int a = 0; a < 3; ++a)
            if (a < dl) add_bit(wj ^ u[a] ^ (neg[a] ? 0xffffffffu : 0u));
          if (hv != 0) add_bit(hv > 0 ? ~wj : wj);
          nterms += dl + (hv != 0 ? 1 : 0);
        }
        const long long U = warp_sliced_total<Q>(cnt, lane);  // lane r: replica r's warp total
        const long long B = (long long)warp_sum(nterms);
        acci = lane < LPS ? 2 * U - B : 0;  // (lanes beyond the group's replicas carry nothing)
      } else if (LAT && LPS <= 16 && A.en_fast && (!FLOAT || fx)) {
        // Lattice, site-parallel, in site order: lane = site j loads its word,
        // the words of its +x, +y (+z) neighbours (wrapping; every bond once,
        // from the site it leaves in the + direction), those bonds' couplings
        // and its field, all coalesced, forms their terms (fixed-point integers
        // or integers) and adds its part to each of the LPS replicas' int64
        // sums; one exchange per warp then gives lane r the warp total of
        // replica r.  Integer sums: the order does not matter.
        // Site j's part of E_r (its forward bonds and its field), with b the
        // spin bit (1 = +1) and d_a = b xor the +a neighbour's bit (1 = the
        // bond is not satisfied):  -h s - sum_a J_a s s_a
        //   = (h - sum_a J_a)  +  2 (sum_a d_a J_a - b h)   (terms in units),
        // so each replica only adds the terms its bits select; the site constant
        // is the same for every replica and is added once per lane.
        constexpr int NV = LPS <= 16 ? LPS : 16;
        int64_t acc[NV];
        int64_t csum = 0;
#pragma unroll
        for (int r = 0; r < NV; ++r) acc[r] = 0;
        const int dl = I.lat_d;
        const int64_t so = I.spin_off;
        for (int base = (blockIdx.x * nw + warp) * 32; base < n; base += gridDim.x * nw * 32) {
          const int j = base + lane;
          if (j >= n) continue;
          int q1, q2;
          if (A.divL_m) {
            q1 = (int)(((uint64_t)j * A.divL_m) >> A.divL_k);
            q2 = (int)(((uint64_t)q1 * A.divL_m) >> A.divL_k);
          } else {
            q1 = j / L;
            q2 = q1 / L;
          }
          const int x = j - q1 * L, y = q1 - q2 * L;  // (z = q2)
          int nb[3];
          nb[0] = x == L - 1 ? j - (L - 1) : j + 1;
          nb[1] = y == L - 1 ? j - (L - 1) * L : j + L;
          nb[2] = q2 == L - 1 ? j - (L - 1) * L * L : j + L * L;
          const uint32_t wj = swg[j];
          uint32_t d[3];
          int64_t tk[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            d[a] = 0u;
            tk[a] = 0;
            if (a < dl) {
              d[a] = swg[nb[a]];
              const int64_t jp = (int64_t)a * G.nsp + so + j;
              tk[a] = FLOAT ? xr_term(__ldg(reinterpret_cast<const float *>(G.Jfwd) + jp), ub)
                            : (int64_t)__ldg(reinterpret_cast<const int8_t *>(G.Jfwd) + jp);
            }
          }
          const int64_t th = FLOAT ? xr_term(__ldg(reinterpret_cast<const float *>(G.h) + so + j), ub)
                                   : (int64_t)__ldg(reinterpret_cast<const int8_t *>(G.h) + so + j);
          int64_t c = th;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (a >= dl) break;
            const uint32_t da = wj ^ d[a];
            c -= tk[a];
#pragma unroll
            for (int r = 0; r < NV; ++r)
              if ((da >> r) & 1u) acc[r] += tk[a];
          }
          csum += c;
#pragma unroll
          for (int r = 0; r < NV; ++r)
            if ((wj >> r) & 1u) acc[r] -= th;
        }
#pragma unroll
        for (int r = 0; r < NV; ++r) acc[r] = 2 * acc[r] + csum;
        const int64_t tot = warp_sums_to_lanes<NV>(acc, lane);
        if (FLOAT) {
          acci = (long long)(tot >> 32);
          accl = (unsigned long long)(uint32_t)tot;
        } else {
          acci = (long long)tot;
        }
      } else if constexpr (LAT) {
        // Lattice: lane = position stages the position's word, its forward
        // neighbours' words (those with a larger index, so each bond counts
        // once) and its terms - fixed-point integers, FP32 values or integers -
        // in shared memory in one round trip; the per-replica steps then read
        // shared memory only.
        uint32_t *sW = s_stage + warp * 704;      // [32] words
        uint32_t *sN = sW + 32;                   // [6][32] forward neighbour words
        uint32_t *sT = sW + 224;                  // [7][32] x 2: terms (kk 0..5, field)
        uint32_t *sM = sW + 672;                  // [32] forward mask
        for (int base = (blockIdx.x * nw + warp) * 32; base < n; base += gridDim.x * nw * 32) {
          const int v1 = base + lane;
          if (v1 < n) {
            const int j1 = __ldg(G.order + I.spin_off + v1);
            const uint32_t meta1 = __ldg(G.meta + I.spin_off + v1);
            sW[lane] = swg[j1];
            uint32_t fwd = 0u;
#pragma unroll
            for (int kk = 0; kk < 6; ++kk)
              if (kk < 2 * I.lat_d) {
                const int i = lat_nbr(j1, meta1, kk, L);
                if (i > j1) {
                  fwd |= 1u << kk;
                  sN[kk * 32 + lane] = swg[i];
                  const int64_t jp = (int64_t)kk * G.nsp + I.spin_off + v1;
                  int64_t t;
                  if (FLOAT) {
                    const float w = __ldg(reinterpret_cast<const float *>(G.Jpos) + jp);
                    t = fx ? xr_term(w, ub) : (int64_t)__float_as_uint(w);
                  } else {
                    t = __ldg(reinterpret_cast<const int8_t *>(G.Jpos) + jp);
                  }
                  reinterpret_cast<int64_t *>(sT)[kk * 32 + lane] = t;
                }
              }
            int64_t th;
            if (FLOAT) {
              const float hv = __ldg(reinterpret_cast<const float *>(G.h) + I.spin_off + j1);
              th = fx ? xr_term(hv, ub) : (int64_t)__float_as_uint(hv);
            } else {
              th = __ldg(reinterpret_cast<const int8_t *>(G.h) + I.spin_off + j1);
            }
            reinterpret_cast<int64_t *>(sT)[6 * 32 + lane] = th;
            sM[lane] = fwd;
          }
          __syncwarp();
          const int cnt = min(32, n - base);
          for (int src = sub; src < cnt; src += SPW) {
            const uint32_t bj = (sW[src] >> ln) & 1u;
            const uint32_t fwd = sM[src];
            const int64_t *T = reinterpret_cast<const int64_t *>(sT);
            if (FLOAT && fx) {
              const int64_t th = T[6 * 32 + src];
              xe_add(acci, accl, bj ? -th : th);
#pragma unroll
              for (int kk = 0; kk < 6; ++kk)
                if ((fwd >> kk) & 1u) {
                  const int64_t t = T[kk * 32 + src];
                  xe_add(acci, accl, (((sN[kk * 32 + src] >> ln) & 1u) ^ bj) ? t : -t);
                }
            } else if (FLOAT) {
              const double hv = (double)__uint_as_float((uint32_t)T[6 * 32 + src]);
              double e = bj ? hv : -hv;
#pragma unroll
              for (int kk = 0; kk < 6; ++kk)
                if ((fwd >> kk) & 1u) {
                  const double w = (double)__uint_as_float((uint32_t)T[kk * 32 + src]);
                  e += (((sN[kk * 32 + src] >> ln) & 1u) ^ bj) ? -w : w;
                }
              accd -= e;
            } else {
              const int hv = (int)T[6 * 32 + src];
              int e = bj ? hv : -hv;
#pragma unroll
              for (int kk = 0; kk < 6; ++kk)
                if ((fwd >> kk) & 1u) {
                  const int w = (int)T[kk * 32 + src];
                  e += (((sN[kk * 32 + src] >> ln) & 1u) ^ bj) ? -w : w;
                }
              acci -= e;
            }
          }
          __syncwarp();
        }
      } else {
      // 32 positions per warp step: one coalesced read of their site indices
        // and lattice metadata, then SPW sites at a time, several steps unrolled
        // so that their neighbour reads are in flight together
        for (int base = (blockIdx.x * nw + warp) * 32; base < n; base += gridDim.x * nw * 32) {
          const int v1 = base + lane;
          const int j1 = v1 < n ? ((LAT && !A.sequential) ? __ldg(G.order + I.spin_off + v1) : v1) : 0;
          const uint32_t meta1 = (LAT && v1 < n) ? __ldg(G.meta + I.spin_off + v1) : 0u;
  #pragma unroll 4
        for (int st = 0; st < 32 / SPW; ++st) {
          const int src = st * SPW + sub;
          const int v = base + src;
          const int j = __shfl_sync(0xffffffffu, j1, src);
          const uint32_t meta = __shfl_sync(0xffffffffu, meta1, src);
          if (v >= n) continue;
          const int64_t gj = I.spin_off + j;
          const uint32_t bj = (swg[j] >> ln) & 1u;
          const uint32_t k0 = LAT ? 0u : __ldg(G.row + gj);
          const uint32_t k1 = LAT ? (uint32_t)(2 * I.lat_d) : __ldg(G.row + gj + 1);
          if (FLOAT) {
            const float hv = __ldg(reinterpret_cast<const float *>(G.h) + gj);
            double e = bj ? (double)hv : -(double)hv;
            if (fx) {
              const int64_t th = xr_term(hv, ub);
              xe_add(acci, accl, bj ? -th : th);
            }
            for (uint32_t kk = k0; kk < k1; ++kk) {
              int i;
              float w;
              if (LAT) {
                i = lat_nbr(j, meta, (int)kk, L);
                w = __ldg(reinterpret_cast<const float *>(G.Jpos) + (int64_t)kk * G.nsp + I.spin_off + v);
              } else {
                i = __ldg(G.col + kk);
                w = __ldg(reinterpret_cast<const float *>(G.J) + kk);
              }
              if (i > j) {
                const bool differ = ((swg[i] >> ln) & 1u) ^ bj;
                if (fx) {
                  const int64_t t = xr_term(w, ub);
                  xe_add(acci, accl, differ ? t : -t);
                } else {
                  e += differ ? -(double)w : (double)w;
                }
              }
            }
            if (!fx) accd -= e;
          } else {
            const int hv = __ldg(reinterpret_cast<const int8_t *>(G.h) + gj);
            int e = bj ? hv : -hv;
            for (uint32_t kk = k0; kk < k1; ++kk) {
              int i, w;
              if (LAT) {
                i = lat_nbr(j, meta, (int)kk, L);
                w = __ldg(reinterpret_cast<const int8_t *>(G.Jpos) + (int64_t)kk * G.nsp + I.spin_off + v);
              } else {
                i = __ldg(G.col + kk);
                w = __ldg(reinterpret_cast<const int8_t *>(G.J) + kk);
              }
              if (i > j) e += (((swg[i] >> ln) & 1u) ^ bj) ? -w : w;
            }
            acci -= e;
          }
        }
        }
      }
      // hyper-edges (CSR instances only)
      for (int64_t wi = (int64_t)blockIdx.x * nw + warp; wi < (I.n_hyper + SPW - 1) / SPW;
           wi += (int64_t)gridDim.x * nw) {
        const int e = (int)(wi * SPW + sub);
        if (e >= I.n_hyper) continue;
        const int64_t ge = I.hyper_off + e;
        uint32_t neg = 0;
        for (uint32_t q = __ldg(G.hptr + ge), qe = __ldg(G.hptr + ge + 1); q < qe; ++q)
          neg ^= ~(swg[__ldg(G.hmem + q)] >> ln) & 1u;
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
    }
    // lanes of the SPW sub-warps hold different spins of the same replica: fold them
    for (int o = LPS; o < 32; o <<= 1) {
      accd += __shfl_xor_sync(0xffffffffu, accd, o);
      acci += __shfl_xor_sync(0xffffffffu, acci, o);
      accl += __shfl_xor_sync(0xffffffffu, accl, o);
    }
    if (!(S.round_end || S.final_pass)) continue;  // (uniform across the grid)
    const bool dbl = FLOAT && !fx;
    long long *ri = reinterpret_cast<long long *>(&s_red[0][0]);
    __syncthreads();
    if (dbl) s_red[warp][lane] = accd;
    else ri[warp * 32 + lane] = acci;
    __syncthreads();
    if (warp == 0) {
      double a = 0.0;
      long long b = 0;
      for (int w = 0; w < nw; ++w) {
        if (dbl) a = w == 0 ? s_red[0][lane] : a + s_red[w][lane];
        else b += ri[w * 32 + lane];
      }
      if (dbl) A.partial[((size_t)blockIdx.x * A.G + g) * 32 + lane] = a;
      else if (b) atomicAdd(A.eacc + ((size_t)g * 32 + lane) * 2, (unsigned long long)b);
    }
    if (fx) {
      __syncthreads();
      reinterpret_cast<unsigned long long *>(ri)[warp * 32 + lane] = accl;
      __syncthreads();
      if (warp == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < nw; ++w) b += reinterpret_cast<unsigned long long *>(ri)[w * 32 + lane];
        if (b) atomicAdd(A.eacc + ((size_t)g * 32 + lane) * 2 + 1, b);
      }
    }
    __syncthreads();
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(A.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last CTA: totals in CTA order, then per-group bookkeeping
  for (int g = 0; g < A.G; ++g) {
    GroupState &S = A.gs[g];
    if (!(S.round_end || S.final_pass)) continue;
    if (FLOAT && !fx) {
      // FP64: warp w adds the partials of CTAs w, w + nw, ... (fixed order),
      // then warp 0 adds the warps' sums in ascending order: deterministic
      double a = 0.0;
      // (independent loads: unrolled so that several are in flight at once;
      // the additions keep their order)
#pragma unroll 8
      for (int cta = warp; cta < (int)gridDim.x; cta += nw) a += A.partial[((size_t)cta * A.G + g) * 32 + lane];
      __syncthreads();
      s_red[warp][lane] = a;
      __syncthreads();
      if (warp == 0) {
        double t = s_red[0][lane];
        for (int w = 1; w < nw; ++w) t += s_red[w][lane];
        S.E[lane] = t;
      }
    } else if (warp == 0) {
      // integer sums: take the totals and leave zeros for the next pass
      unsigned long long *ea = A.eacc + ((size_t)g * 32 + lane) * 2;
      const long long hi = (long long)atomicExch(ea, 0ull);
      if (fx) S.E[lane] = xe_value(hi, atomicExch(ea + 1, 0ull), ub);
      else S.E[lane] = (double)hi;
    }
    __syncthreads();
    if (warp == 0) {
      // lane = replica: minima, best energies and the next descent's lanes
      if (S.final_pass) {
        __syncwarp();
        if (lane == 0) S.final_pass = 0;
      } else {
        const uint32_t cr = S.convround;
        bool better = false;
        if ((cr >> lane) & 1u) {
          S.minima[lane] += 1;
          const double e = S.E[lane];
          if (e < S.best[lane]) {
            S.best[lane] = e;
            better = true;
          }
        }
        const uint32_t upd = __ballot_sync(0xffffffffu, better);
        const int k1 = S.k + 1;
        const bool go = k1 < A.restarts && ((S.lane_valid >> lane) & 1u) && (A.budget <= 0 || S.total[lane] < A.budget);
        const uint32_t start = __ballot_sync(0xffffffffu, go);
        __syncwarp();  // every lane has read the group state before lane 0 rewrites it
        if (lane == 0) {
          S.upd = upd;
          S.k = k1;
          S.start = start;
          S.active = start;
          S.convround = 0;
          S.d = 0;
          S.round_end = 0;
          if (!start) S.done = 1;
          atomicAdd(A.stats + 3, (unsigned long long)__popc(start));
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    int all = 1;
    for (int g = 0; g < A.G; ++g) all = all && A.gs[g].done;
    *A.all_done = all;
    *A.counter = 0;
  }
}

// Best-state copies and random starts decided by the last bookkeeping pass.
// One warp owns 32 / LPS consecutive blocks of 128 sites: it first copies the
// improved lanes' current words into the best-state words, then draws the new
// starts for the same sites, so the copy never sees a new start.
template <int LPS>
__global__ void __launch_bounds__(kST) sweep_restart(SweepArgs A) {
  pdl_prologue();
  const int n = A.I.n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int g = 0; g < A.G; ++g) {
    const GroupState &S = A.gs[g];
    const uint32_t upd = S.upd, start = S.start;
    if (!(upd | start)) continue;
    const int nwb = (n + 127) / 128;
    uint32_t *swg = A.sw + (size_t)g * n;
    uint32_t *bwg = A.bw + (size_t)g * n;
    uint32_t *fmg = A.fm + (size_t)g * n;
    // One warp step covers P = 32 / LPS blocks of 128 sites: lane l draws the
    // bits of replica l % LPS for block w0 + l / LPS, so that a warp transpose
    // of the 32 lanes' words hands lane u, in bit field j, the word of site u of
    // the same 32-site quarter of block w0 + j.
    constexpr int P = 32 / LPS;
    constexpr uint32_t lmask = LPS == 32 ? 0xffffffffu : ((1u << LPS) - 1u);
    for (int w0 = (blockIdx.x * nw + warp) * P; w0 < nwb; w0 += gridDim.x * nw * P) {
      if (upd)
        for (int t = lane; t < 128 * P; t += 32) {
          const int i = w0 * 128 + t;
          if (i < n) bwg[i] = (bwg[i] & ~upd) | (swg[i] & upd);
        }
      __syncwarp();
      if (start) {
        const int wl = w0 + lane / LPS, rl = lane % LPS;
        const uint4 x = (wl < nwb && ((start >> rl) & 1u))
                            ? start_bits(A.seed, (uint32_t)wl, (uint32_t)(32 * g + rl), (uint32_t)S.k, (uint32_t)A.b)
                            : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t mine = warp_transpose32(word_of(x, q), lane);  // field j: site u of block w0 + j
#pragma unroll
          for (int j = 0; j < P; ++j) {
            const int i = (w0 + j) * 128 + q * 32 + lane;
            if (i < n) {
              const uint32_t word = (mine >> (j * LPS)) & lmask;
              swg[i] = (swg[i] & ~start) | (word & start);
              const uint32_t f = fmg[i];
              if (f & start) fmg[i] = f & ~start;
            }
          }
        }
      }
      __syncwarp();
    }
  }
}

__global__ void sweep_mark_final(SweepArgs A) {
  const int g = threadIdx.x;
  if (g >= A.G) return;
  GroupState &S = A.gs[g];
  uint32_t need = 0;
  for (int r = 0; r < 32; ++r)
    if (((S.lane_valid >> r) & 1u) && S.minima[r] == 0) need |= 1u << r;
  S.final_pass = need ? 1 : 0;
  if (threadIdx.x == 0) *A.counter = 0;
}

__global__ void sweep_output(SweepArgs A) {
  const int n = A.I.n;
  const int64_t tot = (int64_t)A.R * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / n), i = (int)(t % n);
    const int g = r / 32, l = r % 32;
    const GroupState &S = A.gs[g];
    const uint32_t w = S.minima[l] > 0 ? A.bw[(size_t)g * n + i] : A.sw[(size_t)g * n + i];
    A.spins[(int64_t)A.R * A.I.spin_off + t] = ((w >> l) & 1u) ? 1 : -1;
  }
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < A.R) {
    const int g = (int)t / 32, l = (int)t % 32;
    const GroupState &S = A.gs[g];
    const double e = S.minima[l] > 0 ? S.best[l] : S.E[l];
    const int64_t o = (int64_t)A.b * A.R + t;
    A.energy[o] = e;
    if (A.energy_i32) A.energy_i32[o] = (int32_t)e;
    if (A.minima) A.minima[o] = S.minima[l];
  }
}

struct SweepGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

struct SweepState : FamilyState {
  size_t bytes = 0;
  void *mem = nullptr;
  int32_t *h_done = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::map<std::string, SweepGraph> graphs;  // instantiated sweep chunks by configuration
};


// ISING_SWEEP_DEBUG=1: launch without graphs, synchronise and report after
// every launch (diagnostics only).
bool sweep_debug() {
  static const int on = [] {
    const char *v = std::getenv("ISING_SWEEP_DEBUG");
    return v && v[0] == '1' ? 1 : 0;
  }();
  return on != 0;
}

void debug_step(const char *what, int c, cudaStream_t s) {
  if (!sweep_debug()) return;
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaStreamSynchronize(s);
  std::fprintf(stderr, "[sweep] %s %d: launch=%s sync=%s\n", what, c, cudaGetErrorString(e1), cudaGetErrorString(e2));
  std::fflush(stderr);
}

constexpr size_t visit_smem(int, int, bool) {
  return 0;  // the visits keep their per-position data in registers
}

// Launch, with programmatic stream serialization when pdl is set (see
// pdl_prologue); a launch error is left for the caller's cudaGetLastError.
template <typename... KArgs, typename... Args>
void launch_pdl(bool pdl, void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int MODE, int LPS, bool LAT>
void enqueue_visit(const SweepArgs &A, int c, int grid, cudaStream_t s) {
  launch_pdl(A.pdl != 0, sweep_visit<MODE, LPS, LAT>, grid, kST, visit_smem(MODE, LPS, LAT), s, A, (int32_t)c);
  debug_step("visit", c, s);
}

template <int LPS, bool LAT>
void enqueue_round_end(const SweepArgs &A, int mode, cudaStream_t s) {
  if (mode == 1) launch_pdl(A.pdl != 0, sweep_energy<true, LPS, LAT>, A.grid_e, kST, 0, s, A);
  else launch_pdl(A.pdl != 0, sweep_energy<false, LPS, LAT>, A.grid_e, kST, 0, s, A);
  debug_step("energy", 0, s);
  launch_pdl(A.pdl != 0, sweep_restart<LPS>, A.grid_e, kST, 0, s, A);
  debug_step("restart", 0, s);
}

template <int LPS, bool LAT>
void enqueue_sweep(const SweepArgs &A, int mode, int ncls, int grid_v, cudaStream_t s, bool round_end = true) {
  for (int c = 0; c < ncls; ++c) {
    if (mode == 0) enqueue_visit<0, LPS, LAT>(A, c, grid_v, s);
    else if (mode == 1) enqueue_visit<1, LPS, LAT>(A, c, grid_v, s);
    else enqueue_visit<2, LPS, LAT>(A, c, grid_v, s);
  }
  launch_pdl(A.pdl != 0, sweep_end, (A.G + 7) / 8, 256, 0, s, A);
  debug_step("end", 0, s);
  if (round_end) enqueue_round_end<LPS, LAT>(A, mode, s);
}

// Load every kernel of this configuration before any graph capture, so the
// capture never triggers module loading.
template <int LPS, bool LAT>
cudaError_t preload(int mode) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaSuccess;
  if (mode == 0) e = cudaFuncGetAttributes(&fa, sweep_visit<0, LPS, LAT>);
  else if (mode == 1) {
    e = cudaFuncSetAttribute(sweep_visit<1, LPS, LAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)visit_smem(1, LPS, LAT));
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, sweep_visit<1, LPS, LAT>);
  }
  else e = cudaFuncGetAttributes(&fa, sweep_visit<2, LPS, LAT>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, sweep_end);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, sweep_energy<true, LPS, LAT>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, sweep_energy<false, LPS, LAT>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, sweep_restart<LPS>);
  return e;
}

// Resident CTAs per SM of the visit kernel of this configuration.
template <int LPS, bool LAT>
int visit_ctas_per_sm(int mode) {
  int k = 0;
  cudaError_t e;
  if (mode == 0)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, sweep_visit<0, LPS, LAT>, kST, visit_smem(0, LPS, LAT));
  else if (mode == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, sweep_visit<1, LPS, LAT>, kST, visit_smem(1, LPS, LAT));
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, sweep_visit<2, LPS, LAT>, kST, visit_smem(2, LPS, LAT));
  return (e == cudaSuccess && k > 0) ? k : 8;
}

template <int LPS, bool LAT>
cudaError_t run_instance(ising_handle *h, SweepArgs A, int mode, cudaStream_t s) {
  SweepState &S = family_state<SweepState>(h->sweep_st);
  const InstDesc &I = A.I;
  const int ncls = A.sequential ? I.n : I.ncls;
  int maxcls = 1;
  if (A.sequential) maxcls = 1;
  else
    for (int c = 0; c < I.ncls; ++c)
      maxcls = std::max(maxcls, h->h_cls[I.cls_off + c + 1] - h->h_cls[I.cls_off + c]);
  const int64_t items = mode == 2 ? (int64_t)A.G * maxcls : (int64_t)A.G * ((maxcls + 32 / LPS - 1) / (32 / LPS)) * 32;
  cudaError_t e0 = preload<LPS, LAT>(mode);
  if (e0 != cudaSuccess) return e0;
  // one wave of resident CTAs at most: the visits loop over their positions,
  // so a larger grid only adds CTA start-up and barrier cost per visit
  const int grid_v = (int)std::max<int64_t>(
      1, std::min<int64_t>((items + kST - 1) / kST, (int64_t)h->sm_count * visit_ctas_per_sm<LPS, LAT>(mode)));
  if (sweep_debug())
    std::fprintf(stderr, "[sweep] n=%d ncls=%d G=%d LPS=%d mode=%d grid_v=%d grid_e=%d lattice=%d seq=%d\n", I.n,
                 ncls, A.G, LPS, mode, grid_v, A.grid_e, A.lattice, A.sequential);
  sweep_init<<<1, 32, 0, s>>>(A);
  debug_step("init", 0, s);
  sweep_restart<LPS><<<A.grid_e, kST, 0, s>>>(A);
  h->launches += 2;
  debug_step("restart0", 0, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // The round-end kernels (energy pass, restarts) follow every kRoundEnd-th
  // sweep of a captured chunk: most of their launches find no round ended, and
  // a group whose round ended only waits (no active lane: it visits and counts
  // nothing) until they come.
  constexpr int kRoundEnd = 4;
  // upper bound on the sweeps any group can need
  // (each round may wait kRoundEnd - 1 sweeps for its round-end kernels)
  int64_t max_sweeps_total = (int64_t)A.restarts * (A.max_sweeps + kRoundEnd) + A.restarts;
  if (A.budget > 0)
    max_sweeps_total =
        std::min<int64_t>(max_sweeps_total, (int64_t)A.R * A.budget * kRoundEnd + A.max_sweeps + kRoundEnd);
  // Capture a chunk of sweeps once per configuration (cached) and replay it
  // until every group is done, polling a done flag one chunk behind so the GPU
  // always has queued work.  A graph holds at most kMaxNodes launches; when one
  // sweep alone needs more (many colour classes, e.g. the sequential schedule)
  // sweeps are launched directly instead.  (A device-side loop - a conditional
  // WHILE node, optionally with an IF node around the round-end kernels - was
  // measured slightly slower on GB300, and its kernels are not visible to ncu.)
  constexpr int kMaxNodes = 512;
  const int per_sweep = ncls + 3;
  const bool use_graph = per_sweep <= kMaxNodes && !sweep_debug();
  const int chunk = use_graph ? std::max(1, std::min(16, kMaxNodes / per_sweep)) : 1;
  // the first sweep runs with direct launches, the rest from the graph
  enqueue_sweep<LPS, LAT>(A, mode, ncls, grid_v, s);
  h->launches += per_sweep;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cudaGraphExec_t exec = nullptr;
  if (use_graph) {
    // everything the captured launches bake in besides the handle's own arrays
    char key[320];
    std::snprintf(key, sizeof key, "%d/%d/%d/%d/%d/%d/%d/%d/%d/%d/%llu/%p/%d/%d/%d/%d/%p/%d/%d", A.b, A.R, A.G, A.LPS,
                  A.max_sweeps, A.restarts, A.budget, A.refresh, A.sequential, A.lattice,
                  (unsigned long long)A.seed, (void *)A.sw, mode, grid_v, chunk, ncls, (void *)A.cflag, A.nchunk,
                  A.en_fast + 2 * A.en_count);
    auto it = S.graphs.find(key);
    if (it == S.graphs.end()) {
      SweepGraph sg;
      cudaStream_t cs = nullptr;
      if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return e;
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        for (int k = 0; k < chunk; ++k)
          enqueue_sweep<LPS, LAT>(A, mode, ncls, grid_v, cs, (k % kRoundEnd) == kRoundEnd - 1 || k == chunk - 1);
        e = cudaStreamEndCapture(cs, &sg.graph);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&sg.exec, sg.graph, 0);
      cudaStreamDestroy(cs);
      if (e != cudaSuccess) {
        if (sg.graph) cudaGraphDestroy(sg.graph);
        return e;
      }
      it = S.graphs.emplace(key, sg).first;
    }
    exec = it->second.exec;
  }
  const int64_t max_chunks = max_sweeps_total / chunk + 2;
  int64_t launched = 0;
  for (;;) {
    // sweeps of a captured chunk without round-end kernels launch two fewer
    int with_re = 0;
    for (int k = 0; k < chunk; ++k) with_re += ((k % kRoundEnd) == kRoundEnd - 1 || k == chunk - 1) ? 1 : 0;
    h->launches += (uint64_t)chunk * per_sweep - (use_graph ? (uint64_t)(chunk - with_re) * 2 : 0);
    kt_begin(h, "sweep_chunk", s);
    if (use_graph) {
      if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) break;
    } else {
      enqueue_sweep<LPS, LAT>(A, mode, ncls, grid_v, s);
      if ((e = cudaGetLastError()) != cudaSuccess) break;
    }
    kt_end(h, s);
    cudaMemcpyAsync(S.h_done + (launched & 1), A.all_done, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaEventRecord(S.ev[launched & 1], s);
    ++launched;
    if (sweep_debug()) std::fprintf(stderr, "[sweep] chunk %lld queued\n", (long long)launched);
    if (launched >= 2) {
      // look one chunk behind so the GPU always has queued work
      cudaEventSynchronize(S.ev[launched & 1]);
      if (S.h_done[launched & 1]) break;
    }
    if (launched >= max_chunks) break;
  }
  if (e != cudaSuccess) return e;
  // energies of the final states of replicas that never converged
  sweep_mark_final<<<1, 32, 0, s>>>(A);
  h->launches += 3;
  if (mode == 1) sweep_energy<true, LPS, LAT><<<A.grid_e, kST, 0, s>>>(A);
  else sweep_energy<false, LPS, LAT><<<A.grid_e, kST, 0, s>>>(A);
  const int64_t tot = (int64_t)A.R * I.n;
  sweep_output<<<(int)std::min<int64_t>((tot + kST - 1) / kST, (int64_t)h->sm_count * 16), kST, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace

void sweep_free(ising_handle *h) {
  if (!h->sweep_st) return;
  SweepState &S = static_cast<SweepState &>(*h->sweep_st);
  for (auto &kv : S.graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    cudaGraphDestroy(kv.second.graph);
  }
  cudaFree(S.mem);
  if (S.h_done) cudaFreeHost(S.h_done);
  for (auto &e : S.ev)
    if (e) cudaEventDestroy(e);
  h->sweep_st.reset();
}

cudaError_t launch_sweep(ising_handle *h, const ising_search_params *p, int32_t R, int8_t *spins, double *E,
                         int32_t *E32, int32_t *minima, const uint64_t *seeds_host, cudaStream_t s) {
  SweepState &S = family_state<SweepState>(h->sweep_st);
  const int LPS = R > 16 ? 32 : (R > 8 ? 16 : 8);
  const int G = (R + 31) / 32;
  if (LPS < 32 && R > LPS) return cudaErrorInvalidValue;
  const bool fl = h->dtype == ISING_F32;
  const int mode = fl ? 1 : (h->msc_ok ? 2 : 0);
  const int grid_e = h->sm_count * 4;
  // scratch: sw, fm, bw, pend [G][nmax]; F [G][nmax][LPS]; gs [G]; partial [grid_e][G][32]; eacc [G][32][2];
  // counter; done
  const size_t words = (size_t)G * h->nmax;
  auto up256 = [](size_t b) { return (b + 255) / 256 * 256; };
  const int32_t nchunk = (h->nmax / 2 + 31) / 32 + 1;
  const size_t cflag_bytes = (size_t)G * 2 * nchunk * sizeof(uint16_t);
  const size_t need = 4 * up256(words * 4) + (fl ? up256(words * LPS * 4) : 0) + up256(G * sizeof(GroupState)) +
                      up256((size_t)grid_e * G * 32 * 8) + up256((size_t)G * 32 * 16) + 2 * 256 +
                      up256(cflag_bytes);
  cudaError_t e;
  if (need > S.bytes) {
    for (auto &kv : S.graphs) {  // captured against the old scratch
      cudaGraphExecDestroy(kv.second.exec);
      cudaGraphDestroy(kv.second.graph);
    }
    S.graphs.clear();
    cudaFree(S.mem);
    S.mem = nullptr;
    S.bytes = 0;
    if ((e = cudaMalloc(&S.mem, need)) != cudaSuccess) return e;
    S.bytes = need;
  }
  if (!S.h_done && (e = cudaMallocHost(&S.h_done, 2 * sizeof(int32_t))) != cudaSuccess) return e;
  for (auto &ev : S.ev)
    if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
  char *base = (char *)S.mem;
  auto take = [&](size_t bytes) {
    char *p0 = base;
    base += (bytes + 255) / 256 * 256;
    return (void *)p0;
  };
  SweepArgs A;
  A.g = h->graph();
  A.R = R;
  A.G = G;
  A.LPS = LPS;
  A.max_sweeps = p->max_sweeps;
  A.restarts = p->restarts;
  A.budget = p->sweep_budget;
  A.refresh = p->refresh_every;
  A.sequential = p->schedule == ISING_SCHED_SEQUENTIAL ? 1 : 0;
  A.sw = (uint32_t *)take(words * 4);
  A.fm = (uint32_t *)take(words * 4);
  A.bw = (uint32_t *)take(words * 4);
  A.pend = (uint32_t *)take(words * 4);
  A.F = fl ? (float *)take(words * LPS * 4) : nullptr;
  A.gs = (GroupState *)take(G * sizeof(GroupState));
  A.grid_e = grid_e;
  A.partial = (double *)take((size_t)grid_e * G * 32 * 8);
  A.eacc = (unsigned long long *)take((size_t)G * 32 * 16);
  A.counter = (unsigned int *)take(64);
  A.all_done = (int32_t *)take(64);
  uint16_t *cflag_mem = (uint16_t *)take(cflag_bytes);
  A.nchunk = nchunk;
  A.stats = h->d_stats;
  A.spins = spins;
  A.energy = E;
  A.energy_i32 = E32;
  A.minima = minima;
  for (int32_t b = 0; b < h->n_inst; ++b) {
    A.I = h->inst[b];
    A.b = b;
    A.seed = seeds_host[b];
    A.lattice = (A.I.lat_d > 0 && !A.sequential) ? 1 : 0;
    {
      // site-parallel energies: at most `per_warp` terms, each below 2^ebits,
      // go into one int64 before the high/low split of the block reduction
      const int64_t sites_lane = ((int64_t)A.I.n + (int64_t)grid_e * kST - 1) / ((int64_t)grid_e * kST);
      const int64_t per_warp = 32 * sites_lane * (A.I.lat_d + 1);
      int lg = 0;
      while (((int64_t)1 << lg) <= per_warp) ++lg;
      // (the lane sums are doubled and offset by the site constants: one more bit)
      A.en_fast = (A.lattice && LPS <= 16 && A.I.ebits >= 0 && A.I.ebits + lg + 1 <= 62) ? 1 : 0;
      // bit-sliced counts: at most 4 terms per site, sites_lane sites per lane, below 2^8
      A.en_count = (A.lattice && mode == 2 && 4 * sites_lane <= 255) ? 1 : 0;
      A.pdl = mode == 2 ? 1 : 0;
    }
    if ((e = cudaMemsetAsync(A.fm, 0, words * 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(A.eacc, 0, (size_t)G * 32 * 16, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(A.pend, 0, words * 4, s)) != cudaSuccess) return e;
    // chunk flags: the two-class parity colouring of an even-sided lattice puts
    // site j at class position j >> 1 (class order is index order)
    // (FP32 lattices only: in the multi-spin-coded visits, a thread per site,
    // the flag traffic measured slower than the scan it saves)
    const bool chunked = A.lattice && h->lat_parity && A.I.ncls == 2 && A.I.lat_L % 2 == 0 && mode == 1;
    A.divL_m = 0;
    A.divL_k = 0;
    if (A.lattice && A.I.n <= (1 << 24)) {
      // q = floor(x / L) for 0 <= x < 2^24 as (x m) >> k with m = ceil(2^k / L),
      // k = 24 + ceil(log2 L): the error term x (m L - 2^k) / (L 2^k) stays below 1 / L
      int lg = 0;
      while ((1 << lg) < A.I.lat_L) ++lg;
      A.divL_k = 24 + lg;
      A.divL_m = (((uint64_t)1 << A.divL_k) + (uint64_t)A.I.lat_L - 1) / (uint64_t)A.I.lat_L;
    }
    // (the flagged visits find their sites by that division)
    A.cflag = (chunked && A.divL_m) ? cflag_mem : nullptr;
    if (A.cflag && (e = cudaMemsetAsync(cflag_mem, 0, cflag_bytes, s)) != cudaSuccess) return e;
    if (A.lattice) {
      if (LPS == 32) e = run_instance<32, true>(h, A, mode, s);
      else if (LPS == 16) e = run_instance<16, true>(h, A, mode, s);
      else e = run_instance<8, true>(h, A, mode, s);
    } else {
      if (LPS == 32) e = run_instance<32, false>(h, A, mode, s);
      else if (LPS == 16) e = run_instance<16, false>(h, A, mode, s);
      else e = run_instance<8, false>(h, A, mode, s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace isg
