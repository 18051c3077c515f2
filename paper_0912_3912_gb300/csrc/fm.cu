// fm.cu — the paper's pass-based local search with hill climbing (Sec. IV,
// Fig. 3) for instances of up to 4096 spins.
//
// From each random start (Philox, the counter layout of ising_local_search)
// the search runs passes.  A pass computes every spin's gain -2 s_i f_i, then
// n times: takes the largest gain among the spins not yet moved in this pass
// (ties to the lowest index), applies that move even when the gain is
// negative (hill climbing), locks the spin, updates its neighbours' fields,
// and records the prefix whose running energy is strictly the lowest so far
// (the earliest such prefix).  The pass is then rolled back to that prefix; a
// new pass follows while the pass lowered the energy strictly (for float
// couplings by more than 1e-9 relative, so FP64 rounding cannot fake an
// improvement), else the pass's start is the result.
//
// The values are those of FP64 arithmetic in the definition's order: fields
// summed as h_i, then the CSR row in stored order, then the incident
// hyper-edges in ascending edge order; a move of spin i adds 2 J_ij s_i to its
// CSR neighbours' fields and each incident hyper-edge's term to its other
// members.  Where FP64 computes an instance's values exactly, the kernels hold
// them as 64-bit integers (one unit per instance, or per spin), with the same
// results and no FP64 on the per-move path.
//
// One warp per search.  The paper keeps the gains in a heap (Fig. 4);
// fm_kernel keeps per-warp maxima of 32-spin blocks in shared memory and takes
// the move's spin by warp reductions over them (gains compared as
// order-preserving integers); fm_reg_kernel holds a small instance's fields in
// the lanes' registers.  Both select the heap's spin.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdlib>
#include <map>
#include <type_traits>
#include <vector>

#include "device_common.cuh"

namespace isg {

namespace {

constexpr int kFT = 256;           // threads per CTA
constexpr int kFW = kFT / 32;
constexpr int kFmMaxSpins = 4096;
// arithmetic of a search (InstDesc::fx53): FP64 as defined; int64 in one unit
// per instance; int64 fields in per-spin units with FP64 energies
constexpr int kFp64 = 0, kFx = 1, kFxSpin = 2;
// a move that changes more fields than this recomputes every block maximum
constexpr int kTouched = 64;

struct FmArgs {
  DevGraph g;
  int32_t n_work, R_out, restarts, max_passes;
  int32_t split;              // 1: one start per work unit (work = item * restarts + start)
  const int2 *items;          // (instance, replica), largest instances first
  const uint64_t *seeds;      // [instances]
  int32_t *queue;
  int8_t *spins;              // [instance block: R_out x n] results
  double *energy;             // [instance][R_out]
  int32_t *passes;            // [instance][R_out] or null
  unsigned long long *stats;
};

// value k of coupling array p as FP64; ct: 0 int8, 1 FP32, 2 FP64 values
__device__ __forceinline__ double value_of(const void *p, int ct, int64_t k) {
  return ct == 2 ? __ldg(reinterpret_cast<const double *>(p) + k)
                 : (ct == 1 ? (double)__ldg(reinterpret_cast<const float *>(p) + k)
                            : (double)__ldg(reinterpret_cast<const int8_t *>(p) + k));
}
__device__ __forceinline__ double coupling(const DevGraph &G, int ct, int64_t k) { return value_of(G.J, ct, k); }
__device__ __forceinline__ double field_h(const DevGraph &G, int ct, int64_t gi) { return value_of(G.h, ct, gi); }
__device__ __forceinline__ double coupling_e(const DevGraph &G, int ct, int64_t e) { return value_of(G.hJ, ct, e); }
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

// ---- the same search in exact integers ----------------------------------
// When every field, gain and energy value of an instance is an integer
// multiple of a unit u (2^(ebase - 150) for FP32 couplings, 1 for int8) below
// 2^53 in magnitude (InstDesc::fx53), FP64 computes all of them without
// rounding; the search then runs on 64-bit integers in units of u and gives
// bit-identical results with no FP64 arithmetic on the per-move path.

// spin product of hyper-edge e except `skip` (-1: all), as +1 or -1
__device__ __forceinline__ int hyper_sign(const DevGraph &G, int64_t e, const int8_t *s, int skip) {
  int neg = 0;
  for (uint32_t q = __ldg(G.hptr + e), qe = __ldg(G.hptr + e + 1); q < qe; ++q) {
    const int m = __ldg(G.hmem + q);
    if (m != skip) neg ^= s[m] < 0;
  }
  return neg ? -1 : 1;
}

// coupling or field k of array p in units of u
__device__ __forceinline__ long long fx_of(const void *p, bool fl, int64_t k, int unit) {
  return fl ? (long long)xr_term(__ldg(reinterpret_cast<const float *>(p) + k), unit)
            : (long long)__ldg(reinterpret_cast<const int8_t *>(p) + k);
}

// order-preserving key of the gain -2 s f (|gain| < 2^54: never key 0)
__device__ __forceinline__ unsigned long long gain_key_fx(long long f, int8_t s) {
  const long long g = s > 0 ? -2 * f : 2 * f;
  return (unsigned long long)g ^ 0x8000000000000000ull;
}

// v * 2^(unit - 150) as an FP64 value, built from its bits (|v| < 2^53:
// exact, no rounding), for fields held in per-spin units
__device__ __forceinline__ double fx_double(long long v, int unit) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  const unsigned long long mant = (a << (lz + 1)) >> 12;  // the bits below the leading one
  const unsigned long long ex = (unsigned long long)(63 - lz + unit - 150 + 1023);
  return __longlong_as_double((long long)(sign | (ex << 52) | mant));
}

// E in units of u by one warp (integer sums: the order does not matter)
__device__ __forceinline__ long long fm_energy_fx(const DevGraph &G, const InstDesc &I, bool fl, const int8_t *s,
                                                  int lane, int unit) {
  long long acc = 0;
  for (int i = lane; i < I.n; i += 32) {
    const int64_t gi = I.spin_off + i;
    const int8_t si = s[i];
    for (uint32_t k = __ldg(G.row + gi), ke = __ldg(G.row + gi + 1); k < ke; ++k) {
      const int j = __ldg(G.col + k);
      if (j > i) {
        const long long t = fx_of(G.J, fl, k, unit);
        acc -= (si == s[j]) ? t : -t;
      }
    }
    const long long th = fx_of(G.h, fl, gi, unit);
    acc -= si > 0 ? th : -th;
  }
  for (int e = lane; e < I.n_hyper; e += 32) {
    const int64_t ge = I.hyper_off + e;
    const long long t = fx_of(G.hJ, fl, ge, unit);
    acc -= hyper_sign(G, ge, s, -1) > 0 ? t : -t;
  }
  return warp_sum(acc);
}

// E (Eq. 1 extended by Eq. 6) by one warp: pairs once (j > i), fields,
// hyper-edges; lane partial sums, then the warp sum (a fixed order).  FP64
// instances (ct 2): the sequential compensated sum the C ABI defines for
// them, by lane 0, the same value in every lane.
__device__ __forceinline__ double fm_energy(const DevGraph &G, const InstDesc &I, int ct, const int8_t *s, int lane) {
  if (ct == 2) {
    double E = 0.0;
    if (lane == 0) E = energy_f64_seq(G, I, s);
    return __shfl_sync(0xffffffffu, E, 0);
  }
  double acc = 0.0;
  for (int i = lane; i < I.n; i += 32) {
    const int64_t gi = I.spin_off + i;
    const double si = (double)s[i];
    for (uint32_t k = __ldg(G.row + gi), ke = __ldg(G.row + gi + 1); k < ke; ++k) {
      const int j = __ldg(G.col + k);
      if (j > i) acc -= coupling(G, ct, k) * si * (double)s[j];
    }
    acc -= field_h(G, ct, gi) * si;
  }
  for (int e = lane; e < I.n_hyper; e += 32) {
    const int64_t ge = I.hyper_off + e;
    acc -= coupling_e(G, ct, ge) * hyper_prod(G, ge, s, -1);
  }
  return warp_sum(acc);
}

// bytes of shared memory one warp needs for an instance of n spins in
// arithmetic M: fields (FP64 or int64), block maxima (key, index), lock bits
// and their snapshot at the best prefix, dirty bits, spins and, in per-spin
// units, the spins' field units
__host__ __device__ constexpr size_t fm_warp_bytes(int n, int M) {
  return (size_t)n * (M == 2 ? 10 : 9) + (size_t)((n + 31) / 32) * 18 + 16 + 2 * 64;
}

// The warp's maximum of (key, index) pairs: the largest key, among equal keys
// the lowest index.  Every lane receives it.  Keys of real gains are never 0
// (see gain_key), so key 0 marks "no candidate".
struct KeyIdx {
  unsigned long long key;
  int idx;
};
__device__ __forceinline__ KeyIdx warp_argmax(unsigned long long key, int idx) {
  const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  const int mi = __reduce_min_sync(0xffffffffu, (hi == mhi && lo == mlo) ? idx : 0x7fffffff);
  return {((unsigned long long)mhi << 32) | mlo, mi};
}

// Per-warp state of one search, carved out of the warp's shared memory.
struct FmState {
  double *f;                // [n] fields
  unsigned long long *bkey; // [nb] largest unlocked gain key of each 32-spin block (0: none)
  uint32_t *lock;           // [nb] spins moved in this pass
  uint32_t *best;           // [nb] spins moved up to the best prefix so far
  uint32_t *dirty;          // [4] blocks whose maximum must be recomputed
  int16_t *bidx;            // [nb] the spin of each block maximum (lowest of equal keys)
  int16_t *touched;         // [kTouched] spins whose fields the current move changed (-1: none)
  int8_t *s;                // [n] spins
  uint8_t *un;              // [n] each spin's field unit (per-spin integer form only)
  int n, nb;
};
__device__ __forceinline__ FmState fm_state(uint8_t *base, int n) {
  FmState S;
  S.n = n;
  S.nb = (n + 31) / 32;
  S.f = reinterpret_cast<double *>(base);
  S.bkey = reinterpret_cast<unsigned long long *>(S.f + n);
  S.lock = reinterpret_cast<uint32_t *>(S.bkey + S.nb);
  S.best = S.lock + S.nb;
  S.dirty = S.best + S.nb;
  S.bidx = reinterpret_cast<int16_t *>(S.dirty + 4);
  S.touched = S.bidx + S.nb;
  S.s = reinterpret_cast<int8_t *>(S.touched + kTouched);
  S.un = reinterpret_cast<uint8_t *>(S.s + n);
  return S;
}

// gain key of unlocked spin c in arithmetic M
template <int M>
__device__ __forceinline__ unsigned long long spin_key(const FmState &S, int c) {
  if constexpr (M == kFx)
    return gain_key_fx(reinterpret_cast<const long long *>(S.f)[c], S.s[c]);
  else if constexpr (M == kFxSpin)
    return gain_key(fx_double(reinterpret_cast<const long long *>(S.f)[c], S.un[c]), S.s[c]);
  else
    return gain_key(S.f[c], S.s[c]);
}

// block j's maximum over its unlocked spins, one lane per spin
template <int M>
__device__ __forceinline__ void block_max(const FmState &S, int j, int lane) {
  const int i = (j << 5) + lane;
  unsigned long long key = 0ull;
  if (i < S.n && !((S.lock[j] >> lane) & 1u)) key = spin_key<M>(S, i);
  const KeyIdx m = warp_argmax(key, i);
  if (lane == 0) {
    S.bkey[j] = m.key;
    S.bidx[j] = (int16_t)m.idx;
  }
}

// One warp per search (instance, replica, a range of starts): no CTA barriers
// on the per-move path.  The move's spin is the maximum over the cached block
// maxima; a move recomputes only the blocks it touched (the moved spin's and
// those of the spins whose fields changed).  M: the arithmetic (kFp64, kFx,
// kFxSpin); every form computes the same values as FP64 in the definition's
// order, so all give identical moves.
template <int M, int FL>
__global__ void __launch_bounds__(kFT, 3) fm_kernel(FmArgs A, int nmax) {
  constexpr bool INT = M != kFp64;
  using T = std::conditional_t<INT, long long, double>;       // fields
  using TE = std::conditional_t<M == kFx, long long, double>;  // running energy
  extern __shared__ __align__(16) uint8_t fm_smem[];
  const DevGraph &G = A.g;
  constexpr int ct = FL;        // coupling values: 0 int8, 1 FP32, 2 FP64
  constexpr bool fl = FL == 1;  // FP32 couplings (the integer forms' scaling)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t *base = fm_smem + (size_t)warp * ((fm_warp_bytes(nmax, M) + 15) & ~(size_t)15);
  unsigned long long c_moves = 0, c_passes = 0, c_starts = 0;
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(A.queue, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= A.n_work) break;
    // split starts: one start per work unit, results to slot r * restarts + k
    const int it = A.split ? w / A.restarts : w;
    const int k0 = A.split ? w % A.restarts : 0, k1 = A.split ? k0 + 1 : A.restarts;
    const int b = A.items[it].x, r = A.items[it].y;
    const int slot = A.split ? r * A.restarts + k0 : r;
    const InstDesc I = G.inst[b];
    const int n = I.n;
    const int64_t so = I.spin_off;
    const int unit = I.ebase;  // kFx with FP32 couplings: u = 2^(unit - 150)
    const double scale = (M == kFx && fl) ? __longlong_as_double((long long)(unit - 150 + 1023) << 52) : 1.0;
    const FmState S = fm_state(base, n);
    T *f = reinterpret_cast<T *>(S.f);
    int8_t *s = S.s;
    if constexpr (M == kFxSpin)
      for (int i = lane; i < n; i += 32) S.un[i] = (uint8_t)__ldg(G.runit + so + i);
    // spin i's unit in the integer forms
    auto unit_of = [&](int i) -> int {
      if constexpr (M == kFxSpin) return S.un[i];
      return unit;
    };
    const uint64_t seed = A.seeds[b];
    // E of the current spins in FP64 (the same value in every lane); kFx also
    // returns the integer it is exactly
    auto energy = [&](long long &Ei) -> double {
      if constexpr (M == kFx) {
        Ei = fm_energy_fx(G, I, fl, s, lane, unit);
        return (double)Ei * scale;
      } else {
        Ei = 0;
        return fm_energy(G, I, ct, s, lane);
      }
    };
    double E_all = DBL_MAX;
    int total_passes = 0;
    int8_t *out = A.spins + (int64_t)A.R_out * so + (int64_t)slot * n;
    for (int k = k0; k < k1; ++k) {
      for (int i = lane; i < n; i += 32) {
        const uint4 x = start_bits(seed, (uint32_t)(i >> 7), (uint32_t)r, (uint32_t)k, (uint32_t)b);
        s[i] = ((word_of(x, (i & 127) >> 5) >> (i & 31)) & 1u) ? 1 : -1;
      }
      __syncwarp();
      long long EstarI;
      double Estar = energy(EstarI);
      int passes = 0;
      for (;;) {
        ++passes;
        // fields: h, the CSR row in order, then the hyper-edges in ascending order
        for (int i = lane; i < n; i += 32) {
          const int64_t gi = so + i;
          if constexpr (INT) {
            const int ui = unit_of(i);
            long long acc = fx_of(G.h, fl, gi, ui);
            for (uint32_t kk = __ldg(G.row + gi), ke = __ldg(G.row + gi + 1); kk < ke; ++kk) {
              const long long t = fx_of(G.J, fl, kk, ui);
              acc += s[__ldg(G.col + kk)] > 0 ? t : -t;
            }
            for (uint32_t u = __ldg(G.inc_ptr + gi), ue = __ldg(G.inc_ptr + gi + 1); u < ue; ++u) {
              const int64_t e = __ldg(G.inc_edge + u);
              const long long t = fx_of(G.hJ, fl, e, ui);
              acc += hyper_sign(G, e, s, i) > 0 ? t : -t;
            }
            f[i] = acc;
          } else {
            double acc = field_h(G, ct, gi);
            for (uint32_t kk = __ldg(G.row + gi), ke = __ldg(G.row + gi + 1); kk < ke; ++kk)
              acc += coupling(G, ct, kk) * (double)s[__ldg(G.col + kk)];
            for (uint32_t u = __ldg(G.inc_ptr + gi), ue = __ldg(G.inc_ptr + gi + 1); u < ue; ++u) {
              const int64_t e = __ldg(G.inc_edge + u);
              acc += coupling_e(G, ct, e) * hyper_prod(G, e, s, i);
            }
            f[i] = acc;
          }
        }
        for (int j = lane; j < S.nb; j += 32) S.lock[j] = S.best[j] = 0u;
        if (lane < 4) S.dirty[lane] = 0u;
        __syncwarp();
        for (int j = 0; j < S.nb; ++j) block_max<M>(S, j, lane);
        __syncwarp();
        TE Ecur, Ebest;  // lane 0's copies are used
        if constexpr (M == kFx)
          Ecur = EstarI;
        else
          Ecur = Estar;
        Ebest = Ecur;
        bool any_best = false;  // the pass found a prefix below its start
        for (int step = 0; step < n; ++step) {
          // the largest gain among unlocked spins, ties to the lowest index:
          // blocks in ascending order per lane, then across lanes
          unsigned long long bk = 0ull;
          int bi = 0x7fffffff;
          for (int j = lane; j < S.nb; j += 32) {
            const unsigned long long key = S.bkey[j];
            if (key > bk) {
              bk = key;
              bi = S.bidx[j];
            }
          }
          const int i = warp_argmax(bk, bi).idx;
          // the moved spin's row and incidence bounds, loaded before its
          // bookkeeping so that the loads overlap it
          const int64_t gi = so + i;
          const uint32_t r0 = __ldg(G.row + gi), r1 = __ldg(G.row + gi + 1);
          const uint32_t u0 = __ldg(G.inc_ptr + gi), u1 = __ldg(G.inc_ptr + gi + 1);
          bool new_best = false;
          if (lane == 0) {
            TE gain;
            if constexpr (M == kFx)
              gain = s[i] > 0 ? -2 * f[i] : 2 * f[i];
            else if constexpr (M == kFxSpin)
              gain = -2.0 * (double)s[i] * fx_double(f[i], S.un[i]);
            else
              gain = -2.0 * (double)s[i] * f[i];
            Ecur -= gain;  // apply the move
            if (Ecur < Ebest) {
              Ebest = Ecur;
              new_best = true;
            }
            S.lock[i >> 5] |= 1u << (i & 31);
            S.dirty[i >> 10] |= 1u << ((i >> 5) & 31);  // its block lost its maximum
            s[i] = (int8_t)-s[i];
          }
          __syncwarp();
          // neighbours' fields: the CSR row (distinct columns, one lane each),
          // then the hyper-edges in order, each by its members in parallel
          // (distinct within an edge); every changed field's spin goes to
          // the touched list (CSR entries first, then the edges' members)
          const int8_t snew = s[i];
          for (uint32_t kk = r0 + lane; kk < r1; kk += 32) {
            const int c = __ldg(G.col + kk);
            if constexpr (INT) {
              const long long t2 = 2 * fx_of(G.J, fl, kk, unit_of(c));
              f[c] += snew > 0 ? t2 : -t2;
            } else {
              f[c] += coupling(G, ct, kk) * (2.0 * (double)snew);
            }
            if (kk - r0 < (uint32_t)kTouched) S.touched[kk - r0] = (int16_t)c;
          }
          uint32_t n_touched = r1 - r0;
          for (uint32_t u = u0; u < u1; ++u) {
            __syncwarp();
            const int64_t e = __ldg(G.inc_edge + u);
            const uint32_t q0 = __ldg(G.hptr + e), q1 = __ldg(G.hptr + e + 1);
            int neg = 0;  // parity of the members' negative spins
            for (uint32_t q = q0 + lane; q < q1; q += 32) neg ^= s[__ldg(G.hmem + q)] < 0;
            const int par = __popc(__ballot_sync(0xffffffffu, neg)) & 1;
            for (uint32_t q = q0 + lane; q < q1; q += 32) {
              const int m = __ldg(G.hmem + q);
              const uint32_t slot_t = n_touched + (q - q0);
              if (slot_t < (uint32_t)kTouched) S.touched[slot_t] = (int16_t)(m == i ? -1 : m);
              if (m == i) continue;
              const bool minus = par ^ (s[m] < 0);  // the other members' product is -1
              if constexpr (INT) {
                const long long w2 = 2 * fx_of(G.hJ, fl, e, unit_of(m));
                f[m] += minus ? -w2 : w2;
              } else {
                const double w2 = 2.0 * coupling_e(G, ct, e);
                f[m] += w2 * (minus ? -1.0 : 1.0);
              }
            }
            n_touched += q1 - q0;
          }
          // the earliest strictly lowest prefix so far ends here: remember
          // which spins it moved (every spin moves once per pass, so the
          // lock bits are that set)
          if (__shfl_sync(0xffffffffu, (int)new_best, 0)) {
            any_best = true;
            for (int j = lane; j < S.nb; j += 32) S.best[j] = S.lock[j];
          }
          __syncwarp();
          // Block maxima after the move.  The moved spin's block is recomputed
          // (its maximum is now locked).  A touched unlocked spin elsewhere
          // either raises its block's maximum (applied one spin at a time, the
          // larger key or on equal keys the lower index winning) or, when it
          // was that maximum and its key fell, marks the block for a recompute.
          // A move touching more than kTouched fields recomputes every block.
          if (n_touched <= (uint32_t)kTouched) {
            const int jm = i >> 5;
            for (uint32_t t0 = 0; t0 < n_touched; t0 += 32) {  // at most two rounds
              const uint32_t t = t0 + lane;
              const int ct = t < n_touched ? S.touched[t] : -1;
              unsigned long long kt = 0ull;
              bool raise = false;
              if (ct >= 0 && (ct >> 5) != jm && !((S.lock[ct >> 5] >> (ct & 31)) & 1u)) {
                kt = spin_key<M>(S, ct);
                const int jb = ct >> 5;
                const unsigned long long ok = S.bkey[jb];
                const int oi = S.bidx[jb];
                if (oi == ct && kt < ok)
                  atomicOr(S.dirty + (jb >> 5), 1u << (jb & 31));
                else
                  raise = oi == ct || kt > ok || (kt == ok && ct < oi);
              }
              // apply the raises one lane at a time against the current maximum
              unsigned pend = __ballot_sync(0xffffffffu, raise);
              while (pend) {
                const int L = __ffs(pend) - 1;
                pend &= pend - 1u;
                if (lane == L) {
                  const int jb = ct >> 5;
                  const unsigned long long ok = S.bkey[jb];
                  const int oi = S.bidx[jb];
                  if (oi == ct ? kt >= ok : (kt > ok || (kt == ok && ct < oi))) {
                    S.bkey[jb] = kt;
                    S.bidx[jb] = (int16_t)ct;
                  }
                }
                __syncwarp();
              }
            }
          } else {
            for (int dw = lane; dw < 4; dw += 32) S.dirty[dw] = 0xffffffffu;
          }
          __syncwarp();
          for (int dw = 0; dw < (S.nb + 31) / 32; ++dw) {
            unsigned d = S.dirty[dw];
            if (dw == (S.nb - 1) >> 5 && (S.nb & 31)) d &= (1u << (S.nb & 31)) - 1u;
            while (d) {
              const int jb = __ffs(d) - 1;
              d &= d - 1u;
              block_max<M>(S, (dw << 5) + jb, lane);
            }
          }
          __syncwarp();
          if (lane < 4) S.dirty[lane] = 0u;
          __syncwarp();
        }
        // roll back to the best prefix: every spin moved once, so the spins
        // outside that prefix's set are flipped back
        __syncwarp();
        for (int i = lane; i < n; i += 32)
          if (!((S.best[i >> 5] >> (i & 31)) & 1u)) s[i] = (int8_t)-s[i];
        __syncwarp();
        long long EnewI;
        const double Enew = energy(EnewI);
        const double margin = fl ? 1e-9 * (1.0 + fabs(Estar)) : 0.0;
        c_moves += (unsigned long long)n;
        if (Enew < Estar - margin && (A.max_passes <= 0 || passes < A.max_passes)) {
          Estar = Enew;
          EstarI = EnewI;
          continue;
        }
        if (Enew < Estar - margin) {
          Estar = Enew;  // pass cap reached after an improving pass: keep it
        } else if (any_best) {  // back to the pass's start
          for (int i = lane; i < n; i += 32)
            if ((S.best[i >> 5] >> (i & 31)) & 1u) s[i] = (int8_t)-s[i];
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
        for (int i = lane; i < n; i += 32) out[i] = s[i];
      }
      __syncwarp();
    }
    if (lane == 0) {
      A.energy[(int64_t)b * A.R_out + slot] = E_all;
      if (A.passes) A.passes[(int64_t)b * A.R_out + slot] = total_passes;
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

// Small instances in the one-unit integer form (kFx, n <= 32 * S, S = 8 or 16):
// lane l holds the fields, spin bits, lock bits and best-prefix bits of spins
// l, l + 32, ... in registers.  A move's arg-max is each lane's maximum over
// its own unlocked spins (registers only) and one warp reduction; the changed
// fields travel through a 32-entry list in shared memory to the lanes that
// hold them.  The spins are also kept in shared memory for the neighbour reads
// of the per-pass field and energy sums.  Same moves as fm_kernel.
constexpr int kRegMaxSpins = 32 * 16;
// per warp: fields staged at a pass's start, list deltas, spins, list spins
__host__ __device__ constexpr size_t reg_warp_bytes(int S) { return (size_t)32 * S * 9 + 32 * 8 + 32 * 4; }

template <bool FL, int S>
__global__ void __launch_bounds__(kFT, S <= 8 ? 2 : 1) fm_reg_kernel(FmArgs A) {
  constexpr int kRegSlots = S;
  extern __shared__ __align__(16) uint8_t fm_smem[];
  const DevGraph &G = A.g;
  constexpr bool fl = FL;
  constexpr int ct = FL ? 1 : 0;
  (void)ct;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t *base = fm_smem + (size_t)warp * reg_warp_bytes(S);
  long long *fsc = reinterpret_cast<long long *>(base);  // [32 S] fields at a pass's start
  long long *ldv = fsc + 32 * S;                          // [32] field changes
  int8_t *s = reinterpret_cast<int8_t *>(ldv + 32);       // [32 S] spins
  int32_t *ldc = reinterpret_cast<int32_t *>(s + 32 * S); // [32] the changed fields' spins
  unsigned long long c_moves = 0, c_passes = 0, c_starts = 0;
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(A.queue, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= A.n_work) break;
    const int it = A.split ? w / A.restarts : w;
    const int k0 = A.split ? w % A.restarts : 0, k1 = A.split ? k0 + 1 : A.restarts;
    const int b = A.items[it].x, r = A.items[it].y;
    const int slot = A.split ? r * A.restarts + k0 : r;
    const InstDesc I = G.inst[b];
    const int n = I.n;
    const int64_t so = I.spin_off;
    const int unit = I.ebase;
    const double scale = fl ? __longlong_as_double((long long)(unit - 150 + 1023) << 52) : 1.0;
    uint32_t vm = 0;  // own slots that are spins of the instance
#pragma unroll
    for (int t = 0; t < kRegSlots; ++t)
      if (lane + 32 * t < n) vm |= 1u << t;
    const uint64_t seed = A.seeds[b];
    int8_t *out = A.spins + (int64_t)A.R_out * so + (int64_t)slot * n;
    double E_all = DBL_MAX;
    int total_passes = 0;
    for (int k = k0; k < k1; ++k) {
      for (int i = lane; i < n; i += 32) {
        const uint4 x = start_bits(seed, (uint32_t)(i >> 7), (uint32_t)r, (uint32_t)k, (uint32_t)b);
        s[i] = ((word_of(x, (i & 127) >> 5) >> (i & 31)) & 1u) ? 1 : -1;
      }
      __syncwarp();
      long long EstarI = fm_energy_fx(G, I, fl, s, lane, unit);
      double Estar = (double)EstarI * scale;
      int passes = 0;
      for (;;) {
        ++passes;
        // own fields: h, the CSR row in order, then the hyper-edges ascending,
        // staged in shared memory and then taken into registers
        for (int i = lane; i < n; i += 32) {
          const int64_t gi = so + i;
          long long acc = fx_of(G.h, fl, gi, unit);
          for (uint32_t kk = __ldg(G.row + gi), ke = __ldg(G.row + gi + 1); kk < ke; ++kk) {
            const long long tj = fx_of(G.J, fl, kk, unit);
            acc += s[__ldg(G.col + kk)] > 0 ? tj : -tj;
          }
          for (uint32_t u = __ldg(G.inc_ptr + gi), ue = __ldg(G.inc_ptr + gi + 1); u < ue; ++u) {
            const int64_t e = __ldg(G.inc_edge + u);
            const long long te = fx_of(G.hJ, fl, e, unit);
            acc += hyper_sign(G, e, s, i) > 0 ? te : -te;
          }
          fsc[i] = acc;
        }
        __syncwarp();
        long long fr[kRegSlots];
        uint32_t sb = 0;  // own spins that are +1
#pragma unroll
        for (int t = 0; t < kRegSlots; ++t) {
          const int i = lane + 32 * t;
          fr[t] = i < n ? fsc[i] : 0;
          if (i < n && s[i] > 0) sb |= 1u << t;
        }
        uint32_t lk = 0, bb = 0;  // own lock bits, own bits of the best prefix's spins
        long long Ecur = EstarI, Ebest = EstarI;
        bool any_best = false;
        for (int step = 0; step < n; ++step) {
          unsigned long long bk = 0ull;
          int bi = 0x7fffffff;
#pragma unroll
          for (int t = 0; t < kRegSlots; ++t) {
            if (((vm & ~lk) >> t) & 1u) {
              const long long g = ((sb >> t) & 1u) ? -2 * fr[t] : 2 * fr[t];
              const unsigned long long key = (unsigned long long)g ^ 0x8000000000000000ull;
              if (key > bk) {  // ascending slots: the lower index keeps equal keys
                bk = key;
                bi = lane + 32 * t;
              }
            }
          }
          const KeyIdx m = warp_argmax(bk, bi);
          const int i = m.idx;
          Ecur -= (long long)(m.key ^ 0x8000000000000000ull);  // the move's gain
          const bool new_best = Ecur < Ebest;
          if (new_best) Ebest = Ecur;
          const int8_t snew = (int8_t)-s[i];
          if (lane == (i & 31)) {
            lk |= 1u << (i >> 5);
            sb ^= 1u << (i >> 5);
          }
          if (new_best) {
            any_best = true;
            bb = lk;
          }
          const int64_t gi = so + i;
          const uint32_t r0 = __ldg(G.row + gi), r1 = __ldg(G.row + gi + 1);
          const uint32_t u0 = __ldg(G.inc_ptr + gi), u1 = __ldg(G.inc_ptr + gi + 1);
          __syncwarp();
          if (lane == 0) s[i] = snew;
          __syncwarp();
          // CSR neighbours, 32 entries at a time through the list
          for (uint32_t c0 = r0; c0 < r1; c0 += 32) {
            const uint32_t kk = c0 + lane;
            if (kk < r1) {
              const long long t2 = 2 * fx_of(G.J, fl, kk, unit);
              ldc[lane] = __ldg(G.col + kk);
              ldv[lane] = snew > 0 ? t2 : -t2;
            }
            __syncwarp();
            const int cnt = (int)min(32u, r1 - c0);
            for (int q = 0; q < cnt; ++q) {
              const int c = ldc[q];
              const long long d = (c & 31) == lane ? ldv[q] : 0;
              const int ts = c >> 5;
#pragma unroll
              for (int t = 0; t < kRegSlots; ++t) fr[t] += t == ts ? d : 0;
            }
            __syncwarp();
          }
          // hyper-edges in order, their members 32 at a time
          for (uint32_t u = u0; u < u1; ++u) {
            const int64_t e = __ldg(G.inc_edge + u);
            const uint32_t q0 = __ldg(G.hptr + e), q1 = __ldg(G.hptr + e + 1);
            int neg = 0;
            for (uint32_t q = q0 + lane; q < q1; q += 32) neg ^= s[__ldg(G.hmem + q)] < 0;
            const int par = __popc(__ballot_sync(0xffffffffu, neg)) & 1;
            const long long w2 = 2 * fx_of(G.hJ, fl, e, unit);
            for (uint32_t c0 = q0; c0 < q1; c0 += 32) {
              const uint32_t q = c0 + lane;
              if (q < q1) {
                const int mm = __ldg(G.hmem + q);
                const bool minus = par ^ (s[mm] < 0);
                ldc[lane] = mm == i ? -1 : mm;
                ldv[lane] = minus ? -w2 : w2;
              }
              __syncwarp();
              const int cnt = (int)min(32u, q1 - c0);
              for (int qq = 0; qq < cnt; ++qq) {
                const int c = ldc[qq];
                const long long d = c >= 0 && (c & 31) == lane ? ldv[qq] : 0;
                const int ts = c >> 5;
#pragma unroll
                for (int t = 0; t < kRegSlots; ++t) fr[t] += t == ts ? d : 0;
              }
              __syncwarp();
            }
          }
        }
        // roll back to the best prefix: own spins outside its set flip back
        const uint32_t back = vm & ~bb;
#pragma unroll
        for (int t = 0; t < kRegSlots; ++t)
          if ((back >> t) & 1u) s[lane + 32 * t] = (int8_t)-s[lane + 32 * t];
        __syncwarp();
        const long long EnewI = fm_energy_fx(G, I, fl, s, lane, unit);
        const double Enew = (double)EnewI * scale;
        const double margin = fl ? 1e-9 * (1.0 + fabs(Estar)) : 0.0;
        c_moves += (unsigned long long)n;
        if (Enew < Estar - margin && (A.max_passes <= 0 || passes < A.max_passes)) {
          Estar = Enew;
          EstarI = EnewI;
          continue;
        }
        if (Enew < Estar - margin) {
          Estar = Enew;
        } else if (any_best) {
#pragma unroll
          for (int t = 0; t < kRegSlots; ++t)
            if (((vm & bb) >> t) & 1u) s[lane + 32 * t] = (int8_t)-s[lane + 32 * t];
          __syncwarp();
        }
        break;
      }
      total_passes += passes;
      c_passes += (unsigned long long)passes;
      c_starts += 1;
      if (Estar < E_all) {
        E_all = Estar;
        for (int i = lane; i < n; i += 32) out[i] = s[i];
      }
      __syncwarp();
    }
    if (lane == 0) {
      A.energy[(int64_t)b * A.R_out + slot] = E_all;
      if (A.passes) A.passes[(int64_t)b * A.R_out + slot] = total_passes;
    }
    __syncwarp();
  }
  if (lane == 0 && c_starts) {
    atomicAdd(A.stats + 0, c_moves);
    atomicAdd(A.stats + 1, c_moves);
    atomicAdd(A.stats + 3, c_starts);
    atomicAdd(A.stats + 4, c_passes);
  }
}

// After split starts: per (instance, replica) the best start (strictly lower
// energy, ties keep the earlier start), its spins, and the pass count summed
// over the starts.  One warp per (instance, replica).
__global__ void fm_best_start_kernel(const InstDesc *inst, int32_t n_inst, int32_t R, int32_t restarts,
                                     const int8_t *spins_k, const double *E_k, const int32_t *passes_k,
                                     int8_t *spins, double *E, int32_t *passes) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wid >= (int64_t)n_inst * R) return;
  const int b = (int)(wid / R), r = (int)(wid % R);
  const InstDesc I = inst[b];
  const int64_t base = (int64_t)b * R * restarts + (int64_t)r * restarts;
  int best = 0;
  double Eb = E_k[base];
  int tp = passes_k ? passes_k[base] : 0;
  for (int k = 1; k < restarts; ++k) {
    const double e = E_k[base + k];
    if (e < Eb) {
      Eb = e;
      best = k;
    }
    if (passes_k) tp += passes_k[base + k];
  }
  const int8_t *src = spins_k + (int64_t)R * restarts * I.spin_off + ((int64_t)r * restarts + best) * I.n;
  int8_t *dst = spins + (int64_t)R * I.spin_off + (int64_t)r * I.n;
  for (int i = lane; i < I.n; i += 32) dst[i] = src[i];
  if (lane == 0) {
    E[(int64_t)b * R + r] = Eb;
    if (passes) passes[(int64_t)b * R + r] = tp;
  }
}

// device buffers per handle, kept across calls: the (instance, replica)
// list, the work-queue counters and, for split starts, every start's result
struct FmBufs : FamilyState {
  int2 *items = nullptr;
  size_t items_bytes = 0;
  int32_t *queues = nullptr;
  size_t queues_bytes = 0;
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  // side streams for overlapping the groups' launches, with fork/join events
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
};

template <typename P>
cudaError_t grow(P *&p, size_t &have, size_t need) {
  if (have >= need) return cudaSuccess;
  cudaFree(p);
  p = nullptr;
  have = 0;
  void *q = nullptr;
  const cudaError_t e = cudaMalloc(&q, need);
  if (e != cudaSuccess) return e;
  p = static_cast<P *>(q);
  have = need;
  return e;
}

constexpr size_t kSplitScratchMax = size_t(1) << 30;  // bytes of per-start results at most
constexpr int kSideStreams = 4;

cudaError_t ensure_side(FmBufs &B) {
  if (!B.side.empty()) return cudaSuccess;
  cudaError_t e = cudaEventCreateWithFlags(&B.fork, cudaEventDisableTiming);
  for (int j = 0; j < kSideStreams && e == cudaSuccess; ++j) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) break;
    B.side.push_back(st);
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) break;
    B.join.push_back(ev);
  }
  if (e != cudaSuccess || (int)B.join.size() != kSideStreams) {
    for (cudaStream_t st : B.side) cudaStreamDestroy(st);
    for (cudaEvent_t ev : B.join) cudaEventDestroy(ev);
    if (B.fork) cudaEventDestroy(B.fork);
    B.side.clear();
    B.join.clear();
    B.fork = nullptr;
    return e != cudaSuccess ? e : cudaErrorUnknown;
  }
  return cudaSuccess;
}

// One launch group: instances of one arithmetic (FX or FP64) whose size falls
// in (lo, hi], so that each warp's shared memory is sized for hi.
struct FmPart {
  int mode;  // kFp64 / kFx / kFxSpin
  int nmax;
  int64_t first, count;  // range of the item list
};

// Warps per CTA (one search each) and CTAs per SM for instances of up to
// nmax spins: the most searches per SM that shared memory and registers allow,
// the larger CTA among equals.
template <int M, int FL>
cudaError_t fm_shape(const ising_handle *h, int nmax, int &warps, size_t &smem, int &per_sm) {
  const size_t per_warp = (fm_warp_bytes(nmax, M) + 15) & ~(size_t)15;
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  cudaError_t e;
  const int wmax = (int)std::max<size_t>(1, std::min<size_t>(kFW, (size_t)smem_optin / per_warp));
  if ((e = cudaFuncSetAttribute(fm_kernel<M, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(per_warp * wmax))) != cudaSuccess)
    return e;
  int best = -1;
  for (int w = wmax; w >= 1; --w) {
    int c = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, fm_kernel<M, FL>, w * 32, per_warp * w)) != cudaSuccess)
      return e;
    if (c * w > best) {
      best = c * w;
      warps = w;
      per_sm = std::max(c, 1);
    }
  }
  smem = per_warp * warps;
  return cudaSuccess;
}

// the register kernel's shape: 8 warps per CTA, as many CTAs per SM as fit
template <bool FL, int S>
cudaError_t fm_reg_shape(const ising_handle *h, int &warps, size_t &smem, int &per_sm) {
  (void)h;
  warps = kFW;
  smem = reg_warp_bytes(S) * kFW;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(fm_reg_kernel<FL, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fm_reg_kernel<FL, S>, kFT, smem)) !=
      cudaSuccess)
    return e;
  per_sm = std::max(per_sm, 1);
  return cudaSuccess;
}

}  // namespace

int fm_max_spins() { return kFmMaxSpins; }

// Launches over every (instance, replica): one per group of instances of like
// arithmetic and size, plus a selection launch when the starts run in
// parallel.  seeds: device [instances].
cudaError_t launch_fm(ising_handle *h, int32_t R, const ising_fm_params *fp, int8_t *spins, double *E,
                      int32_t *passes, cudaStream_t s) {
  const int32_t restarts = fp->restarts, max_passes = fp->max_passes;
  const int64_t n_items = (int64_t)h->n_inst * R;
  if (n_items > 0x7fffffff) return cudaErrorInvalidValue;
  FmBufs &B = family_state<FmBufs>(h->fm_st);
  cudaError_t e;
  // groups: one-unit integer instances, per-spin-unit ones, then FP64;
  // within each, size classes (0, 256], (256, 512], ... (2048, 4096],
  // largest first
  auto cls = [](int n) {
    int c = 0;
    while (c < 4 && n > (256 << c)) ++c;
    return c;
  };
  std::vector<int32_t> ord(h->n_inst);
  for (int32_t b = 0; b < h->n_inst; ++b) ord[b] = b;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) {
    const InstDesc &x = h->inst[a], &y = h->inst[c];
    auto rank = [](int m) { return m == kFx ? 0 : (m == kFxSpin ? 1 : 2); };
    if (x.fx53 != y.fx53) return rank(x.fx53) < rank(y.fx53);
    return x.n > y.n;
  });
  std::vector<int2> items;
  std::vector<FmPart> parts;
  items.reserve((size_t)n_items);
  for (int32_t b : ord) {
    const InstDesc &D = h->inst[b];
    const int mode = D.fx53;
    if (parts.empty() || parts.back().mode != mode || cls(parts.back().nmax) != cls(D.n))
      parts.push_back({mode, D.n, (int64_t)items.size(), 0});
    for (int32_t r = 0; r < R; ++r) items.push_back(make_int2(b, r));
    parts.back().count += R;
  }
  if ((e = grow(B.items, B.items_bytes, (size_t)n_items * sizeof(int2))) != cudaSuccess) return e;
  if ((e = grow(B.queues, B.queues_bytes, parts.size() * sizeof(int32_t))) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(B.items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(B.queues, 0, parts.size() * sizeof(int32_t), s)) != cudaSuccess) return e;

  // Starts run in parallel (one per warp, the best chosen afterwards) when
  // the searches alone would leave the GPU underfilled.
  int warps0 = 0, per_sm0 = 0;
  size_t smem0 = 0;
  const bool fl = h->dtype == ISING_F32, f64 = h->dtype == ISING_F64;
  if ((e = f64  ? fm_shape<kFp64, 2>(h, h->nmax, warps0, smem0, per_sm0)
           : fl ? fm_shape<kFx, 1>(h, h->nmax, warps0, smem0, per_sm0)
                : fm_shape<kFx, 0>(h, h->nmax, warps0, smem0, per_sm0)) != cudaSuccess)
    return e;
  const int64_t resident = (int64_t)h->sm_count * per_sm0 * warps0;
  const size_t sp_bytes = ((size_t)R * restarts * h->total_spins + 15) & ~(size_t)15;
  const size_t e_bytes = (size_t)n_items * restarts * sizeof(double);
  const size_t p_bytes = (size_t)n_items * restarts * sizeof(int32_t);
  // fp->starts overrides the choice (both give the same results).
  const bool want = fp->starts ? fp->starts == 2 : n_items < 4 * resident;
  const bool split = want && restarts > 1 && (int64_t)n_items * restarts <= 0x7fffffff &&
                     sp_bytes + e_bytes + p_bytes <= kSplitScratchMax;
  int8_t *sp_k = nullptr;
  double *E_k = nullptr;
  int32_t *P_k = nullptr;
  if (split) {
    if ((e = grow(B.scratch, B.scratch_bytes, sp_bytes + e_bytes + p_bytes)) != cudaSuccess) return e;
    sp_k = static_cast<int8_t *>(B.scratch);
    E_k = reinterpret_cast<double *>(sp_k + sp_bytes);
    P_k = reinterpret_cast<int32_t *>(E_k + (size_t)n_items * restarts);
  }

  // Groups launch largest size class first and, within a class, the group
  // with fewer searches first: its CTAs take their SMs at once, and its
  // searches (as long as the class's others) do not wait for the big group's
  // persistent CTAs to retire.  With several groups they go to side streams
  // (forked from and joined back into s), so that a group's CTAs take the SMs
  // as the previous group's retire instead of waiting for its last search.
  std::vector<size_t> order(parts.size());
  for (size_t q = 0; q < parts.size(); ++q) order[q] = q;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) {
    const int ca = cls(parts[a].nmax), cc = cls(parts[c].nmax);
    return ca != cc ? ca > cc : parts[a].count < parts[c].count;
  });
  const bool fan = parts.size() > 1;
  if (fan) {
    if ((e = ensure_side(B)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(B.fork, s)) != cudaSuccess) return e;
    for (cudaStream_t st : B.side)
      if ((e = cudaStreamWaitEvent(st, B.fork, 0)) != cudaSuccess) return e;
  }
  cudaError_t le = cudaSuccess;
  for (size_t o = 0; o < order.size() && le == cudaSuccess; ++o) {
    const size_t q = order[o];
    const FmPart &P = parts[q];
    cudaStream_t ls = fan ? B.side[o % B.side.size()] : s;
    const int nmax = P.nmax;  // the group's largest instance
    int warps = 0, per_sm = 0;
    size_t smem = 0;
    // Small one-unit instances take the register kernel when the group's
    // searches fit in one wave of it (latency-bound); larger groups keep the
    // shared-memory kernel, which holds more searches per SM.
    const int64_t work = split ? P.count * restarts : P.count;
    const bool reg8 = nmax <= 256;
    bool reg = P.mode == kFx && nmax <= kRegMaxSpins && fp->reg_kernel >= 0;
    if (reg) {
      le = fl ? (reg8 ? fm_reg_shape<true, 8>(h, warps, smem, per_sm) : fm_reg_shape<true, 16>(h, warps, smem, per_sm))
              : (reg8 ? fm_reg_shape<false, 8>(h, warps, smem, per_sm)
                      : fm_reg_shape<false, 16>(h, warps, smem, per_sm));
      if (le != cudaSuccess) break;
      reg = work <= (int64_t)h->sm_count * per_sm * warps || fp->reg_kernel == 1;
    }
    // int8 couplings are always exact in one unit (mode kFx); FP64 couplings
    // take the FP64 form
    if (!reg)
      le = f64 ? fm_shape<kFp64, 2>(h, nmax, warps, smem, per_sm)
           : !fl ? fm_shape<kFx, 0>(h, nmax, warps, smem, per_sm)
           : P.mode == kFx ? fm_shape<kFx, 1>(h, nmax, warps, smem, per_sm)
           : P.mode == kFxSpin ? fm_shape<kFxSpin, 1>(h, nmax, warps, smem, per_sm)
                               : fm_shape<kFp64, 1>(h, nmax, warps, smem, per_sm);
    if (le != cudaSuccess) break;
    FmArgs A;
    A.g = h->graph();
    A.n_work = (int32_t)(split ? P.count * restarts : P.count);
    A.R_out = split ? R * restarts : R;
    A.restarts = restarts;
    A.max_passes = max_passes;
    A.split = split ? 1 : 0;
    A.items = B.items + P.first;
    A.seeds = h->d_seeds;
    A.queue = B.queues + q;
    A.spins = split ? sp_k : spins;
    A.energy = split ? E_k : E;
    A.passes = split ? P_k : passes;
    A.stats = h->d_stats;
    const int64_t ctas_needed = ((int64_t)A.n_work + warps - 1) / warps;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)h->sm_count * per_sm, ctas_needed));
    if (reg && fl && reg8)
      fm_reg_kernel<true, 8><<<grid, warps * 32, smem, ls>>>(A);
    else if (reg && fl)
      fm_reg_kernel<true, 16><<<grid, warps * 32, smem, ls>>>(A);
    else if (reg && reg8)
      fm_reg_kernel<false, 8><<<grid, warps * 32, smem, ls>>>(A);
    else if (reg)
      fm_reg_kernel<false, 16><<<grid, warps * 32, smem, ls>>>(A);
    else if (f64)
      fm_kernel<kFp64, 2><<<grid, warps * 32, smem, ls>>>(A, nmax);
    else if (!fl)
      fm_kernel<kFx, 0><<<grid, warps * 32, smem, ls>>>(A, nmax);
    else if (P.mode == kFx)
      fm_kernel<kFx, 1><<<grid, warps * 32, smem, ls>>>(A, nmax);
    else if (P.mode == kFxSpin)
      fm_kernel<kFxSpin, 1><<<grid, warps * 32, smem, ls>>>(A, nmax);
    else
      fm_kernel<kFp64, 1><<<grid, warps * 32, smem, ls>>>(A, nmax);
    h->launches += 1;
    le = cudaGetLastError();
  }
  if (fan)  // join every side stream back into s, also after a failed launch
    for (size_t j = 0; j < B.side.size(); ++j) {
      cudaError_t je = cudaEventRecord(B.join[j], B.side[j]);
      if (je == cudaSuccess) je = cudaStreamWaitEvent(s, B.join[j], 0);
      if (le == cudaSuccess) le = je;
    }
  if (le != cudaSuccess) return le;
  if (!split) return cudaSuccess;
  const int64_t threads = n_items * 32;
  fm_best_start_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(h->d_inst, h->n_inst, R, restarts, sp_k,
                                                                         E_k, P_k, spins, E, passes);
  h->launches += 1;
  return cudaGetLastError();
}

void fm_free(ising_handle *h) {
  if (!h->fm_st) return;
  FmBufs &B = static_cast<FmBufs &>(*h->fm_st);
  cudaFree(B.items);
  cudaFree(B.queues);
  cudaFree(B.scratch);
  for (cudaStream_t st : B.side) cudaStreamDestroy(st);
  for (cudaEvent_t ev : B.join) cudaEventDestroy(ev);
  if (B.fork) cudaEventDestroy(B.fork);
  h->fm_st.reset();
}

}  // namespace isg
