// device_common.cuh — device helpers shared by the kernels: Philox4x32-10
// random starts, bit-packed spin access and deterministic block reductions.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace isg {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// published multiply/xor round function with its Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// 128 random start bits for spins 128*w .. 128*w+127 of replica r, descent k,
// instance b (the counter layout of the C ABI).
__device__ __forceinline__ uint4 start_bits(uint64_t seed, uint32_t w, uint32_t r, uint32_t k,
                                            uint32_t b) {
  return philox4x32_10(make_uint4(w, r, k, b),
                       make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)));
}

__device__ __forceinline__ uint32_t word_of(const uint4 &x, int t) {
  return t == 0 ? x.x : (t == 1 ? x.y : (t == 2 ? x.z : x.w));
}

// ---- exact field refresh without FP64 arithmetic ------------------------
// A refresh is defined as a sequential FP64 sum of FP32 terms (field, then the
// couplings) rounded once to FP32.  When every partial sum of that sequence is
// exactly representable in FP64 the sequence never rounds, and the result is
// the round-to-nearest FP32 value of the exact sum.  With e the biased
// exponents of the nonzero terms this holds when min e >= 24 (no subnormals),
// max e <= 200 and k terms of at most 24 + (max e - min e) bits sum below 2^53.
// The exact sum is then formed in 64-bit fixed point with unit 2^(emin - 150).
struct XRange {
  int emin = 256, emax = -1, k = 0;
};

__device__ __forceinline__ void xr_see(XRange &r, float w) {
  const uint32_t a = __float_as_uint(w) & 0x7fffffffu;
  r.k += 1;
  if (a) {
    const int e = (int)(a >> 23);
    r.emin = min(r.emin, e);
    r.emax = max(r.emax, e);
  }
}

__device__ __forceinline__ bool xr_exact(const XRange &r) {
  if (r.emax < 0) return true;  // every term is zero
  const int lg = 32 - __clz(r.k);  // 2^lg > k
  return r.emin >= 24 && r.emax <= 200 && (r.emax - r.emin) + 24 + lg <= 53;
}

// w as a signed integer multiple of 2^(unit - 150); needs unit <= e(w) <= unit + 38.
__device__ __forceinline__ int64_t xr_term(float w, int unit) {
  const uint32_t b = __float_as_uint(w), a = b & 0x7fffffffu;
  if (!a) return 0;
  const int64_t t = (int64_t)((a & 0x7fffffu) | 0x800000u) << ((int)(a >> 23) - unit);
  return (b >> 31) ? -t : t;
}

// RN32(s * 2^(unit - 150)) for |s| <= 2^53, unit >= 24: the integer is
// rounded once to FP32 and scaled by an exact power of two.
__device__ __forceinline__ float xr_round(int64_t s, int unit) {
  return __ll2float_rn(s) * __int_as_float((unit - 23) << 23);
}

// ---- FP64 instances ---------------------------------------------------------
// The energy of one configuration of an ISING_F64 instance, as the C ABI
// defines it: Neumaier's compensated sum (Neumaier 1974) of the terms
// -J_ij s_i s_j (row i in stored order, j > i) and -h_i s_i for i = 0..n-1,
// then -J_e prod_{k in e} s_k over the hyper-edges in order; every step one
// IEEE FP64 addition (no contraction), by one thread.
__device__ inline double energy_f64_seq(const DevGraph &G, const InstDesc &I, const int8_t *s) {
  const double *J = reinterpret_cast<const double *>(G.J);
  const double *h = reinterpret_cast<const double *>(G.h);
  const double *hJ = reinterpret_cast<const double *>(G.hJ);
  double sum = 0.0, comp = 0.0;
  auto add = [&](double x) {
    const double t = __dadd_rn(sum, x);
    if (fabs(sum) >= fabs(x)) comp = __dadd_rn(comp, __dadd_rn(__dsub_rn(sum, t), x));
    else comp = __dadd_rn(comp, __dadd_rn(__dsub_rn(x, t), sum));
    sum = t;
  };
  for (int i = 0; i < I.n; ++i) {
    const int64_t gi = I.spin_off + i;
    for (uint32_t k = G.row[gi], ke = G.row[gi + 1]; k < ke; ++k) {
      const int j = G.col[k];
      if (j > i) {
        const double w = J[k];
        add(s[i] == s[j] ? -w : w);
      }
    }
    const double hv = h[gi];
    add(s[i] > 0 ? -hv : hv);
  }
  for (int e = 0; e < I.n_hyper; ++e) {
    const int64_t ge = I.hyper_off + e;
    int neg = 0;
    for (uint32_t q = G.hptr[ge], qe = G.hptr[ge + 1]; q < qe; ++q) neg ^= s[G.hmem[q]] < 0;
    const double w = hJ[ge];
    add(neg ? w : -w);
  }
  return __dadd_rn(sum, comp);
}

// ---- exact energies ------------------------------------------------------
// Energy terms as integers t (unit 2^(ebase - 150), |t| < 2^62) accumulated as
// a signed high part (t >> 32) and an unsigned low part (t & 0xffffffff):
// integer sums, so the total does not depend on the order of the additions.
__device__ __forceinline__ void xe_add(long long &hi, unsigned long long &lo, int64_t t) {
  hi += (long long)(t >> 32);
  lo += (unsigned long long)(uint32_t)t;
}

// Round the exact total hi * 2^32 + lo (times the unit) once to FP64.
__device__ __forceinline__ double xe_value(long long hi, unsigned long long lo, int ebase) {
  hi += (long long)(lo >> 32);
  lo &= 0xffffffffull;
  const double v = __fma_rn((double)hi, 4294967296.0, (double)lo);
  return v * __longlong_as_double((long long)(ebase - 150 + 1023) << 52);
}

// 32 x 32 bit transpose across a warp: lane i holds row i (bit c = column c);
// returns column `lane` (bit i = row i's bit `lane`).  Five exchange stages,
// each swapping the off-diagonal halves of 2j x 2j blocks between lanes i and i^j.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t v, int lane) {
  const uint32_t m[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int j = 16 >> s;
    const uint32_t t = __shfl_xor_sync(0xffffffffu, v, j);
    v = (lane & j) ? ((v & ~m[s]) | ((t & ~m[s]) >> j)) : ((v & m[s]) | ((t & m[s]) << j));
  }
  return v;
}

// Warp total of bit-sliced per-lane counters: plane q of every lane holds bit
// q of 32 counters (one per bit position r).  A butterfly of bit-sliced adds
// leaves every lane with the warp-wide sums (Q + 5 planes); lane r then reads
// counter r's total from bit r of each plane.
template <int Q>
__device__ __forceinline__ long long warp_sliced_total(const uint32_t (&acc)[Q], int lane) {
  uint32_t w[Q + 5];
#pragma unroll
  for (int q = 0; q < Q + 5; ++q) w[q] = q < Q ? acc[q] : 0u;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int j = 16 >> s;
    uint32_t carry = 0u;
#pragma unroll
    for (int q = 0; q < Q + 5; ++q) {
      const uint32_t o = __shfl_xor_sync(0xffffffffu, w[q], j);
      const uint32_t x = w[q];
      w[q] = x ^ o ^ carry;
      carry = (x & o) | (x & carry) | (o & carry);
    }
  }
  long long total = 0;
#pragma unroll
  for (int q = 0; q < Q + 5; ++q) total += (long long)((w[q] >> lane) & 1u) << q;
  return total;
}

template <class T>
__device__ __forceinline__ T ldg_val(const void *p, int64_t i) {
  return __ldg(reinterpret_cast<const T *>(p) + i);
}

// Warp sum with a fixed butterfly order (deterministic).
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum in a fixed order: butterfly inside each warp, then warps in
// ascending order by thread 0.  `red` holds one slot per warp.  The result is
// returned to every thread.
template <class T>
__device__ T block_sum(T v, T *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    T acc = red[0];
    for (int w = 1; w < nw; ++w) acc += red[w];
    red[0] = acc;
  }
  __syncthreads();
  T out = red[0];
  __syncthreads();
  return out;
}

}  // namespace isg
