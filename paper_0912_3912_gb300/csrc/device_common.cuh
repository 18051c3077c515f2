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
