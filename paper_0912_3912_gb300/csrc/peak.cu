// peak.cu — measured issue rate of 32-bit logic operations on the current GPU,
// the denominator of the roofline of the multi-spin-coded kernels (whose
// work is word-wide and/or/xor on 32 replicas at a time), and the replica-bit
// rate of the same logic on 32- and 64-bit words (the multi-spin word width).
//
// Every thread runs eight dependent-in-turn chains of three-input logic ops
// (lop3.b32) on registers; with 2048 resident threads per SM the scheduler
// always has independent instructions, so the kernel runs at the rate the
// logic pipe issues.  Lane-ops/s = threads x iterations x ops per iteration /
// elapsed time.
#include <cuda_runtime.h>

#include <cstdint>

#include "ising.h"

namespace {

constexpr int kPT = 256;        // threads per CTA
constexpr int kChains = 8;      // independent registers per thread
constexpr int kUnroll = 16;     // rounds over the chains per loop iteration

__global__ void __launch_bounds__(kPT) logic_peak_kernel(uint32_t *out, int iters, uint32_t seed) {
  uint32_t x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = seed ^ (uint32_t)(threadIdx.x * kChains + i) ^ (blockIdx.x << 16);
  const uint32_t y = seed * 2654435761u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i)
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[i]) : "r"(x[(i + 1) % kChains]), "r"(y));
  }
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc ^= x[i];
  if (acc == seed) out[0] = acc;  // keeps every chain live
}

// Chains of two-input XORs on words of W (32 or 64 bits), each one PTX xor of
// that width kept in place (volatile), for the replica-bit rate of multi-spin
// coding at either word width.
__device__ __forceinline__ void xor_w(uint32_t &x, uint32_t y) { asm volatile("xor.b32 %0, %0, %1;" : "+r"(x) : "r"(y)); }
__device__ __forceinline__ void xor_w(unsigned long long &x, unsigned long long y) {
  asm volatile("xor.b64 %0, %0, %1;" : "+l"(x) : "l"(y));
}

template <typename W>
__global__ void __launch_bounds__(kPT) logic_bits_kernel(W *out, int iters, uint32_t seed) {
  W x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = (W)(seed ^ (uint32_t)(threadIdx.x * kChains + i)) * (W)0x9E3779B97F4A7C15ull;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) xor_w(x[i], x[(i + 1) % kChains]);
  }
  W acc = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc ^= x[i];
  if (acc == (W)seed) out[0] = acc;  // keeps every chain live
}

template <typename W>
ising_status bits_rate(double *bit_ops_per_s) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, logic_bits_kernel<W>, kPT, 0) != cudaSuccess ||
      per_sm < 1)
    return ISING_ERR_CUDA;
  W *out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  ising_status st = ISING_OK;
  if (cudaMalloc(&out, sizeof(W)) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    st = ISING_ERR_CUDA;
  } else {
    const int grid = sms * per_sm;
    const int iters = sizeof(W) == 8 ? 2048 : 4096;  // about 10 ms each at 2 GHz
    double best = 0.0;
    logic_bits_kernel<W><<<grid, kPT, 0, s>>>(out, 64, 1u);  // warm-up
    for (int rep = 0; rep < 3 && st == ISING_OK; ++rep) {
      float ms = 0.0f;
      if (cudaEventRecord(a, s) != cudaSuccess) st = ISING_ERR_CUDA;
      logic_bits_kernel<W><<<grid, kPT, 0, s>>>(out, iters, 2u + (uint32_t)rep);
      if (st == ISING_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(b, s) != cudaSuccess ||
                             cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
        st = ISING_ERR_CUDA;
      if (st == ISING_OK && ms > 0.0f) {
        // one XOR per chain step on sizeof(W) x 8 replica bits
        const double ops = (double)grid * kPT * (double)iters * kUnroll * kChains * (8.0 * sizeof(W));
        const double rate = ops / (ms * 1e-3);
        if (rate > best) best = rate;
      }
    }
    if (st == ISING_OK) *bit_ops_per_s = best;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  return st;
}

}  // namespace

extern "C" ising_status ising_logic_bits_rate(int32_t word_bits, double *bit_ops_per_s) {
  if (!bit_ops_per_s || (word_bits != 32 && word_bits != 64)) return ISING_ERR_INVALID_ARG;
  *bit_ops_per_s = 0.0;
  return word_bits == 32 ? bits_rate<uint32_t>(bit_ops_per_s) : bits_rate<unsigned long long>(bit_ops_per_s);
}

extern "C" ising_status ising_logic_peak(double *lane_ops_per_s) {
  if (!lane_ops_per_s) return ISING_ERR_INVALID_ARG;
  *lane_ops_per_s = 0.0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, logic_peak_kernel, kPT, 0) != cudaSuccess || per_sm < 1)
    return ISING_ERR_CUDA;
  uint32_t *out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  ising_status st = ISING_OK;
  if (cudaMalloc(&out, sizeof(uint32_t)) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    st = ISING_ERR_CUDA;
  } else {
    const int grid = sms * per_sm;
    const int iters = 4096;  // about 10 ms at 2 GHz
    double best = 0.0;
    logic_peak_kernel<<<grid, kPT, 0, s>>>(out, 64, 1u);  // warm-up
    for (int rep = 0; rep < 3 && st == ISING_OK; ++rep) {
      float ms = 0.0f;
      if (cudaEventRecord(a, s) != cudaSuccess) st = ISING_ERR_CUDA;
      logic_peak_kernel<<<grid, kPT, 0, s>>>(out, iters, 2u + (uint32_t)rep);
      if (st == ISING_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(b, s) != cudaSuccess ||
                             cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
        st = ISING_ERR_CUDA;
      if (st == ISING_OK && ms > 0.0f) {
        const double ops = (double)grid * kPT * (double)iters * kUnroll * kChains;
        const double rate = ops / (ms * 1e-3);
        if (rate > best) best = rate;
      }
    }
    if (st == ISING_OK) *lane_ops_per_s = best;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  return st;
}
