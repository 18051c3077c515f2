// selftest.cu — ising_check_rounding: the integer-only rounding the field
// refresh uses (xr_round_int) checked against the hardware int64 -> FP32
// conversion (xr_round) on a device the library runs on.
#include "device_common.cuh"

namespace isg {

namespace {

// Case t: a value |s| <= 2^53 and a unit in [24, 200].  Three quarters of the
// cases put the leading one at a random bit m in [24, 53) and a constructed
// tail below the kept 24 bits: exactly half a unit in the last place, one
// above, one below, or random; the rest are random integers of random length
// (including short ones, kept whole) and the extremes 0 and +/-2^53.
__device__ void rounding_case(uint64_t seed, uint64_t t, int64_t &s, int &unit) {
  const uint4 x = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), 0x52u, 0x4E44u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  unit = 24 + (int)(x.w % 177u);
  const uint64_t rnd = ((uint64_t)x.y << 32) | x.z;
  uint64_t mag;
  const uint32_t kind = x.x & 7u;
  if (kind < 6) {
    const int m = 24 + (int)((x.x >> 3) % 29u);  // 24 .. 52
    const int sh = m - 23;
    const uint64_t sig = (1ull << 23) | (rnd & 0x7fffffull);
    const uint64_t half = 1ull << (sh - 1), lowmask = (1ull << sh) - 1ull;
    uint64_t low;
    switch (kind) {
      case 0: low = half; break;
      case 1: low = half + 1; break;
      case 2: low = half - 1; break;
      default: low = (rnd >> 23) & lowmask; break;
    }
    mag = (sig << sh) | (low & lowmask);
  } else if (kind == 6) {
    const int len = (int)((x.x >> 3) % 54u);  // 0 .. 53 bits
    mag = len == 0 ? 0 : (rnd & ((1ull << len) - 1ull));
  } else {
    mag = (x.x >> 3) & 1u ? (1ull << 53) : 0ull;
  }
  s = ((x.w >> 16) & 1u) ? -(int64_t)mag : (int64_t)mag;
}

__global__ void check_rounding_kernel(uint64_t seed, int64_t count, unsigned long long *bad) {
  unsigned long long mine = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t s;
    int unit;
    rounding_case(seed, (uint64_t)t, s, unit);
    if (__float_as_uint(xr_round(s, unit)) != __float_as_uint(xr_round_int(s, unit))) ++mine;
  }
  if (mine) atomicAdd(bad, mine);
}

}  // namespace

}  // namespace isg

extern "C" ising_status ising_check_rounding(uint64_t seed, int64_t count, uint64_t *mismatches) {
  using namespace isg;
  if (count < 0 || !mismatches) return ISING_ERR_INVALID_ARG;
  unsigned long long *d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) return ISING_ERR_OOM;
  ising_status st = ISING_OK;
  unsigned long long h = 0;
  int dev = 0, sms = 0;
  if (cudaMemset(d, 0, sizeof(unsigned long long)) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    st = ISING_ERR_CUDA;
  } else {
    check_rounding_kernel<<<sms * 8, 256>>>(seed, count, d);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(&h, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = ISING_ERR_CUDA;
  }
  cudaFree(d);
  *mismatches = h;
  return st;
}
