// noalloc.cu — ising_energy_noalloc: the energy evaluation of ising_energy for
// callers that cannot allocate device memory.
//
// Some callers own all of the device memory through their own pool allocator
// (a framework that reserves the device up front), or run where a cudaMalloc
// would synchronise the whole device and stall their other streams.  They can
// neither create a handle (ising_create uploads the instance into memory it
// allocates) nor let ising_energy grow its scratch on first use.  This entry
// point takes the instance and the configurations as the caller's own device
// buffers and keeps its only scratch - the per-chunk partial sums of the
// two-pass, fixed-order reduction - in the file-scope array below.
//
// The array exists once per device that loads this library and lives until the
// process exits.  Every call shares it and overwrites it (the first pass writes
// every slot the second pass reads, so nothing needs clearing between calls);
// calls that overlap on the GPU - on different streams, or from different
// threads without ordering - race on it.
#include <mutex>

#include "device_common.cuh"

namespace isg {

namespace {

constexpr int kNaChunk = 4096;      // spins per partial sum
constexpr int kNaThreads = 256;
constexpr int kNaMaxDevices = 64;

// 65,536 partial sums (512 KiB): chunks(n) * replicas must not exceed this.
static __device__ __align__(256) double g_noalloc_partials[ISING_NOALLOC_MAX_PARTIALS];

std::mutex g_na_mutex;
double *g_na_ptr[kNaMaxDevices] = {nullptr};

template <bool FLOAT>
__global__ void __launch_bounds__(kNaThreads)
noalloc_partial(int32_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                const void *__restrict__ J, const void *__restrict__ h, const int8_t *__restrict__ spins,
                int32_t nchunks, double *partials) {
  __shared__ double redd[kNaThreads / 32];
  __shared__ long long redi[kNaThreads / 32];
  const int r = blockIdx.x / nchunks, c = blockIdx.x % nchunks;
  const int8_t *s = spins + (int64_t)r * n;
  const int i0 = c * kNaChunk, i1 = min(n, i0 + kNaChunk);
  if (FLOAT) {
    const float *Jf = reinterpret_cast<const float *>(J);
    const float *hf = reinterpret_cast<const float *>(h);
    double acc = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const double si = (double)s[i];
      double e = hf ? (double)__ldg(hf + i) * si : 0.0;
      for (int64_t k = __ldg(row_ptr + i), ke = __ldg(row_ptr + i + 1); k < ke; ++k) {
        const int j = __ldg(col + k);
        if (j > i) e += (double)__ldg(Jf + k) * si * (double)s[j];
      }
      acc -= e;
    }
    acc = block_sum(acc, redd);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  } else {
    const int8_t *Ji = reinterpret_cast<const int8_t *>(J);
    const int8_t *hi = reinterpret_cast<const int8_t *>(h);
    long long acc = 0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const int si = s[i];
      int e = hi ? (int)__ldg(hi + i) * si : 0;
      for (int64_t k = __ldg(row_ptr + i), ke = __ldg(row_ptr + i + 1); k < ke; ++k) {
        const int j = __ldg(col + k);
        if (j > i) e += (int)__ldg(Ji + k) * si * (int)s[j];
      }
      acc -= e;
    }
    acc = block_sum(acc, redi);
    if (threadIdx.x == 0) partials[blockIdx.x] = (double)acc;
  }
}

__global__ void noalloc_finish(int32_t replicas, int32_t nchunks, const double *partials, double *E) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= replicas) return;
  double acc = 0.0;
  for (int c = 0; c < nchunks; ++c) acc += partials[(int64_t)r * nchunks + c];
  E[r] = acc;
}

// Device address of the scratch array for the current device.  Outside stream
// capture it is looked up on every call (cudaGetSymbolAddress allocates
// nothing), so a context that was torn down and recreated - cudaDeviceReset, or
// the primary context released and retained again - never leaves a stale
// address behind.  While `stream` is capturing, the address recorded by the
// last uncaptured call on this device is used instead (a lookup there could
// load the module, which capture forbids).
cudaError_t scratch_address(cudaStream_t stream, double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<double *>(p);
  } else if (!g_na_ptr[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace isg

extern "C" ising_status ising_energy_noalloc(int32_t n, const int64_t *row_ptr_dev, const int32_t *col_dev,
                                             const void *J_dev, const void *h_dev, ising_dtype dtype,
                                             const int8_t *spins_dev, int32_t replicas, double *energy_dev,
                                             cudaStream_t stream) {
  using namespace isg;
  if (n < 1 || replicas < 1 || !row_ptr_dev || !col_dev || !J_dev || !spins_dev || !energy_dev)
    return ISING_ERR_INVALID_ARG;
  if (dtype != ISING_I8 && dtype != ISING_F32) return ISING_ERR_INVALID_ARG;
  const int64_t nchunks = (n + kNaChunk - 1) / kNaChunk;
  if (nchunks * (int64_t)replicas > (int64_t)ISING_NOALLOC_MAX_PARTIALS) return ISING_ERR_UNSUPPORTED;
  double *partials = nullptr;
  if (scratch_address(stream, &partials) != cudaSuccess) return ISING_ERR_CUDA;
  const int blocks = (int)(nchunks * replicas);
  if (dtype == ISING_F32)
    noalloc_partial<true><<<blocks, kNaThreads, 0, stream>>>(n, row_ptr_dev, col_dev, J_dev, h_dev, spins_dev,
                                                             (int32_t)nchunks, partials);
  else
    noalloc_partial<false><<<blocks, kNaThreads, 0, stream>>>(n, row_ptr_dev, col_dev, J_dev, h_dev, spins_dev,
                                                              (int32_t)nchunks, partials);
  if (cudaGetLastError() != cudaSuccess) return ISING_ERR_CUDA;
  noalloc_finish<<<(replicas + 255) / 256, 256, 0, stream>>>(replicas, (int32_t)nchunks, partials, energy_dev);
  if (cudaGetLastError() != cudaSuccess) return ISING_ERR_CUDA;
  return ISING_OK;
}
