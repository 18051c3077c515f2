// dense_push.cu — the late part of a dense descent: the paper's incremental
// gain update (Sec. IV), one warp per replica on CUDA cores.
//
// After the first sweeps of a descent on tensor cores (dense_tc.cu) most
// replicas flip few spins per sweep, and the number of sweeps a replica needs
// varies widely (for SK n = 4096, from about 20 to over 100).  Recomputing a
// block's fields as a GEMM costs the same whether one spin or a hundred flip,
// and in lockstep every replica pays for the slowest one.  Here each replica
// proceeds on its own: its FP32 fields f_i = h_i + sum_j J_ij s_j live in
// shared memory, a sweep visits the spins in index order (sequential
// schedule), and a flip of spin i adds 2 J_ij s_i (s_i the new value) to every
// field f_j, reading row i of J (row i = column i, J symmetric; J_ii = 0 leaves
// f_i unchanged).  Fields change only at flips, so the warp evaluates 128
// spins at once (four 32-spin ballots) and jumps to the first spin that flips;
// the spins it passes over keep their decisions, as in a one-by-one visit.
//
// A replica leaves when a sweep flips nothing (a 1-flip minimum), or at the
// descent's sweep cap or the sweep budget.  It then records its energy
//     E = -1/2 sum_i s_i (f_i + h_i)
// (FP64 sum in a fixed order; the search uses it only to keep the best state)
// and writes its spins back.
#include <cuda_bf16.h>

#include <algorithm>

#include "dense.cuh"
#include "device_common.cuh"

namespace isg {

namespace {

constexpr int kMaxWarps = 16;
constexpr int kBatch = 8;  // coupling-row float4 loads in flight per lane

struct PushArgs {
  int32_t n, R, max_sweeps, budget;
  const float *J;      // [n][n]
  const float *h;      // [n]
  const float *F;      // [R][n] fields at entry
  __nv_bfloat16 *S;    // [Rp][n] spins
  DenseRep *rep;       // [R]
  int32_t *counter;    // next replica to take (zero at launch)
  unsigned long long *stats;
};

// f_j += c J_ij for all j; c = +/-2, so c J_ij is exact and each field sees one
// rounding, as when its update is added on its own.
__device__ __forceinline__ void push_row(float *F, const float *__restrict__ Jrow, float c, int n, int lane) {
  const float4 *J4 = reinterpret_cast<const float4 *>(Jrow);
  float4 *F4 = reinterpret_cast<float4 *>(F);
  const int n4 = n >> 2;  // a multiple of 32 * kBatch when n % 1024 == 0; tail handled below
  int t = lane;
  for (; t + 32 * (kBatch - 1) < n4; t += 32 * kBatch) {
    float4 j[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) j[u] = __ldg(J4 + t + 32 * u);
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      float4 f = F4[t + 32 * u];
      f.x = __fmaf_rn(c, j[u].x, f.x);
      f.y = __fmaf_rn(c, j[u].y, f.y);
      f.z = __fmaf_rn(c, j[u].z, f.z);
      f.w = __fmaf_rn(c, j[u].w, f.w);
      F4[t + 32 * u] = f;
    }
  }
  for (; t < n4; t += 32) {
    const float4 j = __ldg(J4 + t);
    float4 f = F4[t];
    f.x = __fmaf_rn(c, j.x, f.x);
    f.y = __fmaf_rn(c, j.y, f.y);
    f.z = __fmaf_rn(c, j.z, f.z);
    f.w = __fmaf_rn(c, j.w, f.w);
    F4[t] = f;
  }
}

__global__ void __launch_bounds__(kMaxWarps * 32) dense_push_kernel(PushArgs A) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = A.n, nw = n >> 5;
  float *F = reinterpret_cast<float *>(smem4) + (size_t)warp * (n + nw);  // n fields, then nw spin words
  uint32_t *bits = reinterpret_cast<uint32_t *>(F + n);
  unsigned long long c_evals = 0, c_flips = 0, c_sweeps = 0;
  for (;;) {
    int r = 0;
    if (lane == 0) r = atomicAdd(A.counter, 1);
    r = __shfl_sync(0xffffffffu, r, 0);
    if (r >= A.R) break;
    DenseRep st = A.rep[r];
    if (!st.active) continue;
    const float4 *src = reinterpret_cast<const float4 *>(A.F + (size_t)r * n);
    for (int t = lane; t < (n >> 2); t += 32) reinterpret_cast<float4 *>(F)[t] = src[t];
    __nv_bfloat16 *row = A.S + (size_t)r * n;
    for (int w = 0; w < nw; ++w) {
      const uint32_t m = __ballot_sync(0xffffffffu, __bfloat162float(row[32 * w + lane]) > 0.0f);
      if (lane == 0) bits[w] = m;
    }
    __syncwarp();
    for (;;) {  // sweeps
      int nfl = 0;
      int pos = 0;  // next spin to decide
      while (pos < n) {
        const int w0 = pos >> 5;
        uint32_t mm[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int w = w0 + q;
          bool dec = false;
          if (w < nw) {
            const float f = F[32 * w + lane];
            dec = ((bits[w] >> lane) & 1u) ? (f < 0.0f) : (f > 0.0f);
          }
          mm[q] = __ballot_sync(0xffffffffu, dec);
        }
        mm[0] &= 0xffffffffu << (pos & 31);
        int q = 0;
        while (q < 4 && !mm[q]) ++q;
        if (q == 4) {
          pos = 32 * (w0 + 4);
          continue;
        }
        const int w = w0 + q, li = __ffs(mm[q]) - 1, i = 32 * w + li;
        const bool was_up = (bits[w] >> li) & 1u;
        __syncwarp();
        if (lane == 0) bits[w] ^= 1u << li;
        push_row(F, A.J + (size_t)i * n, was_up ? -2.0f : 2.0f, n, lane);
        __syncwarp();
        ++nfl;
        pos = i + 1;
      }
      st.d += 1;
      st.total += 1;
      c_evals += (unsigned long long)n;
      c_sweeps += 1;
      c_flips += (unsigned long long)nfl;
      if (nfl == 0 || st.d >= A.max_sweeps || (A.budget > 0 && st.total >= A.budget)) {
        st.conv = nfl == 0 ? 1 : 0;
        st.active = 0;
        break;
      }
    }
    double acc = 0.0;
    for (int i = lane; i < n; i += 32) {
      const bool up = (bits[i >> 5] >> lane) & 1u;
      const double v = (double)F[i] + (double)__ldg(A.h + i);
      acc += up ? v : -v;
    }
    acc = warp_sum(acc);
    st.E = -0.5 * acc;
    for (int i = lane; i < n; i += 32)
      row[i] = __float2bfloat16_rn(((bits[i >> 5] >> lane) & 1u) ? 1.0f : -1.0f);
    if (lane == 0) A.rep[r] = st;
    __syncwarp();
  }
  if (lane == 0 && c_sweeps) {
    atomicAdd(A.stats + 0, c_evals);
    atomicAdd(A.stats + 1, c_flips);
    atomicAdd(A.stats + 4, c_sweeps);
  }
}

}  // namespace

cudaError_t dense_push_run(int n, int R, int max_sweeps, int budget, const float *J, const float *h, const float *F,
                           __nv_bfloat16 *S, DenseRep *rep, int32_t *counter, unsigned long long *stats, int sm_count,
                           cudaStream_t s) {
  if (n % 32 != 0 || n < 32) return cudaErrorInvalidValue;
  const size_t per_warp = (size_t)(n + n / 32) * sizeof(float);
  int dev = 0, smem_max = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  const int warps = (int)std::min<size_t>(kMaxWarps, (size_t)smem_max / per_warp);
  if (warps < 1) return cudaErrorInvalidValue;
  const size_t smem = per_warp * warps;
  if ((e = cudaFuncSetAttribute(dense_push_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense_push_kernel, warps * 32, smem)) !=
      cudaSuccess)
    return e;
  const int grid = std::max(1, std::min(sm_count * std::max(per_sm, 1), (R + warps - 1) / warps));
  PushArgs A;
  A.n = n;
  A.R = R;
  A.max_sweeps = max_sweeps;
  A.budget = budget;
  A.J = J;
  A.h = h;
  A.F = F;
  A.S = S;
  A.rep = rep;
  A.counter = counter;
  A.stats = stats;
  dense_push_kernel<<<grid, warps * 32, smem, s>>>(A);
  return cudaGetLastError();
}

}  // namespace isg
