// dense_push.cu — the late part of a dense descent: the paper's incremental
// gain update (Sec. IV), one CTA per replica on CUDA cores.
//
// After the first sweeps of a descent on tensor cores (dense_tc.cu) most
// replicas flip few spins per sweep, and the number of sweeps a replica needs
// varies widely (for SK n = 4096, from about 20 to over 100).  Recomputing a
// block's fields as a GEMM costs the same whether one spin or a hundred flip,
// and in lockstep every replica pays for the slowest one.  Here each replica
// proceeds on its own (one CTA of 128 threads): its FP32 fields
// f_i = h_i + sum_j J_ij s_j live in registers (32 per thread at n = 4096), a
// sweep visits the spins in index order (sequential schedule), and a flip of
// spin i adds 2 J_ij s_i (s_i the new value) to every field f_j, reading row i
// of J (row i = column i, J symmetric; J_ii = 0 leaves f_i unchanged).  Per
// flip only the coupling row moves through the memory system.
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

// One CTA per replica: 128 threads for n <= 4096, 256 for n <= 8192, 512 for
// n <= 16384, each with at most kSlots float4 field slots.
constexpr int kSlots = 8;
constexpr int kNone = 0x7fffffff;

struct PushArgs {
  int32_t n, n_eval, R, max_sweeps, budget;  // n: row length (padded); n_eval: the instance's spins
  const float *J;      // [n][n]
  const float *h;      // [n]
  const float *F;      // [R][n] fields at entry
  __nv_bfloat16 *S;    // [Rp][n] spins
  DenseRep *rep;       // [R]
  int32_t *counter;    // next replica to take (zero at launch)
  unsigned long long *stats;
};

// Layout: thread t of TH holds, in slot k, the fields and spins of the four
// spins j = 4 (t + TH k) + e, e = 0..3, so slot k of the CTA covers the
// 4 TH-spin group [4 TH k, 4 TH (k + 1)) in order of (t, e), and a coupling row
// is read as one coalesced float4 per thread and slot.
//
// A sweep visits the groups in order.  In a group every thread evaluates its
// own four spins (those after the last flip), the CTA takes the first one in
// index order that flips (the minimum over the threads, exchanged through
// shared memory at one barrier), and if there is one, every thread adds
// c J_ij to its fields (c = 2 s_i after the flip: exact, so each field sees one
// rounding) and the group is evaluated again after spin i.  The spins it
// passes over keep their decisions, as in a one-by-one visit, because fields
// change only at flips.
//
// NS = slots per thread (groups); GUARD: n is not 4 TH NS, so the last group is
// partial and spins j >= n are masked out.
template <int NS, bool GUARD, int TH>
__global__ void __launch_bounds__(TH, TH == 128 ? (GUARD ? 6 : 7) : (TH == 256 ? 3 : 1)) dense_push_kernel(PushArgs A) {
  constexpr int kThreads = TH;
  __shared__ int s_r;
  __shared__ int s_min[2][kThreads / 32];
  __shared__ double s_e[kThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int n = A.n;
  // valid bit 4 k + e: spin 4 (t + kThreads k) + e exists
  uint32_t valid = 0xffffffffu;
  if (GUARD) {
    valid = 0;
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (4 * (t + kThreads * k) + e < n) valid |= 1u << (4 * k + e);
  }
  uint32_t c_sweeps = 0;  // flip evaluations = c_sweeps * n
  unsigned long long c_flips = 0;
  int par = 0;  // s_min buffer in use (alternates, so one barrier per exchange suffices)
  for (;;) {
    if (t == 0) s_r = atomicAdd(A.counter, 1);
    __syncthreads();
    const int r = s_r;
    __syncthreads();  // s_r is rewritten only after every thread has read it
    if (r >= A.R) break;
    if (!A.rep[r].active) continue;
    // the only state the sweeps change (the rest of DenseRep stays in memory)
    int st_d = A.rep[r].d, st_total = A.rep[r].total, st_conv = 0;
    float4 f[NS];
    uint32_t sb = 0;  // bit 4 k + e: spin 4 (t + kThreads k) + e is +1
    const float4 *F4 = reinterpret_cast<const float4 *>(A.F + (size_t)r * n);
    __nv_bfloat16 *row = A.S + (size_t)r * n;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const int j = 4 * (t + kThreads * k);
      f[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!GUARD || j < n) {
        f[k] = F4[t + kThreads * k];
        const uint2 sv = *reinterpret_cast<const uint2 *>(row + j);  // four BF16 spins
        // spin e is the BF16 in half e of (sv.x, sv.y); sign bit clear: +1
        const uint32_t nx = ~sv.x, ny = ~sv.y;
        const uint32_t up4 = ((nx >> 15) & 1u) | ((nx >> 30) & 2u) | (((ny >> 15) & 1u) << 2) | (((ny >> 31) & 1u) << 3);
        sb |= up4 << (4 * k);
      }
    }
    sb &= valid;
    for (;;) {  // sweeps
      int nfl = 0;
#pragma unroll
      for (int g = 0; g < NS; ++g) {
        const int j0 = 4 * (t + kThreads * g);
        int from = 4 * kThreads * g;  // first spin of the group still to decide
        for (;;) {
          // this thread's first flipping spin of group g at or after `from`:
          // spin e flips iff its field is nonzero with the sign of its spin
          // (s_e = +1 and f_e < 0, or s_e = -1 and f_e > 0)
          const uint32_t upm = (sb >> (4 * g)) & 0xFu;
          const uint32_t ux = __float_as_uint(f[g].x), uy = __float_as_uint(f[g].y);
          const uint32_t uz = __float_as_uint(f[g].z), uw = __float_as_uint(f[g].w);
          const uint32_t sgn = (ux >> 31) | ((uy >> 30) & 2u) | ((uz >> 29) & 4u) | ((uw >> 28) & 8u);
          const uint32_t nz = ((ux << 1) != 0u ? 1u : 0u) | ((uy << 1) != 0u ? 2u : 0u) |
                              ((uz << 1) != 0u ? 4u : 0u) | ((uw << 1) != 0u ? 8u : 0u);
          const int lim = min(max(from - j0, 0), 4);
          const uint32_t dec = ~(sgn ^ upm) & nz & (0xFu << lim) & (valid >> (4 * g));
          int cand = kNone;
          if (dec & 0xFu) {
            const int e = __ffs(dec) - 1;
            cand = 2 * (j0 + e) + (int)((upm >> e) & 1u);
          }
          // CTA minimum: warp minimum by ballot, then the four warps' minima
          const uint32_t m = __ballot_sync(0xffffffffu, cand != kNone);
          const int wmin = m ? __shfl_sync(0xffffffffu, cand, __ffs(m) - 1) : kNone;
          if (lane == 0) s_min[par][warp] = wmin;
          __syncthreads();
          int best = s_min[par][0];
#pragma unroll
          for (int w = 1; w < kThreads / 32; ++w) best = min(best, s_min[par][w]);
          par ^= 1;
          if (best == kNone) break;
          const int i = best >> 1;
          const float c = (best & 1) ? -2.0f : 2.0f;  // 2 s_i after the flip
          // the owner flips its bit (i lies in group g); everyone adds c J_ij to its fields
          if (((i >> 2) & (kThreads - 1)) == t) sb ^= 1u << (4 * g + (i & 3));
          const float4 *J4 = reinterpret_cast<const float4 *>(A.J + (size_t)i * n);
          float4 jv[NS];
#pragma unroll
          for (int k = 0; k < NS; ++k)
            if (!GUARD || 4 * (t + kThreads * k) < n) jv[k] = __ldg(J4 + t + kThreads * k);
#pragma unroll
          for (int k = 0; k < NS; ++k)
            if (!GUARD || 4 * (t + kThreads * k) < n) {
              f[k].x = __fmaf_rn(c, jv[k].x, f[k].x);
              f[k].y = __fmaf_rn(c, jv[k].y, f[k].y);
              f[k].z = __fmaf_rn(c, jv[k].z, f[k].z);
              f[k].w = __fmaf_rn(c, jv[k].w, f[k].w);
            }
          ++nfl;
          from = i + 1;
        }
      }
      st_d += 1;
      st_total += 1;
      c_sweeps += 1;
      c_flips += (unsigned long long)nfl;
      if (nfl == 0 || st_d >= A.max_sweeps || (A.budget > 0 && st_total >= A.budget)) {
        st_conv = nfl == 0 ? 1 : 0;
        break;
      }
    }
    // E = -1/2 sum_i s_i (f_i + h_i): per-thread sums, then warps, then the CTA
    // in a fixed order; spins written back
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const int j = 4 * (t + kThreads * k);
      if (!GUARD || j < n) {
        const float4 hv = *reinterpret_cast<const float4 *>(A.h + j);
        const float fv[4] = {f[k].x, f[k].y, f[k].z, f[k].w}, hh[4] = {hv.x, hv.y, hv.z, hv.w};
        uint32_t w[2] = {0u, 0u};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const bool up = (sb >> (4 * k + e)) & 1u;
          const double v = (double)fv[e] + (double)hh[e];
          acc += up ? v : -v;
          w[e >> 1] |= (uint32_t)(up ? 0x3F80u : 0xBF80u) << (16 * (e & 1));  // BF16 +1 / -1
        }
        *reinterpret_cast<uint2 *>(row + j) = make_uint2(w[0], w[1]);
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) s_e[warp] = acc;
    __syncthreads();
    if (t == 0) {
      double e = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) e += s_e[w];
      DenseRep &g = A.rep[r];
      g.active = 0;
      g.conv = st_conv;
      g.d = st_d;
      g.total = st_total;
      g.E = -0.5 * e;
    }
  }
  if (t == 0 && c_sweeps) {
    atomicAdd(A.stats + 0, (unsigned long long)c_sweeps * (unsigned long long)A.n_eval);
    atomicAdd(A.stats + 1, c_flips);
    atomicAdd(A.stats + 4, (unsigned long long)c_sweeps);
  }
}

template <int NS, bool GUARD, int TH>
cudaError_t launch_push(const PushArgs &A, int sm_count, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense_push_kernel<NS, GUARD, TH>, TH, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::max(1, std::min(sm_count * per_sm, A.R));
  dense_push_kernel<NS, GUARD, TH><<<grid, TH, 0, s>>>(A);
  return cudaGetLastError();
}

template <int NS, int TH>
cudaError_t launch_push_ns(const PushArgs &A, int sm_count, cudaStream_t s) {
  return A.n == 4 * TH * NS ? launch_push<NS, false, TH>(A, sm_count, s) : launch_push<NS, true, TH>(A, sm_count, s);
}

}  // namespace

cudaError_t dense_push_run(int n, int n_eval, int R, int max_sweeps, int budget, const float *J, const float *h,
                           const float *F, __nv_bfloat16 *S, DenseRep *rep, int32_t *counter,
                           unsigned long long *stats, int sm_count, cudaStream_t s) {
  // whole float4 groups, 16-byte aligned rows, fields in registers: n % 4 == 0, n <= 16384
  if (n % 4 != 0 || n < 4 || n > 4 * 512 * kSlots) return cudaErrorInvalidValue;
  PushArgs A;
  A.n = n;
  A.n_eval = n_eval;
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
  if (n > 4 * 256 * kSlots) {  // 8192 < n <= 16384: 512 threads, 5 to 8 slots
    switch ((n + 4 * 512 - 1) / (4 * 512)) {
      case 5: return launch_push_ns<5, 512>(A, sm_count, s);
      case 6: return launch_push_ns<6, 512>(A, sm_count, s);
      case 7: return launch_push_ns<7, 512>(A, sm_count, s);
      default: return launch_push_ns<8, 512>(A, sm_count, s);
    }
  }
  if (n > 4 * 128 * kSlots) {  // 4096 < n <= 8192: 256 threads, 5 to 8 slots
    switch ((n + 4 * 256 - 1) / (4 * 256)) {
      case 5: return launch_push_ns<5, 256>(A, sm_count, s);
      case 6: return launch_push_ns<6, 256>(A, sm_count, s);
      case 7: return launch_push_ns<7, 256>(A, sm_count, s);
      default: return launch_push_ns<8, 256>(A, sm_count, s);
    }
  }
  switch ((n + 4 * 128 - 1) / (4 * 128)) {
    case 1: return launch_push_ns<1, 128>(A, sm_count, s);
    case 2: return launch_push_ns<2, 128>(A, sm_count, s);
    case 3: return launch_push_ns<3, 128>(A, sm_count, s);
    case 4: return launch_push_ns<4, 128>(A, sm_count, s);
    case 5: return launch_push_ns<5, 128>(A, sm_count, s);
    case 6: return launch_push_ns<6, 128>(A, sm_count, s);
    case 7: return launch_push_ns<7, 128>(A, sm_count, s);
    default: return launch_push_ns<8, 128>(A, sm_count, s);
  }
}

}  // namespace isg
