// dense_energy.cu — energies of the states a dense-instance search returns,
// on 5th-generation tensor cores (tcgen05, TMA, tensor memory), exactly up to
// a stated quantisation of the couplings.
//
// Eq. 1, each pair once:  E_r = - sum_{i<j} J_ij s_ri s_rj - sum_i h_i s_ri.
//
// Error-free splitting (the scheme of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", 2012, specialised to +/-1 operands): with 2^-F the largest
// power of two such that max |J| * 2^F < 2^31, Q_ij = RN(J_ij 2^F) is a 32-bit
// integer (|J_ij - Q_ij 2^-F| <= 2^(-F-1) <= max|J| 2^-31) and is written in
// balanced base 256:  Q = P0 + 256 P1 + 256^2 P2 + 256^3 P3,  P_d in [-128, 128],
// each plane exact in BF16.  Against spins +/-1 every product of a plane GEMM
// is an integer of magnitude <= 128 and every partial sum over K <= 16384 terms
// stays below 2^21 (FP32 holds every integer below 2^24), so the tensor cores'
// FP32 accumulation never rounds: each
// plane's result G_d = P_d . s is exact, whatever the accumulator's rounding
// mode.  The energy is then assembled in integers:
//     E_r = - 2^-F sum_{i<j} Q_ij s_ri s_rj - sum_i h_i s_ri,
// and differs from Eq. 1 by at most (number of pairs) * max|J| * 2^-31.
//
// Each pair once: for a tile of 128 spins I (rows i of J) only columns j > i
// take part - the diagonal block I x I through band copies of the planes with
// the entries j <= i set to zero, the columns to the right of I through the
// planes themselves.  One CTA per (spin tile, replica tile), tiles with the
// most columns first; thread 0 keeps a 2-stage TMA -> MMA pipeline full, a
// stage holding one spin tile [128 x 64] and the four planes' row tiles
// [128 x 64] of the same columns (128-byte swizzled K-major), so that a spin
// tile is loaded once for all four planes; one FP32 accumulator of 128 columns
// per plane in tensor memory; warps 0-3
// then read the four accumulators (warp w: tensor-memory lanes 32w .. 32w+31,
// one replica per thread) and form the tile's integer dot products with the
// replica's spins.  Every wait is bounded; a CTA whose wait gives up records
// ISING_ERR_TIMEOUT, waits (bounded) for its copies and MMAs in flight, frees
// its tensor memory and leaves.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "dense.cuh"
#include "device_common.cuh"
#include "tc.cuh"

namespace isg {

namespace {

constexpr int kEM = 128;                    // replicas per tile (MMA M)
constexpr int kEN = 128;                    // spins per tile (MMA N)
constexpr int kEK = 64;                     // K per chunk (128 bytes of BF16)
constexpr int kESt = 2;                     // pipeline stages
constexpr int kEPl = 4;                     // digit planes
constexpr int kEThreads = 128;              // 4 warps: one thread feeds the pipeline, all read the result
constexpr int kEA = kEM * kEK * 2;          // 16 KB spin tile
constexpr int kEB = kEN * kEK * 2;          // 16 KB plane tile
constexpr int kEStage = kEA + kEPl * kEB;   // 80 KB: a spin tile and the four planes' tiles
constexpr int kESmem = kESt * kEStage + 1024;  // + alignment slack

struct EnArgs {
  int32_t np, Rp;             // padded spins (multiple of 128), padded replicas (multiple of 128)
  const __nv_bfloat16 *S;     // [Rp][np] spins +/-1, 0 in the padding
  const float *h;             // [np] fields, 0 in the padding
  long long *pint;            // [np / 128][Rp] tile partials sum_{i in I, j > i} Q_ij s_i s_j
  double *ph;                 // [np / 128][Rp] tile partials sum_{i in I} h_i s_i
  int32_t *error;             // ISING_ERR_TIMEOUT when a wait gives up
};

__global__ void __launch_bounds__(kEThreads, 1)
    dense_energy_tc(const __grid_constant__ CUtensorMap mapS, const __grid_constant__ CUtensorMap mapP0,
                    const __grid_constant__ CUtensorMap mapP1, const __grid_constant__ CUtensorMap mapP2,
                    const __grid_constant__ CUtensorMap mapP3, const __grid_constant__ CUtensorMap mapU0,
                    const __grid_constant__ CUtensorMap mapU1, const __grid_constant__ CUtensorMap mapU2,
                    const __grid_constant__ CUtensorMap mapU3, EnArgs A) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kESt], empty_bar[kESt], done_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int32_t s_fail;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tm_count = A.Rp / kEM;
  const int tn = blockIdx.x / tm_count, tm = blockIdx.x % tm_count;  // spin tile 0 has the most columns
  const int r0 = tm * kEM, i0 = tn * kEN;
  constexpr int kd = kEN / kEK;                      // band chunks (the diagonal block), per plane
  const int nchunks = kd + (A.np - i0 - kEN) / kEK;  // column chunks (each for all four planes)

  if (tid == 0) {
    for (int s = 0; s < kESt; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&empty_bar[s], 1);
    }
    tc::mbar_init(&done_bar, 1);
    tc::fence_barrier_init();
    tc::prefetch_tmap(&mapS);
    s_fail = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base_s, 512);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_base_s;  // plane d: columns 128 d .. 128 d + 127

  if (tid == 0) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kEM, kEN);
    uint32_t ph_full[kESt], ph_empty[kESt];
    for (int s = 0; s < kESt; ++s) ph_full[s] = ph_empty[s] = 0u;
    int issued = 0, consumed = 0;
    bool ok = true;
    const CUtensorMap *mu[kEPl] = {&mapU0, &mapU1, &mapU2, &mapU3};
    const CUtensorMap *mp[kEPl] = {&mapP0, &mapP1, &mapP2, &mapP3};
    auto load = [&](int q) {
      const int s = q % kESt;
      uint8_t *st = smem + s * kEStage;
      tc::mbar_arrive_expect_tx(&full_bar[s], kEStage);
      if (q < kd) {
        // band chunk: columns i0 + 64 q .. of the diagonal block, band-local
        tc::tma_load_2d(st, &mapS, &full_bar[s], i0 + q * kEK, r0);
#pragma unroll
        for (int d = 0; d < kEPl; ++d) tc::tma_load_2d(st + kEA + d * kEB, mu[d], &full_bar[s], q * kEK, i0);
      } else {
        const int col = i0 + kEN + (q - kd) * kEK;
        tc::tma_load_2d(st, &mapS, &full_bar[s], col, r0);
#pragma unroll
        for (int d = 0; d < kEPl; ++d) tc::tma_load_2d(st + kEA + d * kEB, mp[d], &full_bar[s], col, i0);
      }
    };
    for (; issued < kESt && issued < nchunks; ++issued) load(issued);
    for (int c = 0; c < nchunks && ok; ++c) {
      const int s = c % kESt;
      if (!tc::mbar_wait(&full_bar[s], ph_full[s])) {
        ok = false;
        break;
      }
      ph_full[s] ^= 1u;
      tc::tc_fence_after();
      uint8_t *st = smem + s * kEStage;
      const uint64_t da = tc::smem_desc_k_sw128(st);
#pragma unroll
      for (int d = 0; d < kEPl; ++d) {
        const uint64_t db = tc::smem_desc_k_sw128(st + kEA + d * kEB);
        const uint32_t dst = tmem + (uint32_t)(d * kEN);
#pragma unroll
        for (int kk = 0; kk < kEK / 16; ++kk)
          tc::mma_bf16(dst, da + 2 * kk, db + 2 * kk, idesc, (c > 0 || kk > 0) ? 1u : 0u);
      }
      tc::mma_commit(&empty_bar[s]);
      consumed = c + 1;
      // refill the stage of the previous chunk once its MMAs have read it
      if (c >= 1 && issued < nchunks) {
        const int sp = (c - 1) % kESt;
        if (!tc::mbar_wait(&empty_bar[sp], ph_empty[sp])) {
          ok = false;
          break;
        }
        ph_empty[sp] ^= 1u;
        load(issued++);
      }
    }
    // completion of every MMA issued (also after a failure, so that tensor
    // memory is not freed under a running MMA)
    tc::mma_commit(&done_bar);
    if (!ok) {
      // loads issued but never consumed must land before the CTA leaves
      for (int c = consumed; c < issued; ++c) {
        const int s = c % kESt;
        if (tc::mbar_wait(&full_bar[s], ph_full[s])) ph_full[s] ^= 1u;
      }
      atomicExch(&s_fail, 1);
      atomicExch(A.error, (int32_t)ISING_ERR_TIMEOUT);
    }
  }
  __syncthreads();  // the other threads wait here, not in a poll, while thread 0 feeds the pipeline
  const bool done = tc::mbar_wait(&done_bar, 0);
  tc::tc_fence_after();
  const bool failed = __syncthreads_or(!done || s_fail != 0) != 0;
  if (!failed) {
    const int r = r0 + 32 * warp + lane;
    // the tile's 128 spins of replica r as bits (1 = +1, 0 = -1 or padding) and
    // the field part of the energy in FP64
    const __nv_bfloat16 *srow = A.S + (size_t)r * A.np + i0;
    uint32_t up[kEN / 32];
    double eh = 0.0;
#pragma unroll
    for (int w = 0; w < kEN / 32; ++w) {
      uint32_t bits = 0u;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 sv = *reinterpret_cast<const uint4 *>(srow + 32 * w + 8 * q);
        const uint32_t sw[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float sval = __bfloat162float(__ushort_as_bfloat16((uint16_t)(sw[k >> 1] >> (16 * (k & 1)))));
          const int i = 32 * w + 8 * q + k;
          if (sval > 0.0f) bits |= 1u << (8 * q + k);
          eh += (double)(sval * __ldg(A.h + i0 + i));
        }
      }
      up[w] = bits;
    }
    // sum_i s_i G_d,i for each plane, exact integers (|G| < 2^21, 128 columns)
    long long tot = 0;
#pragma unroll 1
    for (int d = 0; d < kEPl; ++d) {
      long long acc = 0;
#pragma unroll
      for (int w = 0; w < kEN / 32; ++w) {
        uint32_t v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(d * kEN + 32 * w), v);
        int part = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int g = __float2int_rn(__uint_as_float(v[k]));
          part += ((up[w] >> k) & 1u) ? g : -g;
        }
        acc += part;
      }
      tot += acc * (1ll << (8 * d));
    }
    // (padded spins and padded replicas have zero rows in S and J, so their
    // accumulator entries are 0 and contribute nothing)
    A.pint[(size_t)tn * A.Rp + r] = tot;
    A.ph[(size_t)tn * A.Rp + r] = eh;
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// E[r] = - 2^-F sum over tiles of the integer partials - sum of the field
// partials, in tile order.
__global__ void dense_energy_finish(int32_t ntn, int32_t R, int32_t Rp, int32_t F, const long long *pint,
                                    const double *ph, double *E) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  long long qi = 0;
  double hs = 0.0;
  for (int t = 0; t < ntn; ++t) {
    qi += pint[(size_t)t * Rp + r];
    hs += ph[(size_t)t * Rp + r];
  }
  E[r] = -ldexp((double)qi, -F) - hs;
}

// Returned spins (int8 [R][n]) as BF16 +/-1 rows [Rp][np], zeros in the padding.
__global__ void dense_energy_spins(const int8_t *spins, int32_t n, int32_t np, int32_t R, int64_t total,
                                   __nv_bfloat16 *S) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / np;
    const int i = (int)(t % np);
    const float v = (r < R && i < n) ? (float)spins[r * n + i] : 0.0f;
    S[t] = __float2bfloat16_rn(v);
  }
}

__global__ void dense_absmax(const float *J, int64_t nn, unsigned int *out) {
  float m = 0.0f;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(J[t]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as integers
}

// Balanced base-256 digit d of q: q = sum_d P_d 256^d with P_d in [-128, 128).
__device__ __forceinline__ int digit(long long q, int d) {
  for (int k = 0; k < d; ++k) {
    const long long p = ((q + 128) & 255) - 128;
    q = (q - p) / 256;
  }
  return d == kEPl - 1 ? (int)q : (int)(((q + 128) & 255) - 128);
}

// Digit planes P_d [np][np] and band copies U_d [np][128] (row i, column c:
// entry (i, 128 (i / 128) + c) when that column lies right of i, else 0).
__global__ void dense_planes(const float *J, int32_t np, int32_t F, __nv_bfloat16 *P, __nv_bfloat16 *U) {
  const int64_t nn = (int64_t)np * np;
  const double scale = ldexp(1.0, F);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / np), j = (int)(t % np);
    const long long q = __double2ll_rn((double)J[t] * scale);  // exact scaling by a power of two, one rounding
    const int band0 = (i / kEN) * kEN;
    const bool in_band = j >= band0 && j < band0 + kEN;
#pragma unroll
    for (int d = 0; d < kEPl; ++d) {
      const __nv_bfloat16 v = __float2bfloat16_rn((float)digit(q, d));
      P[(int64_t)d * nn + t] = v;
      if (in_band) U[(int64_t)d * np * kEN + (int64_t)i * kEN + (j - band0)] = j > i ? v : __float2bfloat16_rn(0.0f);
    }
  }
}

}  // namespace

// Builds the digit planes of J [np][np] (np a multiple of 128) into P
// ([4][np][np] BF16) and U ([4][np][128] BF16) and returns the scale exponent
// F in *F_out (2^-F is the unit of the planes).  Waits for the device.
cudaError_t dense_planes_build(const float *J, int np, __nv_bfloat16 *P, __nv_bfloat16 *U, int *F_out, int sm_count,
                               cudaStream_t s) {
  unsigned int *d_max = nullptr, h_max = 0;
  cudaError_t e;
  if ((e = cudaMalloc(&d_max, sizeof(unsigned int))) != cudaSuccess) return e;
  e = cudaMemsetAsync(d_max, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) {
    dense_absmax<<<sm_count * 8, 256, 0, s>>>(J, (int64_t)np * np, d_max);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_max, d_max, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_max);
  if (e != cudaSuccess) return e;
  float amax;
  std::memcpy(&amax, &h_max, sizeof(float));
  // largest F with amax * 2^F < 2^31 (F = 0 for an all-zero J)
  int F = 0;
  if (amax > 0.0f) {
    int ex = 0;
    std::frexp((double)amax, &ex);  // amax in [2^(ex-1), 2^ex)
    F = 31 - ex;
  }
  dense_planes<<<sm_count * 8, 256, 0, s>>>(J, np, F, P, U);
  *F_out = F;
  return cudaGetLastError();
}

cudaError_t dense_energy_run(const int8_t *spins, int n, int np, int R, const float *h, const __nv_bfloat16 *P,
                             const __nv_bfloat16 *U, int F, __nv_bfloat16 *S, long long *pint, double *ph,
                             double *E, int32_t *error, int sm_count, int *launches, cudaStream_t s) {
  if (np % kEN != 0 || n > np || R < 1) return cudaErrorInvalidValue;
  const int Rp = (R + kEM - 1) / kEM * kEM;
  const int64_t total = (int64_t)Rp * np;
  dense_energy_spins<<<(int)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count * 16), 256, 0, s>>>(
      spins, n, np, R, total, S);
  cudaError_t e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  CUtensorMap mS, mP[kEPl], mU[kEPl];
  const int64_t nn = (int64_t)np * np;
  if ((e = tc_encode_2d(&mS, S, (uint64_t)np, (uint64_t)Rp, kEK, kEM)) != cudaSuccess) return e;
  for (int d = 0; d < kEPl; ++d) {
    if ((e = tc_encode_2d(&mP[d], P + d * nn, (uint64_t)np, (uint64_t)np, kEK, kEN)) != cudaSuccess) return e;
    if ((e = tc_encode_2d(&mU[d], U + (int64_t)d * np * kEN, (uint64_t)kEN, (uint64_t)np, kEK, kEN)) != cudaSuccess)
      return e;
  }
  if ((e = cudaFuncSetAttribute(dense_energy_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kESmem)) !=
      cudaSuccess)
    return e;
  EnArgs A;
  A.np = np;
  A.Rp = Rp;
  A.S = S;
  A.h = h;
  A.pint = pint;
  A.ph = ph;
  A.error = error;
  const int ntn = np / kEN;
  dense_energy_tc<<<ntn * (Rp / kEM), kEThreads, kESmem, s>>>(mS, mP[0], mP[1], mP[2], mP[3], mU[0], mU[1], mU[2],
                                                             mU[3], A);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  dense_energy_finish<<<(R + 255) / 256, 256, 0, s>>>(ntn, R, Rp, F, pint, ph, E);
  *launches += 3;
  return cudaGetLastError();
}

}  // namespace isg
