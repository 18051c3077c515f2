// dense.cu — fully connected instances (Sherrington-Kirkpatrick): the
// sequential schedule with fields computed on tensor cores.  Where the
// hand-written kernels apply (n zero-padded to a multiple of 256, at most 16384) a round of the
// search is: the first sweeps of every replica's descent in lockstep on tcgen05
// (dense_tc.cu), each replica's remaining sweeps as incremental gain updates
// (dense_push.cu), then the round's bookkeeping (best state, next restart).
// The block search below, with its GEMMs in cuBLAS, is the comparator and the
// path for other sizes.
//
// For a complete graph every colour class is one spin, so descent is the
// paper's one-move-at-a-time order (Sec. IV).  Spins are visited in blocks of
// B consecutive indices.  Before a block is decided, the fields of its B spins
// for every replica are recomputed from the current configuration as a GEMM,
//     F[b0:b0+B, :] = J[b0:b0+B, :] . S        (S = +/-1 spins, [n][R])
// with J split into two BF16 matrices J = J_hi + J_lo + O(2^-16 |J|) and S
// exact in BF16, accumulated in FP32 (two GEMMs into one FP32 result).  Inside
// the block the spins are then decided one after another, each field corrected
// in FP32 for the block's own earlier flips (+2 J_ij s_j per flipped j), the
// incremental gain update of the paper restricted to the block.  During the
// search, energies (which decide the best state kept) are -1/2 sum_i s_i f_i in
// FP64 over those fields; they carry the BF16-split and FP32 accumulation
// error, so decisions within about 1e-4 of zero may differ from an FP64
// computation.  The returned energies are recomputed from the returned spins
// with the FP32 couplings (FP32 GEMM, FP64 sums), within ~1e-8 relative.
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <cfloat>
#include <cstdlib>
#include <cstring>

#include "dense.cuh"
#include "device_common.cuh"

namespace isg {

bool dense_tc_eligible(int n);
int dense_tc_padded(int n);
cudaError_t dense_tc_run(int n, int n_eval, int R, int Rp, int b, uint64_t seed, const float *J, const float *h,
                         const __nv_bfloat16 *Jhi, const __nv_bfloat16 *Jlo, __nv_bfloat16 *S, float *Fx,
                         DenseRep *rep, int sweeps_a, unsigned long long *stats, int32_t *error,
                         const ising_search_params *p, cudaStream_t s);

namespace {

constexpr int kDB = 128;          // spins per block
constexpr int kTcSweepsA = 3;     // tensor-core sweeps per round before the per-replica continuation

// Zero-padded copies for the tensor-core path: J [n][n] -> Jp [np][np] FP32 and
// its BF16 split, h [n] -> hp [np].
__global__ void dense_pad_split(const float *J, const float *h, int32_t n, int32_t np, float *Jp, float *hp,
                                __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
  const int64_t nn = (int64_t)np * np;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / np), j = (int)(t % np);
    const float w = (i < n && j < n) ? J[(int64_t)i * n + j] : 0.0f;
    if (Jp) Jp[t] = w;
    const __nv_bfloat16 a = __float2bfloat16_rn(w);
    hi[t] = a;
    lo[t] = __float2bfloat16_rn(w - __bfloat162float(a));
    if (hp && t < np) hp[t] = t < n ? h[t] : 0.0f;
  }
}

__global__ void dense_split(const float *J, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t nn) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
    const float w = J[t];
    const __nv_bfloat16 a = __float2bfloat16_rn(w);
    hi[t] = a;
    lo[t] = __float2bfloat16_rn(w - __bfloat162float(a));
  }
}

__global__ void dense_start(int32_t n, int32_t R, int32_t Rp, uint64_t seed, int32_t b, const DenseRep *rep,
                            __nv_bfloat16 *S) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int w = blockIdx.y;
  if (r >= R || !rep[r].active || rep[r].d != 0) return;
  const uint4 x = start_bits(seed, (uint32_t)w, (uint32_t)r, (uint32_t)rep[r].k, (uint32_t)b);
  for (int t = 0; t < 128; ++t) {
    const int i = w * 128 + t;
    if (i >= n) break;
    const uint32_t bit = (word_of(x, t / 32) >> (t % 32)) & 1u;
    S[(int64_t)i * Rp + r] = __float2bfloat16_rn(bit ? 1.0f : -1.0f);
  }
}

// In-block sequential decisions, one thread per replica.
__global__ void __launch_bounds__(256) dense_decide(int32_t n, int32_t R, int32_t Rp, int32_t b0, int32_t bsz,
                                                    const float *__restrict__ J, const float *__restrict__ hf,
                                                    const float *__restrict__ F, __nv_bfloat16 *S, DenseRep *rep) {
  extern __shared__ float sJ[];  // [kDB][kDB] block of J
  for (int t = threadIdx.x; t < bsz * bsz; t += blockDim.x) {
    const int a = t / bsz, c = t % bsz;
    sJ[a * kDB + c] = J[(int64_t)(b0 + a) * n + b0 + c];
  }
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R || !rep[r].active) return;
  uint32_t flipped[kDB / 32], up[kDB / 32];
#pragma unroll
  for (int q = 0; q < kDB / 32; ++q) flipped[q] = up[q] = 0;
  int nflip = 0;
  for (int i = 0; i < bsz; ++i) {
    float f = F[(int64_t)i * Rp + r] + hf[b0 + i];
    const bool s_up = __bfloat162float(S[(int64_t)(b0 + i) * Rp + r]) > 0.0f;
#pragma unroll
    for (int q = 0; q < kDB / 32; ++q) {
      uint32_t m = flipped[q];
      if (q * 32 >= i) m = 0;
      else if (i - q * 32 < 32) m &= (1u << (i - q * 32)) - 1u;
      while (m) {
        const int j = q * 32 + __ffs(m) - 1;
        m &= m - 1;
        const float w2 = 2.0f * sJ[i * kDB + j];
        f = __fadd_rn(f, ((up[q] >> (j - q * 32)) & 1u) ? w2 : -w2);
      }
    }
    const bool flip = s_up ? (f < 0.0f) : (f > 0.0f);
    const bool now_up = flip ? !s_up : s_up;
    if (now_up) up[i / 32] |= 1u << (i % 32);
    if (flip) {
      flipped[i / 32] |= 1u << (i % 32);
      S[(int64_t)(b0 + i) * Rp + r] = __float2bfloat16_rn(now_up ? 1.0f : -1.0f);
      ++nflip;
    }
  }
  rep[r].flips += nflip;
}

__global__ void dense_end(int32_t R, int32_t n, int32_t max_sweeps, int32_t budget, DenseRep *rep, int32_t *active_count,
                          unsigned long long *stats) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  DenseRep &p = rep[r];
  if (!p.active) return;
  p.total += 1;
  p.d += 1;
  atomicAdd(stats + 0, (unsigned long long)n);
  atomicAdd(stats + 1, (unsigned long long)p.flips);
  atomicAdd(stats + 4, 1ull);
  const bool conv = p.flips == 0;
  p.flips = 0;
  if (conv || p.d >= max_sweeps || (budget > 0 && p.total >= budget)) {
    p.active = 0;
    p.conv = conv ? 1 : 0;
    if (conv) atomicAdd(stats + 2, 1ull);
  } else {
    atomicAdd(active_count, 1);
  }
}

// E_r = -1/2 sum_i s_ir (F_ir + 2 h_i) in FP64 (F without h); then best-state
// bookkeeping for the round.
__global__ void dense_energy(int32_t n, int32_t R, int32_t Rp, const __nv_bfloat16 *S, const float *Ff,
                             const float *hf, DenseRep *rep, int8_t *best, int32_t final_pass) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double acc = 0.0;
  for (int i = 0; i < n; ++i)
    acc += (double)__bfloat162float(S[(int64_t)i * Rp + r]) *
           ((double)Ff[(int64_t)i * Rp + r] + 2.0 * (double)hf[i]);
  const double E = -0.5 * acc;
  DenseRep &p = rep[r];
  p.E = E;
  if (final_pass) return;
  if (p.conv) {
    p.minima += 1;
    if (E < p.best) {
      p.best = E;
      for (int i = 0; i < n; ++i) best[(int64_t)r * n + i] = __bfloat162float(S[(int64_t)i * Rp + r]) > 0.0f ? 1 : -1;
    }
  }
}

__global__ void dense_next_round(int32_t R, int32_t restarts, int32_t budget, DenseRep *rep, int32_t *active_count,
                                 unsigned long long *stats) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  DenseRep &p = rep[r];
  p.conv = 0;
  p.k += 1;
  if (p.k < restarts && (budget <= 0 || p.total < budget)) {
    p.active = 1;
    p.d = 0;
    atomicAdd(active_count, 1);
    atomicAdd(stats + 3, 1ull);
  }
}

__global__ void dense_init(int32_t R, DenseRep *rep, unsigned long long *stats) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  DenseRep p;
  p.active = 1;
  p.conv = p.total = p.minima = p.d = p.k = p.flips = 0;
  p.round = 1;
  p.best = DBL_MAX;
  p.E = 0.0;
  rep[r] = p;
  atomicAdd(stats + 3, 1ull);
}

// Returned energies, recomputed from the returned spins with the FP32
// couplings: F = S J by an FP32 GEMM (library), then
// E_r = -1/2 sum_i s_i (F_ri + 2 h_i) in FP64, one warp per replica in a fixed order.  The search's own energies
// come from its BF16 hi+lo fields, whose error grows with n.
__global__ void dense_spins_f32(const int8_t *s, float *Sf, int64_t count) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    Sf[t] = (float)s[t];
}

__global__ void dense_energy_from_fields(const int8_t *s, const float *F, const float *hf, int32_t n, int32_t R,
                                         double *E) {
  const int r = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (r >= R) return;
  double acc = 0.0;  // sum_i s_i (F_i + 2 h_i), F without h: E = -1/2 acc
  for (int i = lane; i < n; i += 32)
    acc += (double)s[(int64_t)r * n + i] * ((double)F[(int64_t)r * n + i] + 2.0 * (double)hf[i]);
  acc = warp_sum(acc);
  if (lane == 0) E[r] = -0.5 * acc;
}

__global__ void dense_output(int32_t n, int32_t R, int32_t Rp, int32_t b, int64_t spin_off, const __nv_bfloat16 *S,
                             const int8_t *best, const DenseRep *rep, int8_t *out, double *E, int32_t *minima) {
  const int64_t tot = (int64_t)R * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / n), i = (int)(t % n);
    out[(int64_t)R * spin_off + t] =
        rep[r].minima > 0 ? best[t] : (__bfloat162float(S[(int64_t)i * Rp + r]) > 0.0f ? 1 : -1);
  }
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < R) {
    const DenseRep &p = rep[t];
    E[(int64_t)b * R + t] = p.minima > 0 ? p.best : p.E;
    if (minima) minima[(int64_t)b * R + t] = p.minima;
  }
}

// End of a round of the tensor-core path, one warp per replica (S replica-major,
// [Rp][n]): count a converged descent, keep its state if it is the best so far
// (strictly lower energy; ties keep the earlier), then start the next restart
// unless the restarts or the sweep budget are used up.
__global__ void dense_round_end(int32_t n, int32_t np, int32_t R, int32_t restarts, int32_t budget,
                                const __nv_bfloat16 *S, DenseRep *rep, int8_t *best, int32_t *active_count,
                                unsigned long long *stats) {
  const int r = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (r >= R) return;
  int copy = 0;
  if (lane == 0) {
    DenseRep p = rep[r];
    if (p.round) {
      p.round = 0;
      if (p.conv) {
        p.minima += 1;
        atomicAdd(stats + 2, 1ull);
        if (p.E < p.best) {
          p.best = p.E;
          copy = 1;
        }
      }
      p.conv = 0;
      p.k += 1;
      if (p.k < restarts && (budget <= 0 || p.total < budget)) {
        p.active = 1;
        p.d = 0;
        p.round = 1;
        atomicAdd(active_count, 1);
        atomicAdd(stats + 3, 1ull);
      }
      rep[r] = p;
    }
  }
  copy = __shfl_sync(0xffffffffu, copy, 0);
  if (copy)
    for (int i = lane; i < n; i += 32)
      best[(int64_t)r * n + i] = __bfloat162float(S[(int64_t)r * np + i]) > 0.0f ? 1 : -1;
}

// Results of the tensor-core path: the best converged state, else the final one
// (S rows of np spins, the first n the instance's).
__global__ void dense_tc_output(int32_t n, int32_t np, int32_t R, const __nv_bfloat16 *S, const int8_t *best,
                                const DenseRep *rep, int8_t *out, double *E, int32_t *minima) {
  const int64_t tot = (int64_t)R * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / n), i = (int)(t % n);
    out[t] = rep[r].minima > 0 ? best[t] : (__bfloat162float(S[(int64_t)r * np + i]) > 0.0f ? 1 : -1);
  }
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < R) {
    const DenseRep &p = rep[t];
    E[t] = p.minima > 0 ? p.best : p.E;
    if (minima) minima[t] = p.minima;
  }
}

struct DenseState : FamilyState {
  cublasHandle_t cublas = nullptr;
  void *workspace = nullptr;
  int32_t n = 0, Rp = 0;
  int32_t inst = -1;
  __nv_bfloat16 *hi = nullptr, *lo = nullptr, *S = nullptr;
  float *F = nullptr, *Ff = nullptr;
  DenseRep *rep = nullptr;
  int8_t *best = nullptr;
  int32_t *active = nullptr, *h_active = nullptr;
  __nv_bfloat16 *S_tc = nullptr;  // [Rp128][np] replica-major spins for the tcgen05 kernel
  // tensor-core path with n padded to np (a multiple of 256): own copies of J
  // (FP32 and BF16 split) and h when np != n, else the unpadded ones
  int32_t np = 0;
  float *Jp = nullptr, *hp = nullptr;
  __nv_bfloat16 *tc_hi = nullptr, *tc_lo = nullptr;
  int64_t fx_floats = 0;  // capacity of Sx and Fx
  int32_t *err = nullptr, *h_err = nullptr;
  int32_t *counter = nullptr;          // work counter of the per-replica continuation
  float *Sx = nullptr, *Fx = nullptr;  // [R][n] returned spins and their FP32 fields
  // returned energies on tensor cores: digit planes of J [4][np][np] and their
  // band copies [4][np][128], spins [Rp128][np], tile partials [np/128][Rp128]
  __nv_bfloat16 *planes = nullptr, *bands = nullptr, *Se = nullptr;
  long long *Epint = nullptr;
  double *Eph = nullptr;
  int32_t planes_F = 0;
};


void free_state(DenseState &D) {
  cudaFree(D.hi);
  cudaFree(D.lo);
  cudaFree(D.S);
  cudaFree(D.F);
  cudaFree(D.Ff);
  cudaFree(D.rep);
  cudaFree(D.best);
  cudaFree(D.active);
  cudaFree(D.workspace);
  cudaFree(D.S_tc);
  cudaFree(D.err);
  cudaFree(D.counter);
  cudaFree(D.Sx);
  cudaFree(D.Fx);
  cudaFree(D.planes);
  cudaFree(D.bands);
  cudaFree(D.Se);
  cudaFree(D.Epint);
  cudaFree(D.Eph);
  if (D.np != D.n) {  // the padded copies are owned only when padding was needed
    cudaFree(D.Jp);
    cudaFree(D.hp);
    cudaFree(D.tc_hi);
    cudaFree(D.tc_lo);
  }
  if (D.h_err) cudaFreeHost(D.h_err);
  if (D.h_active) cudaFreeHost(D.h_active);
  if (D.cublas) cublasDestroy(D.cublas);
  D = DenseState();
}

cublasStatus_t gemm(DenseState &D, int m, int nn, int k, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B,
                    int ldb, float *C, int ldc, float beta) {
  const float alpha = 1.0f;
  return cublasGemmEx(D.cublas, CUBLAS_OP_N, CUBLAS_OP_N, m, nn, k, &alpha, A, CUDA_R_16BF, lda, B, CUDA_R_16BF, ldb,
                      &beta, C, CUDA_R_32F, ldc, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
}

// F[:, rows] = (J_hi + J_lo)[rows, :] . S  for rows b0 .. b0+cnt
bool fields(DenseState &D, int b0, int cnt, float *out) {
  const int n = D.n;
  if (gemm(D, D.Rp, cnt, n, D.S, D.Rp, D.hi + (int64_t)b0 * n, n, out, D.Rp, 0.0f) != CUBLAS_STATUS_SUCCESS)
    return false;
  return gemm(D, D.Rp, cnt, n, D.S, D.Rp, D.lo + (int64_t)b0 * n, n, out, D.Rp, 1.0f) == CUBLAS_STATUS_SUCCESS;
}

// Sx and Fx hold at least `floats` floats each (freed with the state).
cudaError_t ensure_fx(DenseState &D, int64_t floats) {
  if (D.fx_floats >= floats) return cudaSuccess;
  cudaFree(D.Sx);
  cudaFree(D.Fx);
  D.Sx = D.Fx = nullptr;
  D.fx_floats = 0;
  cudaError_t e;
  if ((e = cudaMalloc(&D.Sx, (size_t)floats * sizeof(float))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&D.Fx, (size_t)floats * sizeof(float))) != cudaSuccess) return e;
  D.fx_floats = floats;
  return cudaSuccess;
}

cudaError_t exact_energies(DenseState &D, ising_handle *h, int n, int R, const float *J, const float *hf,
                           const int8_t *out, double *E, cudaStream_t s) {
  cudaError_t e;
  if ((e = ensure_fx(D, (int64_t)D.Rp * n)) != cudaSuccess) return e;
  const int64_t tot = (int64_t)R * n;
  dense_spins_f32<<<(int)std::min<int64_t>((tot + 255) / 256, (int64_t)h->sm_count * 16), 256, 0, s>>>(out, D.Sx, tot);
  // column-major view: F^T (n x R) = J (n x n, symmetric) . S^T (n x R), FP32
  // accurate through the library's BF16x9 emulation (each operand split
  // exactly into three BF16 terms); never TF32.  Used by the comparator only.
  const float one = 1.0f, zero = 0.0f;
  if (cublasSetStream(D.cublas, s) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  if (cublasSetEmulationStrategy(D.cublas, CUBLAS_EMULATION_STRATEGY_EAGER) != CUBLAS_STATUS_SUCCESS)
    return cudaErrorUnknown;
  if (cublasGemmEx(D.cublas, CUBLAS_OP_N, CUBLAS_OP_N, n, R, n, &one, J, CUDA_R_32F, n, D.Sx, CUDA_R_32F, n, &zero,
                   D.Fx, CUDA_R_32F, n, CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT) !=
      CUBLAS_STATUS_SUCCESS)
    return cudaErrorUnknown;
  dense_energy_from_fields<<<(R * 32 + 255) / 256, 256, 0, s>>>(out, D.Fx, hf, n, R, E);
  h->launches += 2;
  return cudaGetLastError();
}

}  // namespace

bool dense_supported(const ising_handle *h, int32_t R) {
  return h->dense && h->d_Jdense && R >= 1 && (int64_t)h->nmax * h->nmax <= (int64_t)1 << 28;
}

void dense_free(ising_handle *h) {
  if (!h->dense_st) return;
  free_state(static_cast<DenseState &>(*h->dense_st));
  h->dense_st.reset();
}

cudaError_t launch_dense(ising_handle *h, const ising_search_params *p, int32_t R, int8_t *spins, double *E,
                         int32_t *E32, int32_t *minima, const uint64_t *seeds_host, cudaStream_t s) {
  (void)E32;
  DenseState &D = family_state<DenseState>(h->dense_st);
  cudaError_t e;
  const int Rp = (R + 7) / 8 * 8;
  int64_t joff = 0;
  for (int32_t b = 0; b < h->n_inst; ++b) {
    const int n = h->inst[b].n;
    if (D.n != n || D.Rp != Rp || D.inst != b) {
      free_state(D);
      if ((e = cudaFuncSetAttribute(dense_decide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(kDB * kDB * sizeof(float)))) != cudaSuccess)
        return e;
      D.n = n;
      D.Rp = Rp;
      D.inst = b;
      if ((e = cudaMalloc(&D.hi, (size_t)n * n * 2)) != cudaSuccess) return e;
      if ((e = cudaMalloc(&D.lo, (size_t)n * n * 2)) != cudaSuccess) return e;
      if ((e = cudaMalloc(&D.S, (size_t)n * Rp * 2)) != cudaSuccess) return e;
      if ((e = cudaMalloc(&D.F, (size_t)kDB * Rp * 4)) != cudaSuccess) return e;
      if ((e = cudaMalloc(&D.Ff, (size_t)n * Rp * 4)) != cudaSuccess) return e;
      if ((e = cudaMalloc(&D.rep, (size_t)R * sizeof(DenseRep))) != cudaSuccess) return e;
      if ((e = cudaMalloc(&D.best, (size_t)R * n)) != cudaSuccess) return e;
      if ((e = cudaMalloc(&D.active, 64)) != cudaSuccess) return e;
      if ((e = cudaMallocHost(&D.h_active, 64)) != cudaSuccess) return e;
      if ((e = cudaMemset(D.S, 0, (size_t)n * Rp * 2)) != cudaSuccess) return e;
      dense_split<<<h->sm_count * 8, 256, 0, s>>>(h->d_Jdense + joff, D.hi, D.lo, (int64_t)n * n);
    }
    const float *J = h->d_Jdense + joff;
    const uint64_t seed = seeds_host[b];

    const float *hf = reinterpret_cast<const float *>(h->d_h) + h->inst[b].spin_off;
    if (dense_tc_eligible(n) && p->dense_variant != ISING_DENSE_LIBRARY) {
      // Rounds of: the first sweeps of every replica's descent on tensor cores
      // (hand-written tcgen05 kernel), then each replica on its own until its
      // descent ends (incremental updates, CUDA cores), then the round's
      // bookkeeping.  The host reads one count per round.
      const int Rp128 = (R + 127) / 128 * 128;
      const int np = dense_tc_padded(n);
      if (!D.S_tc) {
        D.np = np;
        if (np == n) {
          D.Jp = const_cast<float *>(J);
          D.hp = const_cast<float *>(hf);
          D.tc_hi = D.hi;
          D.tc_lo = D.lo;
        } else {
          if ((e = cudaMalloc(&D.Jp, (size_t)np * np * 4)) != cudaSuccess) return e;
          if ((e = cudaMalloc(&D.hp, (size_t)np * 4)) != cudaSuccess) return e;
          if ((e = cudaMalloc(&D.tc_hi, (size_t)np * np * 2)) != cudaSuccess) return e;
          if ((e = cudaMalloc(&D.tc_lo, (size_t)np * np * 2)) != cudaSuccess) return e;
          dense_pad_split<<<h->sm_count * 8, 256, 0, s>>>(J, hf, n, np, D.Jp, D.hp, D.tc_hi, D.tc_lo);
          h->launches += 1;
        }
        if ((e = cudaMalloc(&D.S_tc, (size_t)Rp128 * np * 2)) != cudaSuccess) return e;
        if ((e = cudaMemset(D.S_tc, 0, (size_t)Rp128 * np * 2)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&D.planes, (size_t)4 * np * np * 2)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&D.bands, (size_t)4 * np * 128 * 2)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&D.Se, (size_t)Rp128 * np * 2)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&D.Epint, (size_t)(np / 128) * Rp128 * sizeof(long long))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&D.Eph, (size_t)(np / 128) * Rp128 * sizeof(double))) != cudaSuccess) return e;
        int F = 0;
        if ((e = dense_planes_build(D.Jp, np, D.planes, D.bands, &F, h->sm_count, s)) != cudaSuccess) return e;
        D.planes_F = F;
        h->launches += 2;
        if ((e = cudaMalloc(&D.err, 64)) != cudaSuccess) return e;
        if ((e = cudaMallocHost(&D.h_err, 64)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&D.counter, 64)) != cudaSuccess) return e;
      }
      // [R][np] FP32: exported fields here, returned-energy GEMM operands afterwards
      if ((e = ensure_fx(D, (int64_t)std::max(D.Rp, R) * np)) != cudaSuccess) return e;
      const int sweeps_a = p->dense_tensor_sweeps == 0 ? kTcSweepsA : std::max(0, p->dense_tensor_sweeps);
      if ((e = cudaMemsetAsync(D.err, 0, 4, s)) != cudaSuccess) return e;
      const int rb = (R + 255) / 256, wb = (R * 32 + 255) / 256;
      dense_init<<<rb, 256, 0, s>>>(R, D.rep, h->d_stats);
      h->launches += 1;
      for (;;) {
        kt_begin(h, "dense_tc_kernel", s);
        e = dense_tc_run(np, n, R, Rp128, b, seed, D.Jp, D.hp, D.tc_hi, D.tc_lo, D.S_tc, D.Fx, D.rep, sweeps_a,
                         h->d_stats, D.err, p, s);
        kt_end(h, s);
        if (e != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(D.counter, 0, 4, s)) != cudaSuccess) return e;
        kt_begin(h, "dense_push_kernel", s);
        e = dense_push_run(np, n, R, p->max_sweeps, p->sweep_budget, D.Jp, D.hp, D.Fx, D.S_tc, D.rep, D.counter,
                           h->d_stats, h->sm_count, s);
        kt_end(h, s);
        if (e != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(D.active, 0, 4, s)) != cudaSuccess) return e;
        dense_round_end<<<wb, 256, 0, s>>>(n, np, R, p->restarts, p->sweep_budget, D.S_tc, D.rep, D.best,
                                           D.active, h->d_stats);
        h->launches += 3;
        if ((e = cudaMemcpyAsync(D.h_active, D.active, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(D.h_err, D.err, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if (*D.h_err != 0) return cudaErrorLaunchTimeout;
        if (*D.h_active == 0) break;
      }
      int8_t *outb = spins + (int64_t)R * h->inst[b].spin_off;
      const int64_t tot = (int64_t)R * n;
      dense_tc_output<<<(int)std::min<int64_t>((tot + 255) / 256, (int64_t)h->sm_count * 16), 256, 0, s>>>(
          n, np, R, D.S_tc, D.best, D.rep, outb, E + (int64_t)b * R, minima ? minima + (int64_t)b * R : nullptr);
      h->launches += 1;
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      // energies of the returned states: the library's own tensor-core GEMMs
      // over the exact digit planes of J (dense_energy.cu)
      kt_begin(h, "dense_energy_tc", s);
      int nl = 0;
      e = dense_energy_run(outb, n, np, R, D.hp, D.planes, D.bands, D.planes_F, D.Se, D.Epint, D.Eph,
                           E + (int64_t)b * R, D.err, h->sm_count, &nl, s);
      h->launches += (uint64_t)nl;
      kt_end(h, s);
      if (e != cudaSuccess) return e;
      if ((e = cudaMemcpyAsync(D.h_err, D.err, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
      if (*D.h_err != 0) return cudaErrorLaunchTimeout;
      joff += (int64_t)n * n;
      continue;
    }
    // the comparator: blocks with library GEMMs (cuBLAS), created on first use
    if (!D.cublas) {
      if (cublasCreate(&D.cublas) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
      // a fixed workspace, so that the GEMMs captured into the sweep graph never allocate
      constexpr size_t kWs = 64u << 20;
      if ((e = cudaMalloc(&D.workspace, kWs)) != cudaSuccess) return e;
      if (cublasSetWorkspace(D.cublas, D.workspace, kWs) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    }
    if (cublasSetStream(D.cublas, s) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    const int rb = (R + 255) / 256;
    dense_init<<<rb, 256, 0, s>>>(R, D.rep, h->d_stats);
    // capture one sweep into a graph, replay it sweep by sweep
    cudaStream_t cs;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cublasSetStream(D.cublas, cs);
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    bool ok = e == cudaSuccess;
    if (ok) {
      dense_start<<<dim3(rb, (n + 127) / 128), 256, 0, cs>>>(n, R, Rp, seed, b, D.rep, D.S);
      for (int b0 = 0; b0 < n && ok; b0 += kDB) {
        const int cnt = std::min(kDB, n - b0);
        ok = fields(D, b0, cnt, D.F);
        dense_decide<<<rb, 256, kDB * kDB * sizeof(float), cs>>>(n, R, Rp, b0, cnt, J, hf, D.F, D.S, D.rep);
      }
      cudaMemsetAsync(D.active, 0, 4, cs);
      dense_end<<<rb, 256, 0, cs>>>(R, n, p->max_sweeps, p->sweep_budget, D.rep, D.active, h->d_stats);
      cudaMemcpyAsync(D.h_active, D.active, 4, cudaMemcpyDeviceToHost, cs);
      e = cudaStreamEndCapture(cs, &graph);
      ok = ok && e == cudaSuccess;
    }
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    cublasSetStream(D.cublas, s);
    if (!ok) {
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cs);
      return e != cudaSuccess ? e : cudaErrorUnknown;
    }
    for (int round = 0;; ++round) {
      // one descent round: sweep until no replica is active
      for (int sw = 0;; ++sw) {
        if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) break;
        h->launches += 2 + (n + kDB - 1) / kDB;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        if (*D.h_active == 0) break;
      }
      if (e != cudaSuccess) break;
      fields(D, 0, n, D.Ff);
      dense_energy<<<rb, 256, 0, s>>>(n, R, Rp, D.S, D.Ff, hf, D.rep, D.best, 0);
      cudaMemsetAsync(D.active, 0, 4, s);
      dense_next_round<<<rb, 256, 0, s>>>(R, p->restarts, p->sweep_budget, D.rep, D.active, h->d_stats);
      cudaMemcpyAsync(D.h_active, D.active, 4, cudaMemcpyDeviceToHost, s);
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
      if (*D.h_active == 0) break;
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return e;
    // energies of replicas that never converged: their final states
    dense_energy<<<rb, 256, 0, s>>>(n, R, Rp, D.S, D.Ff, hf, D.rep, D.best, 1);
    const int64_t tot = (int64_t)R * n;
    dense_output<<<(int)std::min<int64_t>((tot + 255) / 256, (int64_t)h->sm_count * 16), 256, 0, s>>>(
        n, R, Rp, b, h->inst[b].spin_off, D.S, D.best, D.rep, spins, E, minima);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exact_energies(D, h, n, R, J, hf, spins + (int64_t)R * h->inst[b].spin_off, E + (int64_t)b * R, s)) !=
        cudaSuccess)
      return e;
    joff += (int64_t)n * n;
  }
  return cudaSuccess;
}

}  // namespace isg
