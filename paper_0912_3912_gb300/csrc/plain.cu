// plain.cu — the plain comparator: the same search semantics written the
// straightforward way.  One instance at a time; one thread per (spin,
// replica); spins as int8, fields as FP32/int32 arrays in global memory (FP64
// instances: every field recomputed in FP64 at each visit); one
// launch per colour class per sweep, plus per-sweep bookkeeping launches; the
// host polls for completion.  No bit packing, no shared-memory residency, no
// persistent kernel, no graph.  It is the baseline the tile, multi-spin coded
// and sweep kernels are measured against at equal results.
#include <cfloat>

#include "device_common.cuh"

namespace isg {

namespace {

struct PlainRep {
  int32_t d, k, total, minima, flips, state;  // state bits: 1 active, 2 start, 4 done, 8 ended
  int32_t converged, pad;
  double best, last;
};

constexpr int kPT = 256;

__global__ void plain_start(const DevGraph G, InstDesc I, int32_t R, int32_t b, uint64_t seed, int8_t *s,
                            uint8_t *fm, PlainRep *rep) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)R * I.n) return;
  const int r = (int)(t / I.n), i = (int)(t % I.n);
  if (!(rep[r].state & 2)) return;
  const uint4 x = start_bits(seed, (uint32_t)(i / 128), (uint32_t)r, (uint32_t)rep[r].k, (uint32_t)b);
  const int q = (i % 128);
  s[t] = ((word_of(x, q / 32) >> (q % 32)) & 1u) ? 1 : -1;
  fm[t] = 0;
}

__global__ void plain_start_done(PlainRep *rep, int32_t R, unsigned long long *stats) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  if (rep[r].state & 2) {
    rep[r].state = 1;
    rep[r].d = 0;
    atomicAdd(stats + 3, 1ull);
  }
}

// KIND: 0 int8 couplings, 1 FP32, 2 FP64
template <int KIND>
__global__ void plain_visit(const DevGraph G, InstDesc I, int32_t R, int32_t c0, int32_t csize, int32_t sequential,
                            int32_t refresh, int8_t *s, uint8_t *fm, float *F, PlainRep *rep) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)R * csize) return;
  const int r = (int)(t / csize), v = c0 + (int)(t % csize);
  if (!(rep[r].state & 1)) return;
  const int j = sequential ? v : __ldg(G.order + I.spin_off + v);
  const int64_t gj = I.spin_off + j;
  int8_t *sr = s + (int64_t)r * I.n;
  uint8_t *fr = fm + (int64_t)r * I.n;
  const uint32_t k0 = __ldg(G.row + gj), k1 = __ldg(G.row + gj + 1);
  const uint32_t e0 = __ldg(G.inc_ptr + gj), e1 = __ldg(G.inc_ptr + gj + 1);
  bool flip;
  if (KIND == 2) {
    // FP64: the field from scratch in the definition's order (h, the CSR row,
    // then the hyper-edges ascending), each step one FP64 addition
    const double *Jd = reinterpret_cast<const double *>(G.J);
    const double *hJ = reinterpret_cast<const double *>(G.hJ);
    double f = __ldg(reinterpret_cast<const double *>(G.h) + gj);
    for (uint32_t k = k0; k < k1; ++k) {
      const double w = __ldg(Jd + k);
      f = __dadd_rn(f, sr[__ldg(G.col + k)] > 0 ? w : -w);
    }
    for (uint32_t q = e0; q < e1; ++q) {
      const int e = __ldg(G.inc_edge + q);
      int neg = 0;
      for (uint32_t m = __ldg(G.hptr + e); m < __ldg(G.hptr + e + 1); ++m) {
        const int mm = __ldg(G.hmem + m);
        if (mm != j) neg ^= sr[mm] < 0;
      }
      const double w = __ldg(hJ + e);
      f = __dadd_rn(f, neg ? -w : w);
    }
    flip = sr[j] > 0 ? (f < 0.0) : (f > 0.0);
  } else if (KIND == 0) {
    const int8_t *Ji = reinterpret_cast<const int8_t *>(G.J);
    const int8_t *hJ = reinterpret_cast<const int8_t *>(G.hJ);
    int f = __ldg(reinterpret_cast<const int8_t *>(G.h) + gj);
    for (uint32_t k = k0; k < k1; ++k) f += (int)__ldg(Ji + k) * (int)sr[__ldg(G.col + k)];
    for (uint32_t q = e0; q < e1; ++q) {
      const int e = __ldg(G.inc_edge + q);
      int p = 1;
      for (uint32_t m = __ldg(G.hptr + e); m < __ldg(G.hptr + e + 1); ++m) {
        const int mm = __ldg(G.hmem + m);
        if (mm != j) p *= sr[mm];
      }
      f += (int)__ldg(hJ + e) * p;
    }
    flip = (int)sr[j] * f < 0;
  } else {
    const float *Jf = reinterpret_cast<const float *>(G.J);
    const float *hJ = reinterpret_cast<const float *>(G.hJ);
    const int d = rep[r].d;
    float f;
    if (d == 0 || (refresh > 0 && d % refresh == 0)) {
      double acc = (double)__ldg(reinterpret_cast<const float *>(G.h) + gj);
      for (uint32_t k = k0; k < k1; ++k) acc = __dadd_rn(acc, (double)__ldg(Jf + k) * (double)sr[__ldg(G.col + k)]);
      for (uint32_t q = e0; q < e1; ++q) {
        const int e = __ldg(G.inc_edge + q);
        double p = 1.0;
        for (uint32_t m = __ldg(G.hptr + e); m < __ldg(G.hptr + e + 1); ++m) {
          const int mm = __ldg(G.hmem + m);
          if (mm != j) p *= (double)sr[mm];
        }
        acc = __dadd_rn(acc, (double)__ldg(hJ + e) * p);
      }
      f = __double2float_rn(acc);
    } else {
      f = F[(int64_t)r * I.n + j];
      for (uint32_t k = k0; k < k1; ++k) {
        const int i = __ldg(G.col + k);
        if (fr[i]) f = __fadd_rn(f, 2.0f * __ldg(Jf + k) * (float)sr[i]);
      }
      for (uint32_t q = e0; q < e1; ++q) {
        const int e = __ldg(G.inc_edge + q);
        float p = 1.0f;
        int par = 0;
        for (uint32_t m = __ldg(G.hptr + e); m < __ldg(G.hptr + e + 1); ++m) {
          const int mm = __ldg(G.hmem + m);
          if (mm != j) {
            p *= (float)sr[mm];
            par ^= fr[mm];
          }
        }
        if (par) f = __fadd_rn(f, 2.0f * __ldg(hJ + e) * p);
      }
    }
    F[(int64_t)r * I.n + j] = f;
    flip = sr[j] > 0 ? (f < 0.0f) : (f > 0.0f);
  }
  if (KIND != 2) fr[j] = flip ? 1 : 0;
  if (flip) {
    sr[j] = (int8_t)-sr[j];
    atomicAdd(&rep[r].flips, 1);
  }
}

__global__ void plain_end(PlainRep *rep, int32_t R, int32_t n, int32_t max_sweeps, int32_t budget,
                          unsigned long long *stats) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R || !(rep[r].state & 1)) return;
  PlainRep &p = rep[r];
  p.total += 1;
  p.d += 1;
  atomicAdd(stats + 0, (unsigned long long)n);
  atomicAdd(stats + 1, (unsigned long long)p.flips);
  atomicAdd(stats + 4, 1ull);
  const bool conv = p.flips == 0;
  p.flips = 0;
  if (conv || p.d >= max_sweeps || (budget > 0 && p.total >= budget)) {
    p.state = 8;
    p.converged = conv ? 1 : 0;
  }
}

template <int KIND>
__global__ void plain_energy(const DevGraph G, InstDesc I, int32_t R, int32_t restarts, int32_t budget,
                             const int8_t *s, int8_t *best, PlainRep *rep, unsigned long long *stats) {
  __shared__ double redd[kPT / 32];
  __shared__ long long redi[kPT / 32];
  __shared__ int s_copy;
  __shared__ double s_E;
  const int r = blockIdx.x;
  if (!(rep[r].state & 8)) return;
  const int8_t *sr = s + (int64_t)r * I.n;
  double E;
  if (KIND == 2) {
    // FP64: one thread, the compensated sequential sum of the definition
    if (threadIdx.x == 0) s_E = energy_f64_seq(G, I, sr);
    __syncthreads();
    E = s_E;
  } else if (KIND == 1) {
    const float *Jf = reinterpret_cast<const float *>(G.J);
    const float *hf = reinterpret_cast<const float *>(G.h);
    const float *hJ = reinterpret_cast<const float *>(G.hJ);
    double acc = 0.0;
    for (int i = threadIdx.x; i < I.n; i += blockDim.x) {
      const int64_t gi = I.spin_off + i;
      double e = (double)hf[gi] * sr[i];
      for (uint32_t k = G.row[gi]; k < G.row[gi + 1]; ++k)
        if (G.col[k] > i) e += (double)Jf[k] * sr[i] * sr[G.col[k]];
      acc -= e;
    }
    for (int e = threadIdx.x; e < I.n_hyper; e += blockDim.x) {
      const int64_t ge = I.hyper_off + e;
      double p = 1.0;
      for (uint32_t q = G.hptr[ge]; q < G.hptr[ge + 1]; ++q) p *= sr[G.hmem[q]];
      acc -= (double)hJ[ge] * p;
    }
    E = block_sum(acc, redd);
  } else {
    const int8_t *Ji = reinterpret_cast<const int8_t *>(G.J);
    const int8_t *hi = reinterpret_cast<const int8_t *>(G.h);
    const int8_t *hJ = reinterpret_cast<const int8_t *>(G.hJ);
    long long acc = 0;
    for (int i = threadIdx.x; i < I.n; i += blockDim.x) {
      const int64_t gi = I.spin_off + i;
      int e = hi[gi] * sr[i];
      for (uint32_t k = G.row[gi]; k < G.row[gi + 1]; ++k)
        if (G.col[k] > i) e += Ji[k] * sr[i] * sr[G.col[k]];
      acc -= e;
    }
    for (int e = threadIdx.x; e < I.n_hyper; e += blockDim.x) {
      const int64_t ge = I.hyper_off + e;
      int p = 1;
      for (uint32_t q = G.hptr[ge]; q < G.hptr[ge + 1]; ++q) p *= sr[G.hmem[q]];
      acc -= (long long)hJ[ge] * p;
    }
    E = (double)block_sum(acc, redi);
  }
  if (threadIdx.x == 0) {
    PlainRep &p = rep[r];
    s_copy = 0;
    if (p.converged) {
      p.minima += 1;
      atomicAdd(stats + 2, 1ull);
      if (E < p.best) {
        p.best = E;
        s_copy = 1;
      }
    }
    p.last = E;
    p.k += 1;
    if (p.k < restarts && (budget <= 0 || p.total < budget)) p.state = 2;
    else p.state = 4;
  }
  __syncthreads();
  if (s_copy)
    for (int i = threadIdx.x; i < I.n; i += blockDim.x) best[(int64_t)r * I.n + i] = sr[i];
}

__global__ void plain_count_done(const PlainRep *rep, int32_t R, int32_t *done) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R && (rep[r].state & 4)) atomicAdd(done, 1);
}

__global__ void plain_output(InstDesc I, int32_t R, int32_t b, const int8_t *s, const int8_t *best,
                             const PlainRep *rep, int8_t *out, double *E, int32_t *E32, int32_t *minima) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (int64_t)R * I.n) {
    const int r = (int)(t / I.n);
    out[(int64_t)R * I.spin_off + t] = rep[r].minima > 0 ? best[t] : s[t];
  }
  if (t < R) {
    const PlainRep &p = rep[t];
    const double e = p.minima > 0 ? p.best : p.last;
    E[(int64_t)b * R + t] = e;
    if (E32) E32[(int64_t)b * R + t] = (int32_t)e;
    if (minima) minima[(int64_t)b * R + t] = p.minima;
  }
}

__global__ void plain_reset(PlainRep *rep, int32_t R) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  PlainRep p;
  p.d = p.k = p.total = p.minima = p.flips = 0;
  p.state = 2;
  p.converged = p.pad = 0;
  p.best = DBL_MAX;
  p.last = 0.0;
  rep[r] = p;
}

struct PlainState : FamilyState {
  size_t cap_elems = 0;
  int32_t cap_R = 0;
  int8_t *s = nullptr, *best = nullptr;
  uint8_t *fm = nullptr;
  float *F = nullptr;
  PlainRep *rep = nullptr;
  int32_t *done = nullptr, *h_done = nullptr;
};


}  // namespace

void plain_free(ising_handle *h) {
  if (!h->plain_st) return;
  PlainState &P = static_cast<PlainState &>(*h->plain_st);
  cudaFree(P.s);
  cudaFree(P.best);
  cudaFree(P.fm);
  cudaFree(P.F);
  cudaFree(P.rep);
  cudaFree(P.done);
  if (P.h_done) cudaFreeHost(P.h_done);
  h->plain_st.reset();
}

// Runs the whole search for every instance, one instance after another.
cudaError_t launch_plain(ising_handle *h, const ising_search_params *p, int32_t R, int8_t *spins, double *E,
                              int32_t *E32, int32_t *minima, const uint64_t *seeds_host, cudaStream_t s) {
  PlainState &P = family_state<PlainState>(h->plain_st);
  const size_t need = (size_t)R * h->nmax;
  cudaError_t e;
  if (need > P.cap_elems || R > P.cap_R) {
    cudaFree(P.s);
    cudaFree(P.best);
    cudaFree(P.fm);
    cudaFree(P.F);
    cudaFree(P.rep);
    if ((e = cudaMalloc(&P.s, need)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&P.best, need)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&P.fm, need)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&P.F, need * sizeof(float))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&P.rep, R * sizeof(PlainRep))) != cudaSuccess) return e;
    if (!P.done && (e = cudaMalloc(&P.done, sizeof(int32_t))) != cudaSuccess) return e;
    if (!P.h_done && (e = cudaMallocHost(&P.h_done, sizeof(int32_t))) != cudaSuccess) return e;
    P.cap_elems = need;
    P.cap_R = R;
  }
  const DevGraph G = h->graph();
  const int kind = h->dtype == ISING_F64 ? 2 : (h->dtype == ISING_F32 ? 1 : 0);
  const int seq = p->schedule == ISING_SCHED_SEQUENTIAL;
  const int rb = (R + kPT - 1) / kPT;
  for (int32_t b = 0; b < h->n_inst; ++b) {
    const InstDesc I = h->inst[b];
    const int64_t tot = (int64_t)R * I.n;
    const int nb = (int)((tot + kPT - 1) / kPT);
    const int32_t *cls = h->h_cls.data() + I.cls_off;
    const int ncls = seq ? I.n : I.ncls;
    plain_reset<<<rb, kPT, 0, s>>>(P.rep, R);
    for (int sweep = 0;; ++sweep) {
      h->launches += 5 + ncls;
      plain_start<<<nb, kPT, 0, s>>>(G, I, R, b, seeds_host[b], P.s, P.fm, P.rep);
      plain_start_done<<<rb, kPT, 0, s>>>(P.rep, R, h->d_stats);
      for (int c = 0; c < ncls; ++c) {
        const int c0 = seq ? c : cls[c], cs = seq ? 1 : cls[c + 1] - cls[c];
        if (cs <= 0) continue;
        const int vb = (int)(((int64_t)R * cs + kPT - 1) / kPT);
        if (kind == 1)
          plain_visit<1><<<vb, kPT, 0, s>>>(G, I, R, c0, cs, seq, p->refresh_every, P.s, P.fm, P.F, P.rep);
        else if (kind == 2)
          plain_visit<2><<<vb, kPT, 0, s>>>(G, I, R, c0, cs, seq, p->refresh_every, P.s, P.fm, P.F, P.rep);
        else
          plain_visit<0><<<vb, kPT, 0, s>>>(G, I, R, c0, cs, seq, p->refresh_every, P.s, P.fm, P.F, P.rep);
      }
      plain_end<<<rb, kPT, 0, s>>>(P.rep, R, I.n, p->max_sweeps, p->sweep_budget, h->d_stats);
      if (kind == 1)
        plain_energy<1><<<R, kPT, 0, s>>>(G, I, R, p->restarts, p->sweep_budget, P.s, P.best, P.rep, h->d_stats);
      else if (kind == 2)
        plain_energy<2><<<R, kPT, 0, s>>>(G, I, R, p->restarts, p->sweep_budget, P.s, P.best, P.rep, h->d_stats);
      else
        plain_energy<0><<<R, kPT, 0, s>>>(G, I, R, p->restarts, p->sweep_budget, P.s, P.best, P.rep, h->d_stats);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if (sweep % 8 == 7) {
        cudaMemsetAsync(P.done, 0, sizeof(int32_t), s);
        plain_count_done<<<rb, kPT, 0, s>>>(P.rep, R, P.done);
        cudaMemcpyAsync(P.h_done, P.done, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if (*P.h_done == R) break;
      }
    }
    plain_output<<<(int)((std::max<int64_t>(tot, R) + kPT - 1) / kPT), kPT, 0, s>>>(I, R, b, P.s, P.best, P.rep,
                                                                                   spins, E, E32, minima);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace isg
