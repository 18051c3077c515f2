// energy.cu — energies of caller-supplied configurations (Eq. 1 extended by
// Eq. 6), int8 spins [instance][replica][spin].  Two passes with a fixed
// summation order: blocks of kChunk spins (and a proportional share of the
// hyper-edges) write partial sums; a second kernel adds them in order.
// FP64 for float couplings; exact int64 for integer couplings; for FP64
// couplings one thread per configuration takes the compensated sequential sum
// the C ABI defines for them.
#include "device_common.cuh"

namespace isg {

namespace {
constexpr int kChunk = 4096;
constexpr int kThreads = 256;

struct EnergyWork {
  int32_t b, r, chunk, nchunks;
};

template <bool FLOAT>
__global__ void __launch_bounds__(kThreads) energy_partial_kernel(DevGraph G, const int8_t *__restrict__ spins,
                                                                  int32_t R, const int4 *__restrict__ work,
                                                                  double *partd, long long *parti) {
  __shared__ double redd[kThreads / 32];
  __shared__ long long redi[kThreads / 32];
  const int4 wk = work[blockIdx.x];  // (b, r, chunk, nchunks)
  const InstDesc I = G.inst[wk.x];
  const int8_t *s = spins + (int64_t)R * I.spin_off + (int64_t)wk.y * I.n;
  const int i0 = wk.z * kChunk, i1 = min(I.n, i0 + kChunk);
  const int e_per = (I.n_hyper + wk.w - 1) / wk.w;
  const int ea = wk.z * e_per, eb = min(I.n_hyper, ea + e_per);
  if (FLOAT) {
    const float *Jf = reinterpret_cast<const float *>(G.J);
    const float *hf = reinterpret_cast<const float *>(G.h);
    const float *hJ = reinterpret_cast<const float *>(G.hJ);
    double acc = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const int64_t gi = I.spin_off + i;
      const double si = (double)s[i];
      double e = (double)__ldg(hf + gi) * si;
      for (uint32_t k = __ldg(G.row + gi), ke = __ldg(G.row + gi + 1); k < ke; ++k) {
        const int j = __ldg(G.col + k);
        if (j > i) e += (double)__ldg(Jf + k) * si * (double)s[j];
      }
      acc -= e;
    }
    for (int e = ea + threadIdx.x; e < eb; e += blockDim.x) {
      const int64_t ge = I.hyper_off + e;
      double p = 1.0;
      for (uint32_t q = __ldg(G.hptr + ge), qe = __ldg(G.hptr + ge + 1); q < qe; ++q)
        p *= (double)s[__ldg(G.hmem + q)];
      acc -= (double)__ldg(hJ + ge) * p;
    }
    acc = block_sum(acc, redd);
    if (threadIdx.x == 0) partd[blockIdx.x] = acc;
  } else {
    const int8_t *Ji = reinterpret_cast<const int8_t *>(G.J);
    const int8_t *hi = reinterpret_cast<const int8_t *>(G.h);
    const int8_t *hJ = reinterpret_cast<const int8_t *>(G.hJ);
    long long acc = 0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const int64_t gi = I.spin_off + i;
      const int si = s[i];
      int e = (int)__ldg(hi + gi) * si;
      for (uint32_t k = __ldg(G.row + gi), ke = __ldg(G.row + gi + 1); k < ke; ++k) {
        const int j = __ldg(G.col + k);
        if (j > i) e += (int)__ldg(Ji + k) * si * (int)s[j];
      }
      acc -= e;
    }
    for (int e = ea + threadIdx.x; e < eb; e += blockDim.x) {
      const int64_t ge = I.hyper_off + e;
      int p = 1;
      for (uint32_t q = __ldg(G.hptr + ge), qe = __ldg(G.hptr + ge + 1); q < qe; ++q)
        p *= (int)s[__ldg(G.hmem + q)];
      acc -= (long long)__ldg(hJ + ge) * p;
    }
    acc = block_sum(acc, redi);
    if (threadIdx.x == 0) parti[blockIdx.x] = acc;
  }
}

__global__ void energy_finish_kernel(const int4 *__restrict__ work, int32_t nwork, const int32_t *__restrict__ first,
                                     int32_t nout, int32_t R, const double *partd, const long long *parti,
                                     bool is_float, double *E, int32_t *E32) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;  // o = b * R + r
  if (o >= nout) return;
  const int w0 = first[o];
  const int nch = work[w0].w;
  if (is_float) {
    double acc = 0.0;
    for (int c = 0; c < nch; ++c) acc += partd[w0 + c];
    E[o] = acc;
  } else {
    long long acc = 0;
    for (int c = 0; c < nch; ++c) acc += parti[w0 + c];
    E[o] = (double)acc;
    if (E32) E32[o] = (int32_t)acc;
  }
  (void)nwork;
  (void)R;
}
// FP64 instances: the defined sequential compensated sum, one thread per
// (instance, replica)
__global__ void energy_f64_kernel(DevGraph G, int32_t n_inst, const int8_t *__restrict__ spins, int32_t R,
                                  double *E) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_inst * R) return;
  const int b = (int)(t / R), r = (int)(t % R);
  const InstDesc I = G.inst[b];
  E[t] = energy_f64_seq(G, I, spins + (int64_t)R * I.spin_off + (int64_t)r * I.n);
}

}  // namespace

void energy_plan_free(ising_handle *h) {
  cudaFree(h->d_en_work);
  cudaFree(h->d_en_first);
  cudaFree(h->d_en_partd);
  cudaFree(h->d_en_parti);
  h->d_en_work = nullptr;
  h->d_en_first = nullptr;
  h->d_en_partd = nullptr;
  h->d_en_parti = nullptr;
  h->en_R = -1;
  h->en_nwork = 0;
}

// Host launcher: builds (once per replica count) the chunk work list, then runs
// the two passes on stream s.  The work list and partial sums live in the handle.
cudaError_t launch_energy(ising_handle *h, const int8_t *spins, int32_t R, double *E, int32_t *E32,
                          cudaStream_t s) {
  cudaError_t e;
  if (h->en_R != R) {
    energy_plan_free(h);
    std::vector<int4> work;
    std::vector<int32_t> first;
    for (int b = 0; b < h->n_inst; ++b) {
      const int nch = (int)((h->inst[b].n + kChunk - 1) / kChunk);
      for (int r = 0; r < R; ++r) {
        first.push_back((int32_t)work.size());
        for (int c = 0; c < nch; ++c) work.push_back(make_int4(b, r, c, nch));
      }
    }
    h->en_nwork = (int32_t)work.size();
    if ((e = cudaMalloc(&h->d_en_work, work.size() * sizeof(int4))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&h->d_en_first, first.size() * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&h->d_en_partd, work.size() * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&h->d_en_parti, work.size() * sizeof(long long))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(h->d_en_work, work.data(), work.size() * sizeof(int4), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return e;
    if ((e = cudaMemcpy(h->d_en_first, first.data(), first.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return e;
    h->en_R = R;
  }
  const DevGraph G = h->graph();
  const bool fl = h->dtype == ISING_F32;
  if (h->dtype == ISING_F64) {
    const int64_t nout = (int64_t)h->n_inst * R;
    energy_f64_kernel<<<(int)((nout + 127) / 128), 128, 0, s>>>(G, h->n_inst, spins, R, E);
    return cudaGetLastError();
  }
  if (fl)
    energy_partial_kernel<true><<<h->en_nwork, kThreads, 0, s>>>(G, spins, R, h->d_en_work, h->d_en_partd, h->d_en_parti);
  else
    energy_partial_kernel<false><<<h->en_nwork, kThreads, 0, s>>>(G, spins, R, h->d_en_work, h->d_en_partd, h->d_en_parti);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nout = h->n_inst * R;
  energy_finish_kernel<<<(nout + 255) / 256, 256, 0, s>>>(h->d_en_work, h->en_nwork, h->d_en_first, nout, R, h->d_en_partd,
                                                          h->d_en_parti, fl, E, E32);
  return cudaGetLastError();
}

}  // namespace isg
