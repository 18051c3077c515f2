// api.cu — the C ABI (include/ising.h): instance validation and upload,
// colouring, planning, dispatch to the kernel families, status strings.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace isg {
cudaError_t launch_plain(ising_handle *h, const ising_search_params *p, int32_t R, int8_t *spins, double *E,
                         int32_t *E32, int32_t *minima, const uint64_t *seeds_host, cudaStream_t s);
cudaError_t launch_sweep(ising_handle *h, const ising_search_params *p, int32_t R, int8_t *spins, double *E,
                         int32_t *E32, int32_t *minima, const uint64_t *seeds_host, cudaStream_t s);
cudaError_t launch_dense(ising_handle *h, const ising_search_params *p, int32_t R, int8_t *spins, double *E,
                         int32_t *E32, int32_t *minima, const uint64_t *seeds_host, cudaStream_t s);
bool dense_supported(const ising_handle *h, int32_t R);
void sweep_free(ising_handle *h);
void dense_free(ising_handle *h);
void plain_free(ising_handle *h);
}  // namespace isg

using namespace isg;

#define CUDA_OK(x)                          \
  do {                                      \
    if ((x) != cudaSuccess) return ISING_ERR_CUDA; \
  } while (0)

DevGraph ising_handle::graph() const {
  DevGraph g;
  g.inst = d_inst;
  g.row = d_row;
  g.col = d_col;
  g.J = d_J;
  g.h = d_h;
  g.inc_ptr = d_inc_ptr;
  g.inc_edge = d_inc_edge;
  g.inc_oth = d_inc_oth;
  g.hptr = d_hptr;
  g.hmem = d_hmem;
  g.hJ = d_hJ;
  g.order = d_order;
  g.cls = d_cls;
  g.meta = d_meta;
  g.Jpos = d_Jpos;
  g.latinfo = d_latinfo;
  g.Jfwd = d_Jfwd;
  g.runit = d_runit;
  g.nsp = total_spins;
  g.dtype = dtype;
  return g;
}

namespace {

// ---------------------------------------------------------------- validation
struct HostInst {
  int32_t n = 0;
  std::vector<int64_t> row;  // n + 1
  std::vector<int32_t> col;
  std::vector<float> Jf;
  std::vector<int8_t> Ji;
  std::vector<double> Jd;  // ISING_F64
  std::vector<float> hf;
  std::vector<int8_t> hi;
  std::vector<double> hd;
  std::vector<int64_t> hptr;
  std::vector<int32_t> hmem;
  std::vector<float> hJf;
  std::vector<int8_t> hJi;
  std::vector<double> hJd;
  std::vector<int32_t> colour;
  int32_t ncls = 0;
  int32_t max_deg = 0;
  int32_t lat_L = 0, lat_d = 0;
};

// Unit (biased exponent) for exact fixed-point energies of an FP32 instance.
// Every nonzero coupling and field is then an integer multiple M << (e - ebase)
// of 2^(ebase - 150) with a 24-bit M; with a spread of at most 38 every term
// fits below 2^62, and the high halves of up to 2^22 terms stay below 2^53 so
// the final conversion to FP64 rounds once.  Returns -1 when that does not hold
// (subnormal values, a wider spread or more terms).
int32_t energy_base_exponent(const HostInst &I, int32_t *emax_out = nullptr) {
  int emin = 256, emax = -1;
  bool sub = false;
  auto see = [&](float v) {
    uint32_t b;
    std::memcpy(&b, &v, 4);
    b &= 0x7fffffffu;
    if (!b) return;
    const int e = (int)(b >> 23);
    if (e == 0 || e == 255) sub = true;
    emin = std::min(emin, e);
    emax = std::max(emax, e);
  };
  for (float v : I.Jf) see(v);
  for (float v : I.hf) see(v);
  for (float v : I.hJf) see(v);
  if (emax_out) *emax_out = emax;
  if (sub) return -1;
  if (emax < 0) return 1;  // all zero
  const int64_t terms = (int64_t)I.col.size() / 2 + I.n + (int64_t)I.hJf.size();
  if (emax - emin > 38 || terms >= (int64_t)1 << 22) return -1;
  return emin;
}

// InstDesc::fx53: with unit u (2^(ebase - 150), or 1 for int8), A = the sum
// of |term| / u over the energy's terms (each pair once, fields, hyper-edge
// couplings) bounds every energy, every field and every partial sum of either
// (each is a signed sum of a subset of those terms); below 2^53 all of them
// are exact in FP64, and the gains, twice a field, are too.
int32_t fp64_exact(const HostInst &I, bool fl, int32_t ebase) {
  if (!fl) return 1;  // |terms| <= 127 and far fewer than 2^45 of them
  if (ebase < 0) return 0;
  auto units = [&](float v) -> unsigned __int128 {
    uint32_t b;
    std::memcpy(&b, &v, 4);
    b &= 0x7fffffffu;
    if (!b) return 0;
    const int e = (int)(b >> 23);
    return (unsigned __int128)((b & 0x7fffffu) | 0x800000u) << (e - ebase);
  };
  unsigned __int128 pairs2 = 0, rest = 0;  // pairs2: both CSR directions, twice the pair sum
  for (float v : I.Jf) pairs2 += units(v);
  for (float v : I.hf) rest += units(v);
  for (float v : I.hJf) rest += units(v);
  return pairs2 / 2 + rest < ((unsigned __int128)1 << 53) ? 1 : 0;
}

// Recognise a periodic hypercubic lattice (side L >= 3, d = 2 or 3, spin index
// x0 + L*x1 + L^2*x2) from the CSR structure alone.
void detect_lattice(HostInst &I) {
  const int32_t n = I.n;
  for (int d = 3; d >= 2; --d) {
    const int32_t L = (int32_t)std::llround(std::pow((double)n, 1.0 / d));
    int64_t p = 1;
    for (int a = 0; a < d; ++a) p *= L;
    if (L < 3 || p != n || I.max_deg != 2 * d) continue;
    bool ok = true;
    for (int32_t i = 0; i < n && ok; ++i) {
      if (I.row[i + 1] - I.row[i] != 2 * d) { ok = false; break; }
      for (int64_t k = I.row[i]; k < I.row[i + 1] && ok; ++k) {
        const int32_t j = I.col[k];
        bool found = false;
        int64_t stride = 1;
        for (int a = 0; a < d && !found; ++a, stride *= L) {
          const int32_t c = (int32_t)((i / stride) % L);
          const int64_t up = i + (((c + 1) % L) - c) * stride, dn = i + (((c + L - 1) % L) - c) * stride;
          found = (j == up) || (j == dn);
        }
        ok = found;
      }
    }
    if (ok) {
      I.lat_L = L;
      I.lat_d = d;
      return;
    }
  }
}

double jval(const HostInst &I, int64_t k, ising_dtype dt) {
  return dt == ISING_F64 ? I.Jd[k] : (dt == ISING_F32 ? (double)I.Jf[k] : (double)I.Ji[k]);
}

ising_status load_desc(const ising_instance_desc &d, ising_dtype dtype, HostInst &I) {
  const bool fl = dtype == ISING_F32, f64 = dtype == ISING_F64;
  if (d.n < 1 || d.n > (1 << 30)) return ISING_ERR_INVALID_ARG;
  if (d.dtype != dtype) return ISING_ERR_INVALID_ARG;
  const int32_t n = d.n;
  I.n = n;
  if (d.J_dense) {
    if (!fl || d.row_ptr || d.col || d.J) return ISING_ERR_INVALID_ARG;
    if ((int64_t)n * (n - 1) > 0x7fffffffLL) return ISING_ERR_UNSUPPORTED;
    I.row.assign(n + 1, 0);
    for (int32_t i = 0; i < n; ++i) {
      if (d.J_dense[(int64_t)i * n + i] != 0.0f) return ISING_ERR_SELF_LOOP;
      for (int32_t j = 0; j < n; ++j) {
        const float w = d.J_dense[(int64_t)i * n + j];
        if (!std::isfinite(w)) return ISING_ERR_INVALID_ARG;
        if (w != d.J_dense[(int64_t)j * n + i]) return ISING_ERR_ASYMMETRIC;
        if (j == i) continue;
        I.col.push_back(j);
        I.Jf.push_back(w);
      }
      I.row[i + 1] = (int64_t)I.col.size();
    }
  } else {
    if (!d.row_ptr) return ISING_ERR_INVALID_ARG;
    if (d.row_ptr[0] != 0) return ISING_ERR_INVALID_ARG;
    for (int32_t i = 0; i < n; ++i)
      if (d.row_ptr[i + 1] < d.row_ptr[i]) return ISING_ERR_INVALID_ARG;
    const int64_t nnz = d.row_ptr[n];
    if (nnz > 0 && (!d.col || !d.J)) return ISING_ERR_INVALID_ARG;
    if (nnz > 0x7fffffffLL) return ISING_ERR_UNSUPPORTED;
    I.row.assign(d.row_ptr, d.row_ptr + n + 1);
    I.col.assign(d.col, d.col + nnz);
    if (fl) {
      I.Jf.assign((const float *)d.J, (const float *)d.J + nnz);
      for (float w : I.Jf)
        if (!std::isfinite(w)) return ISING_ERR_INVALID_ARG;
    } else if (f64) {
      I.Jd.assign((const double *)d.J, (const double *)d.J + nnz);
      for (double w : I.Jd)
        if (!std::isfinite(w)) return ISING_ERR_INVALID_ARG;
    } else {
      I.Ji.assign((const int8_t *)d.J, (const int8_t *)d.J + nnz);
    }
    // structure: range, self loops, repeats; then symmetry of structure and values
    std::vector<std::pair<int32_t, double>> sorted(nnz);
    for (int32_t i = 0; i < n; ++i) {
      for (int64_t k = I.row[i]; k < I.row[i + 1]; ++k) {
        const int32_t j = I.col[k];
        if (j < 0 || j >= n) return ISING_ERR_INVALID_ARG;
        if (j == i) return ISING_ERR_SELF_LOOP;
        sorted[k] = {j, jval(I, k, dtype)};
      }
      std::sort(sorted.begin() + I.row[i], sorted.begin() + I.row[i + 1]);
      for (int64_t k = I.row[i] + 1; k < I.row[i + 1]; ++k)
        if (sorted[k].first == sorted[k - 1].first) return ISING_ERR_INVALID_ARG;
    }
    for (int32_t i = 0; i < n; ++i)
      for (int64_t k = I.row[i]; k < I.row[i + 1]; ++k) {
        const int32_t j = sorted[k].first;
        auto lo = sorted.begin() + I.row[j], hi = sorted.begin() + I.row[j + 1];
        auto it = std::lower_bound(lo, hi, std::make_pair(i, -(double)INFINITY));
        if (it == hi || it->first != i || it->second != sorted[k].second) return ISING_ERR_ASYMMETRIC;
      }
  }
  for (int32_t i = 0; i < n; ++i) I.max_deg = std::max<int32_t>(I.max_deg, (int32_t)(I.row[i + 1] - I.row[i]));
  if (fl) {
    I.hf.assign(n, 0.0f);
    if (d.h) {
      std::memcpy(I.hf.data(), d.h, n * sizeof(float));
      for (float v : I.hf)
        if (!std::isfinite(v)) return ISING_ERR_INVALID_ARG;
    }
  } else if (f64) {
    I.hd.assign(n, 0.0);
    if (d.h) {
      std::memcpy(I.hd.data(), d.h, n * sizeof(double));
      for (double v : I.hd)
        if (!std::isfinite(v)) return ISING_ERR_INVALID_ARG;
    }
  } else {
    I.hi.assign(n, 0);
    if (d.h) std::memcpy(I.hi.data(), d.h, n);
  }
  // hyper-edges
  if (d.n_hyper < 0) return ISING_ERR_INVALID_ARG;
  I.hptr.assign(1, 0);
  if (d.n_hyper > 0) {
    if (!d.hyper_ptr || !d.hyper_members || !d.hyper_J) return ISING_ERR_INVALID_ARG;
    if (d.hyper_ptr[0] != 0) return ISING_ERR_BAD_HYPEREDGE;
    std::vector<int32_t> seen(n, -1);
    for (int32_t e = 0; e < d.n_hyper; ++e) {
      const int64_t a = d.hyper_ptr[e], b = d.hyper_ptr[e + 1];
      if (b - a < 2) return ISING_ERR_BAD_HYPEREDGE;
      for (int64_t q = a; q < b; ++q) {
        const int32_t m = d.hyper_members[q];
        if (m < 0 || m >= n || seen[m] == e) return ISING_ERR_BAD_HYPEREDGE;
        seen[m] = e;
        I.hmem.push_back(m);
      }
      I.hptr.push_back((int64_t)I.hmem.size());
    }
    if (fl) {
      I.hJf.assign((const float *)d.hyper_J, (const float *)d.hyper_J + d.n_hyper);
      for (float v : I.hJf)
        if (!std::isfinite(v)) return ISING_ERR_INVALID_ARG;
    } else if (f64) {
      I.hJd.assign((const double *)d.hyper_J, (const double *)d.hyper_J + d.n_hyper);
      for (double v : I.hJd)
        if (!std::isfinite(v)) return ISING_ERR_INVALID_ARG;
    } else {
      I.hJi.assign((const int8_t *)d.hyper_J, (const int8_t *)d.hyper_J + d.n_hyper);
    }
  }
  // colouring of the conflict graph (CSR edges + pairs inside hyper-edges)
  std::vector<std::vector<int32_t>> inc(n);
  for (int32_t e = 0; e + 1 < (int32_t)I.hptr.size(); ++e)
    for (int64_t q = I.hptr[e]; q < I.hptr[e + 1]; ++q) inc[I.hmem[q]].push_back(e);
  I.colour.assign(n, -1);
  if (d.colour) {
    for (int32_t i = 0; i < n; ++i) {
      if (d.colour[i] < 0 || d.colour[i] >= n) return ISING_ERR_BAD_COLOURING;
      I.colour[i] = d.colour[i];
    }
    for (int32_t i = 0; i < n; ++i) {
      for (int64_t k = I.row[i]; k < I.row[i + 1]; ++k)
        if (I.colour[I.col[k]] == I.colour[i]) return ISING_ERR_BAD_COLOURING;
      for (int32_t e : inc[i])
        for (int64_t q = I.hptr[e]; q < I.hptr[e + 1]; ++q)
          if (I.hmem[q] != i && I.colour[I.hmem[q]] == I.colour[i]) return ISING_ERR_BAD_COLOURING;
    }
  } else {
    // greedy in index order: smallest colour not held by an earlier conflicting spin
    std::vector<int32_t> stamp(n + 1, -1);
    for (int32_t i = 0; i < n; ++i) {
      for (int64_t k = I.row[i]; k < I.row[i + 1]; ++k) {
        const int32_t c = I.colour[I.col[k]];
        if (c >= 0) stamp[c] = i;
      }
      for (int32_t e : inc[i])
        for (int64_t q = I.hptr[e]; q < I.hptr[e + 1]; ++q) {
          const int32_t c = I.colour[I.hmem[q]];
          if (c >= 0) stamp[c] = i;
        }
      int32_t c = 0;
      while (stamp[c] == i) ++c;
      I.colour[i] = c;
    }
  }
  I.ncls = 0;
  for (int32_t c : I.colour) I.ncls = std::max(I.ncls, c + 1);
  if (I.hptr.size() == 1 && !f64) detect_lattice(I);  // (FP64 instances take no lattice path)
  return ISING_OK;
}

// Host-side fault injection for tests (ISING_FAULT): "alloc:k" makes the k-th
// device upload of ising_create fail ("alloc" = the first); "launch" makes
// ising_local_search fail as a failed launch would; "device_timeout" (read by
// the dense tensor-core path) makes one CTA's bounded wait run out.
bool fault_is(const char *what) {
  const char *f = std::getenv("ISING_FAULT");
  return f && std::strncmp(f, what, std::strlen(what)) == 0;
}
int g_alloc_countdown = 0;  // allocations left before the injected failure (0: none)

template <class T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
  if (g_alloc_countdown > 0 && --g_alloc_countdown == 0) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc((void **)dst, std::max<size_t>(1, src.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

void free_handle(ising_handle *h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  for (auto &t : h->ktimers) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  energy_plan_free(h);
  sweep_free(h);
  fm_free(h);
  dense_free(h);
  plain_free(h);
  void *ptrs[] = {h->d_inst, h->d_row, h->d_col, h->d_J, h->d_h, h->d_inc_ptr, h->d_inc_edge, h->d_inc_oth, h->d_hptr,
                  h->d_hmem, h->d_hJ, h->d_order, h->d_cls, h->d_Jdense, h->d_meta, h->d_Jpos, h->d_Jfwd, h->d_latinfo, h->d_runit,
                  h->d_scratch, h->d_tile_args,
                  h->d_seeds, h->d_stats, h->d_queue, h->d_tiles};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (h->h_stats_pinned) cudaFreeHost(h->h_stats_pinned);
  if (h->tile_exec) cudaGraphExecDestroy(h->tile_exec);
  cudaSetDevice(cur);
  delete h;
}

ising_status ensure_scratch(ising_handle *h, size_t bytes) {
  if (bytes <= h->scratch_bytes) return ISING_OK;
  if (h->d_scratch) cudaFree(h->d_scratch);
  h->d_scratch = nullptr;
  h->scratch_bytes = 0;
  if (cudaMalloc(&h->d_scratch, bytes) != cudaSuccess) return ISING_ERR_OOM;
  h->scratch_bytes = bytes;
  return ISING_OK;
}

ising_status validate_params(const ising_search_params *p) {
  if (!p) return ISING_ERR_INVALID_ARG;
  if (p->max_sweeps < 1 || p->restarts < 1 || p->sweep_budget < 0 || p->refresh_every < 0)
    return ISING_ERR_INVALID_ARG;
  if (p->schedule != ISING_SCHED_COLOUR && p->schedule != ISING_SCHED_SEQUENTIAL) return ISING_ERR_INVALID_ARG;
  if (p->kernel < ISING_KERNEL_AUTO || p->kernel > ISING_KERNEL_PLAIN) return ISING_ERR_INVALID_ARG;
  if (p->dense_variant != ISING_DENSE_OWN && p->dense_variant != ISING_DENSE_LIBRARY) return ISING_ERR_INVALID_ARG;
  if (p->cluster_ctas < 0 || p->cluster_ctas > 8 || (p->cluster_ctas & (p->cluster_ctas - 1)))
    return ISING_ERR_INVALID_ARG;
  return ISING_OK;
}

constexpr int kTileSmemLimit = 200 * 1024;

bool tile_fits(const ising_handle *h, int mode) {
  return tile_smem_bytes(mode, h->nmax) <= (size_t)kTileSmemLimit;
}

// Kernel family for these arguments (ISING_KERNEL_AUTO resolved), or negative status.
int32_t resolve_kernel(ising_handle *h, int32_t R, const ising_search_params *p) {
  int32_t k = p->kernel;
  if (h->dtype == ISING_F64)  // FP64 couplings: the plain family only
    return (k == ISING_KERNEL_AUTO || k == ISING_KERNEL_PLAIN) ? ISING_KERNEL_PLAIN : -(int32_t)ISING_ERR_UNSUPPORTED;
  if (k == ISING_KERNEL_AUTO) {
    auto it = h->tuned.find(R);
    if (it != h->tuned.end()) return it->second;
    if (h->dense && dense_supported(h, R)) return ISING_KERNEL_DENSE_TC;
    if (h->msc_ok && tile_fits(h, 2)) return ISING_KERNEL_MSC;
    if (tile_fits(h, h->dtype == ISING_F32 ? 1 : 0)) return ISING_KERNEL_TILE;
    return ISING_KERNEL_SWEEP;
  }
  switch (k) {
    case ISING_KERNEL_TILE:
      return tile_fits(h, h->dtype == ISING_F32 ? 1 : 0) ? k : -(int32_t)ISING_ERR_UNSUPPORTED;
    case ISING_KERNEL_MSC:
      return (h->msc_ok && tile_fits(h, 2)) ? k : -(int32_t)ISING_ERR_UNSUPPORTED;
    case ISING_KERNEL_DENSE_TC:
      return (h->dense && dense_supported(h, R)) ? k : -(int32_t)ISING_ERR_UNSUPPORTED;
    default:
      return k;
  }
}

// Cluster split of the multi-spin-coded lattice path: worth it when the tiles
// alone would leave most SMs idle.  Every instance must split into P
// power-of-two chunks of at least 1024 sites (whole Philox blocks).
int msc_cluster_size(const ising_handle *h, int32_t R, const ising_search_params *p) {
  if (!h->msc_ok || !h->all_lattice || !h->lat_parity || p->schedule != ISING_SCHED_COLOUR) return 0;
  if (p->cluster_ctas == 1) return 0;
  const int64_t tiles = (int64_t)h->n_inst * ((R + 31) / 32);
  for (int P : {8, 4, 2}) {
    if (p->cluster_ctas > 1 && p->cluster_ctas != P) continue;  // restricted to one size
    if (tiles * P > 2 * (int64_t)h->sm_count) continue;
    bool ok = true;
    int d = -1;
    for (const auto &I : h->inst) {
      const int csz = I.n / P;
      if (I.n % P || csz < 1024 || (csz & (csz - 1)) || csz % 128) ok = false;
      if (msc_cluster_smem(csz) + 4096 > 232448) ok = false;  // dynamic + static shared memory of a CTA
      if (d >= 0 && I.lat_d != d) ok = false;
      d = I.lat_d;
    }
    // Clusters of 8 only when every CTA gets an SM of its own and all clusters
    // are resident at once: few replica groups, each spread wider.  With more
    // groups, 4-CTA clusters measured faster than two 8-CTA clusters per SM set.
    if (ok && P == 8 &&
        (tiles * P > (int64_t)h->sm_count ||
         msc_cluster_max_active(const_cast<ising_handle *>(h), (int)tiles, P, h->nmax / P, d) < tiles))
      ok = false;
    if (ok) return P;
  }
  return 0;
}

ising_status run_tile(ising_handle *h, int mode, int32_t R, const ising_search_params *p, int8_t *spins,
                      double *E, int32_t *E32, int32_t *minima, cudaStream_t s) {
  // tiles: (instance, 32-replica group), largest instances first
  const int32_t groups = (R + 31) / 32;
  if (h->tiles_R != R) {
    std::vector<int32_t> ord(h->n_inst);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return h->inst[a].n > h->inst[b].n; });
    std::vector<int2> tiles;
    tiles.reserve((size_t)h->n_inst * groups);
    for (int32_t b : ord)
      for (int32_t g = 0; g < groups; ++g) tiles.push_back(make_int2(b, g));
    if (h->d_tiles) cudaFree(h->d_tiles);
    h->d_tiles = nullptr;
    if (upload(&h->d_tiles, tiles) != cudaSuccess) return ISING_ERR_CUDA;
    h->n_tiles = (int32_t)tiles.size();
    h->tiles_R = R;
  }
  const int P = mode == 3 ? msc_cluster_size(h, R, p) : 0;
  if (P > 0) {
    const size_t bw_bytes = (size_t)h->n_tiles * h->nmax * sizeof(uint32_t);
    ising_status st = ensure_scratch(h, bw_bytes + 256);
    if (st != ISING_OK) return st;
    TileArgs a;
    a.g = h->graph();
    a.tiles = h->d_tiles;
    a.n_tiles = h->n_tiles;
    a.queue = h->d_queue;
    a.R = R;
    a.max_sweeps = p->max_sweeps;
    a.restarts = p->restarts;
    a.budget = p->sweep_budget;
    a.refresh = p->refresh_every;
    a.sequential = 0;
    a.seeds = h->d_seeds;
    a.F = nullptr;
    a.bw = (uint32_t *)h->d_scratch;
    a.nmax = h->nmax;
    a.spins = spins;
    a.energy = E;
    a.energy_i32 = E32;
    a.minima = minima;
    a.stats = h->d_stats;
    CUDA_OK(cudaMemcpyAsync(h->d_tile_args, &a, sizeof(a), cudaMemcpyHostToDevice, s));
    kt_begin(h, "msc_cluster_kernel", s);
    CUDA_OK(launch_msc_cluster(h, h->n_tiles, P, h->nmax / P, h->inst[0].lat_d, s));
    kt_end(h, s);
    h->launches += 1;
    return ISING_OK;
  }
  // FP32 lanes: fields in shared memory for every instance that fits, within a
  // budget that still lets two CTAs share an SM (the kernel is built for two)
  constexpr size_t kFsmBudget = 48 * 1024;
  const int fsm_cap = mode == 1 ? tile_fsm_cap(h->nmax, kFsmBudget) : 0;
  const size_t smem = mode == 1 && fsm_cap > 0 ? (tile_smem_bytes(mode, h->nmax) + 15) / 16 * 16 + (size_t)fsm_cap * 128
                                              : tile_smem_bytes(mode, h->nmax);
  int per_sm = tile_max_ctas_per_sm(mode, smem);
  if (per_sm < 1) return ISING_ERR_UNSUPPORTED;
  const int grid = std::min<int64_t>(h->n_tiles, (int64_t)per_sm * h->sm_count);
  const size_t f_bytes = mode == 1 ? (size_t)grid * h->nmax * 32 * sizeof(float) : 0;
  const size_t bw_bytes = (size_t)grid * h->nmax * sizeof(uint32_t);
  ising_status st = ensure_scratch(h, f_bytes + bw_bytes + 256);
  if (st != ISING_OK) return st;
  TileArgs a;
  a.g = h->graph();
  a.tiles = h->d_tiles;
  a.n_tiles = h->n_tiles;
  a.queue = h->d_queue;
  a.R = R;
  a.max_sweeps = p->max_sweeps;
  a.restarts = p->restarts;
  a.budget = p->sweep_budget;
  a.refresh = p->refresh_every;
  a.sequential = p->schedule == ISING_SCHED_SEQUENTIAL ? 1 : 0;
  a.seeds = h->d_seeds;
  a.F = mode == 1 ? (float *)h->d_scratch : nullptr;
  a.fsm_cap = fsm_cap;
  a.bw = (uint32_t *)((char *)h->d_scratch + ((f_bytes + 255) / 256) * 256);
  a.nmax = h->nmax;
  a.spins = spins;
  a.energy = E;
  a.energy_i32 = E32;
  a.minima = minima;
  a.stats = h->d_stats;
  CUDA_OK(cudaMemcpyAsync(h->d_tile_args, &a, sizeof(a), cudaMemcpyHostToDevice, s));
  // The launch sequence reads its arguments from device memory, so one captured
  // graph serves every call with the same mode, grid and shared memory.
  if (!h->tile_exec || h->tile_exec_key[0] != mode || h->tile_exec_key[1] != grid ||
      h->tile_exec_key[2] != (int32_t)smem) {
    if (h->tile_exec) cudaGraphExecDestroy(h->tile_exec);
    h->tile_exec = nullptr;
    cudaStream_t cs;
    CUDA_OK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaMemsetAsync(h->d_queue, 0, sizeof(int32_t), cs);
      launch_tile(h, mode, grid, smem, cs);
      e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->tile_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      h->tile_exec = nullptr;
      return ISING_ERR_CUDA;
    }
    h->tile_exec_key[0] = mode;
    h->tile_exec_key[1] = grid;
    h->tile_exec_key[2] = (int32_t)smem;
  }
  kt_begin(h, "tile_kernel", s);
  CUDA_OK(cudaGraphLaunch(h->tile_exec, s));
  kt_end(h, s);
  h->launches += 1;
  return ISING_OK;
}

// ---------------------------------------------------------------- tuning cache
// Decisions are keyed by the GPU name and an instance class (dtype, instance
// count, largest instance, lattice / multi-spin eligibility, replicas,
// schedule).  With ISING_TUNE_CACHE=<file> they persist across processes as
// lines of a small JSON object: {"key": family, ...}.
std::string tune_key(const ising_handle *h, int32_t R, const ising_search_params *p) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, h->device);
  char buf[512];
  snprintf(buf, sizeof buf, "%s|dt%d|b%d|n%d|lat%d|msc%d|dense%d|R%d|sched%d|refresh%d", prop.name, h->dtype,
           h->n_inst, h->nmax, h->all_lattice ? 1 : 0, h->msc_ok ? 1 : 0, h->dense ? 1 : 0, R, (int)p->schedule,
           p->refresh_every);
  return buf;
}

std::map<std::string, int32_t> read_tune_file(const char *path) {
  std::map<std::string, int32_t> m;
  FILE *f = path ? fopen(path, "r") : nullptr;
  if (!f) return m;
  char line[1024];
  while (fgets(line, sizeof line, f)) {
    char *a = strchr(line, '"');
    if (!a) continue;
    char *b = strchr(a + 1, '"');
    if (!b) continue;
    char *c = strchr(b, ':');
    if (!c) continue;
    m[std::string(a + 1, b)] = (int32_t)strtol(c + 1, nullptr, 10);
  }
  fclose(f);
  return m;
}

int32_t tune_cache_lookup(const std::string &key) {
  const char *path = getenv("ISING_TUNE_CACHE");
  if (!path) return -1;
  auto m = read_tune_file(path);
  auto it = m.find(key);
  return it == m.end() ? -1 : it->second;
}

void tune_cache_store(const std::string &key, int32_t fam) {
  const char *path = getenv("ISING_TUNE_CACHE");
  if (!path) return;
  auto m = read_tune_file(path);
  m[key] = fam;
  FILE *f = fopen(path, "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t i = 0;
  for (auto &kv : m) fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++i < m.size() ? "," : "");
  fprintf(f, "}\n");
  fclose(f);
}

}  // namespace

namespace isg {

// An NVTX range for the duration of a C-ABI call (visible to profilers that
// record NVTX; a no-op otherwise).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

void kt_begin(ising_handle *h, const char *name, cudaStream_t s) {
  if (!h->timing) return;
  if (h->kt_used == h->ktimers.size()) {
    ising_handle::KTimer t{name, nullptr, nullptr};
    if (cudaEventCreate(&t.a) != cudaSuccess) return;
    if (cudaEventCreate(&t.b) != cudaSuccess) {
      cudaEventDestroy(t.a);
      return;
    }
    h->ktimers.push_back(t);
  }
  h->ktimers[h->kt_used].name = name;
  cudaEventRecord(h->ktimers[h->kt_used].a, s);
}

void kt_end(ising_handle *h, cudaStream_t s) {
  if (!h->timing || h->kt_used == h->ktimers.size()) return;  // (begin could not create its events)
  cudaEventRecord(h->ktimers[h->kt_used].b, s);
  ++h->kt_used;
}

}  // namespace isg

extern "C" {

ising_status ising_create(const ising_instance_desc *descs, int32_t n_instances, ising_handle **out) {
  const NvtxRange nvtx_range("ising_create");
  g_alloc_countdown = 0;
  if (fault_is("alloc")) {
    const char *f = std::getenv("ISING_FAULT");
    g_alloc_countdown = f[5] == ':' ? std::max(1, std::atoi(f + 6)) : 1;
  }
  if (!out) return ISING_ERR_INVALID_ARG;
  *out = nullptr;
  if (!descs || n_instances < 1) return ISING_ERR_INVALID_ARG;
  const ising_dtype dtype = descs[0].dtype;
  if (dtype != ISING_I8 && dtype != ISING_F32 && dtype != ISING_F64) return ISING_ERR_INVALID_ARG;
  const bool fl = dtype == ISING_F32, f64 = dtype == ISING_F64;
  std::vector<HostInst> hin(n_instances);
  bool dense = true, msc = dtype == ISING_I8, hyper = false;
  int64_t absb = 0;
  for (int32_t b = 0; b < n_instances; ++b) {
    ising_status st = load_desc(descs[b], dtype, hin[b]);
    if (st != ISING_OK) return st;
    const HostInst &I = hin[b];
    dense = dense && descs[b].J_dense != nullptr;
    hyper = hyper || I.hptr.size() > 1;
    if (dtype == ISING_I8) {
      for (int8_t w : I.Ji) {
        if (w != 1 && w != -1) msc = false;
        absb += std::abs((int)w);
      }
      absb /= 1;  // each pair appears twice; bound kept conservative
      for (int8_t v : I.hi) {
        if (v < -1 || v > 1) msc = false;
        absb += std::abs((int)v);
      }
      for (int8_t v : I.hJi) absb += std::abs((int)v);
      if (I.hptr.size() > 1 || I.max_deg > 15) msc = false;
    }
  }
  ising_handle *h = new ising_handle();
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  h->n_inst = n_instances;
  h->dtype = dtype;
  h->dense = dense && !hyper;  // hyper-edges on a dense instance: the CSR paths take it
  h->msc_ok = msc;
  h->has_hyper = hyper;
  h->abs_energy_bound = absb;

  // concatenate
  std::vector<InstDesc> inst(n_instances);
  std::vector<uint32_t> row;
  std::vector<int32_t> col, order, cls;
  std::vector<int8_t> Ji, hi, hJi;
  std::vector<float> Jf, hf, hJf;
  std::vector<double> Jd, hd, hJd;
  std::vector<uint32_t> inc_ptr, hptr;
  std::vector<int32_t> inc_edge, hmem;
  std::vector<int2> inc_oth;  // per incidence: the other two members of a 3-member edge
  std::vector<std::pair<int32_t, std::vector<int32_t>>> lat_sites;
  int64_t spin_off = 0, nnz_off = 0, edge_off = 0, mem_off = 0, cls_off = 0;
  for (int32_t b = 0; b < n_instances; ++b) {
    const HostInst &I = hin[b];
    InstDesc &D = inst[b];
    D.n = I.n;
    D.ncls = I.ncls;
    D.spin_off = spin_off;
    D.cls_off = cls_off;
    D.hyper_off = edge_off;
    D.n_hyper = (int32_t)I.hptr.size() - 1;
    D.max_deg = I.max_deg;
    D.lat_L = I.lat_L;
    D.lat_d = I.lat_d;
    int32_t emax = -1;
    D.ebase = fl ? energy_base_exponent(I, &emax) : -1;
    D.fx53 = f64 ? 0 : fp64_exact(I, fl, D.ebase);  // FP64 instances: the FP64 forms only
    D.ebits = f64 ? -1 : (!fl ? 7 : (D.ebase >= 0 ? 24 + std::max(0, emax - D.ebase) : -1));
    h->any_lattice = h->any_lattice || I.lat_d > 0;
    h->all_lattice = (b == 0 ? true : h->all_lattice) && I.lat_d > 0;
    h->nmax = std::max(h->nmax, I.n);
    for (int32_t i = 0; i < I.n; ++i) row.push_back((uint32_t)(nnz_off + I.row[i]));
    col.insert(col.end(), I.col.begin(), I.col.end());
    if (fl) {
      Jf.insert(Jf.end(), I.Jf.begin(), I.Jf.end());
      hf.insert(hf.end(), I.hf.begin(), I.hf.end());
      hJf.insert(hJf.end(), I.hJf.begin(), I.hJf.end());
    } else if (f64) {
      Jd.insert(Jd.end(), I.Jd.begin(), I.Jd.end());
      hd.insert(hd.end(), I.hd.begin(), I.hd.end());
      hJd.insert(hJd.end(), I.hJd.begin(), I.hJd.end());
    } else {
      Ji.insert(Ji.end(), I.Ji.begin(), I.Ji.end());
      hi.insert(hi.end(), I.hi.begin(), I.hi.end());
      hJi.insert(hJi.end(), I.hJi.begin(), I.hJi.end());
    }
    // incidence of hyper-edges per spin, ascending edge id
    std::vector<std::vector<int32_t>> inc(I.n);
    for (int32_t e = 0; e < D.n_hyper; ++e)
      for (int64_t q = I.hptr[e]; q < I.hptr[e + 1]; ++q) inc[I.hmem[q]].push_back(e);
    for (int32_t i = 0; i < I.n; ++i) {
      inc_ptr.push_back((uint32_t)inc_edge.size());
      for (int32_t e : inc[i]) {
        inc_edge.push_back((int32_t)(edge_off + e));
        int2 o = make_int2(-1, -1);
        if (I.hptr[e + 1] - I.hptr[e] == 3) {
          int32_t m[2], k = 0;
          for (int64_t q = I.hptr[e]; q < I.hptr[e + 1]; ++q)
            if (I.hmem[q] != i && k < 2) m[k++] = I.hmem[q];
          if (k == 2) o = make_int2(m[0], m[1]);
        }
        inc_oth.push_back(o);
      }
    }
    for (int32_t e = 0; e < D.n_hyper; ++e) hptr.push_back((uint32_t)(mem_off + I.hptr[e]));
    hmem.insert(hmem.end(), I.hmem.begin(), I.hmem.end());
    // colour classes: spins sorted by (colour, index)
    std::vector<int32_t> cnt(I.ncls + 1, 0);
    for (int32_t c : I.colour) cnt[c + 1]++;
    for (int32_t c = 0; c < I.ncls; ++c) cnt[c + 1] += cnt[c];
    cls.insert(cls.end(), cnt.begin(), cnt.end());
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1), ord(I.n);
    for (int32_t i = 0; i < I.n; ++i) ord[fill[I.colour[i]]++] = i;
    order.insert(order.end(), ord.begin(), ord.end());
    if (I.lat_d > 0) lat_sites.push_back({b, ord});
    spin_off += I.n;
    nnz_off += I.row[I.n];
    edge_off += D.n_hyper;
    mem_off += (int64_t)I.hmem.size();
    cls_off += I.ncls + 1;
  }
  if (nnz_off >= 0xffffffffLL || mem_off >= 0xffffffffLL || (int64_t)inc_edge.size() >= 0xffffffffLL) {
    delete h;
    return ISING_ERR_UNSUPPORTED;
  }
  row.push_back((uint32_t)nnz_off);
  inc_ptr.push_back((uint32_t)inc_edge.size());
  hptr.push_back((uint32_t)mem_off);
  std::vector<int16_t> runit;
  if (fl) {
    // per-spin refresh unit: the same test as the kernels' xr_exact, once here
    runit.assign(spin_off, 0);
    for (int64_t gi = 0; gi < spin_off; ++gi) {
      int emin = 256, emax = -1, k = 0;
      auto see = [&](float v) {
        uint32_t bits;
        std::memcpy(&bits, &v, 4);
        bits &= 0x7fffffffu;
        ++k;
        if (bits) {
          const int e = (int)(bits >> 23);
          emin = std::min(emin, e);
          emax = std::max(emax, e);
        }
      };
      see(hf.empty() ? 0.0f : hf[gi]);
      for (uint32_t kk = row[gi]; kk < row[gi + 1]; ++kk) see(Jf[kk]);
      for (uint32_t q = inc_ptr[gi]; q < inc_ptr[gi + 1]; ++q) see(hJf[inc_edge[q]]);
      int lg = 0;
      while (lg < 31 && (1u << lg) <= (uint32_t)k) ++lg;  // 2^lg > k
      const bool ex = emax < 0 || (emin >= 24 && emax <= 200 && (emax - emin) + 24 + lg <= 53);
      runit[gi] = (int16_t)(emax < 0 ? 24 : (ex ? emin : -1));
    }
    // InstDesc::fx53 = 2: fields exact in FP64 spin by spin (every spin has a
    // refresh unit), though not the energy as one integer sum
    for (int32_t b = 0; b < n_instances; ++b) {
      InstDesc &D = inst[b];
      if (D.fx53) continue;
      bool all = true;
      for (int64_t gi = D.spin_off; gi < D.spin_off + D.n && all; ++gi) all = runit[gi] >= 0;
      if (all) D.fx53 = 2;
    }
  }
  h->inst = inst;
  h->h_cls = cls;
  h->total_spins = spin_off;
  h->total_nnz = nnz_off;
  h->total_edges = edge_off;
  h->total_members = mem_off;

  bool ok = upload(&h->d_inst, inst) == cudaSuccess && upload(&h->d_row, row) == cudaSuccess &&
            upload(&h->d_col, col) == cudaSuccess && upload(&h->d_inc_ptr, inc_ptr) == cudaSuccess &&
            upload(&h->d_inc_edge, inc_edge) == cudaSuccess && upload(&h->d_inc_oth, inc_oth) == cudaSuccess &&
            upload(&h->d_hptr, hptr) == cudaSuccess &&
            upload(&h->d_hmem, hmem) == cudaSuccess && upload(&h->d_order, order) == cudaSuccess &&
            upload(&h->d_cls, cls) == cudaSuccess;
  if (ok) {
    if (fl) {
      ok = upload((float **)&h->d_J, Jf) == cudaSuccess && upload((float **)&h->d_h, hf) == cudaSuccess &&
           upload((float **)&h->d_hJ, hJf) == cudaSuccess;
      ok = ok && upload(&h->d_runit, runit) == cudaSuccess;
    } else if (f64) {
      ok = upload((double **)&h->d_J, Jd) == cudaSuccess && upload((double **)&h->d_h, hd) == cudaSuccess &&
           upload((double **)&h->d_hJ, hJd) == cudaSuccess;
    } else {
      ok = upload((int8_t **)&h->d_J, Ji) == cudaSuccess && upload((int8_t **)&h->d_h, hi) == cudaSuccess &&
           upload((int8_t **)&h->d_hJ, hJi) == cudaSuccess;
    }
  }
  if (ok && h->any_lattice) {
    // lattice metadata in colour order (see DevGraph::meta)
    const int64_t nsp = spin_off;
    std::vector<uint32_t> meta(nsp, 0);
    std::vector<uint16_t> latinfo(nsp, 0);
    std::vector<float> Jpf(fl ? 6 * nsp : 0, 0.0f);
    std::vector<int8_t> Jpi(fl ? 0 : 6 * nsp, 0);
    std::vector<float> Jff(fl ? 3 * nsp : 0, 0.0f);
    std::vector<int8_t> Jfi(fl ? 0 : 3 * nsp, 0);
    h->lat_parity = h->all_lattice;
    for (auto &ls : lat_sites) {
      const HostInst &I = hin[ls.first];
      const InstDesc &D = inst[ls.first];
      if (I.lat_d == 0) continue;
      const int32_t L = I.lat_L;
      if (D.ncls != 2) h->lat_parity = false;
      for (int32_t v = 0; v < I.n; ++v) {
        const int32_t j = ls.second[v];
        if (h->lat_parity) {
          int par = 0;
          for (int32_t a = 0, r = j; a < I.lat_d; ++a, r /= L) par += r % L;
          const int c = v < h->h_cls[D.cls_off + 1] - h->h_cls[D.cls_off] ? 0 : 1;
          if ((par & 1) != c) h->lat_parity = false;
        }
        uint32_t m = 0;
        int kk = 0;
        for (int64_t k = I.row[j]; k < I.row[j + 1]; ++k, ++kk) {
          const int32_t t = I.col[k];
          int64_t stride = 1;
          int dir = -1, wrap = 0;
          for (int a = 0; a < I.lat_d; ++a, stride *= L) {
            const int32_t c = (int32_t)((j / stride) % L);
            if (t == j + (((c + 1) % L) - c) * stride) { dir = 2 * a; wrap = (c == L - 1); break; }
            if (t == j + (((c + L - 1) % L) - c) * stride) { dir = 2 * a + 1; wrap = (c == 0); break; }
          }
          m |= (uint32_t)wrap << kk;
          m |= (uint32_t)dir << (8 + 3 * kk);
          const double w = fl ? (double)I.Jf[k] : (double)I.Ji[k];
          if (w < 0) m |= 1u << (26 + kk);
          latinfo[D.spin_off + v] |= (uint16_t)((wrap << dir) | ((w < 0 ? 1 : 0) << (8 + dir)));
          if (fl) Jpf[(int64_t)kk * nsp + D.spin_off + v] = I.Jf[k];
          else Jpi[(int64_t)kk * nsp + D.spin_off + v] = I.Ji[k];
          if (!(dir & 1)) {  // the bond to the +a neighbour, by site
            if (fl) Jff[(int64_t)(dir >> 1) * nsp + D.spin_off + j] = I.Jf[k];
            else Jfi[(int64_t)(dir >> 1) * nsp + D.spin_off + j] = I.Ji[k];
          }
        }
        meta[D.spin_off + v] = m;
      }
    }
    ok = upload(&h->d_meta, meta) == cudaSuccess && upload(&h->d_latinfo, latinfo) == cudaSuccess &&
         (fl ? upload((float **)&h->d_Jpos, Jpf) : upload((int8_t **)&h->d_Jpos, Jpi)) == cudaSuccess &&
         (fl ? upload((float **)&h->d_Jfwd, Jff) : upload((int8_t **)&h->d_Jfwd, Jfi)) == cudaSuccess;
  }
  if (ok && dense) {
    std::vector<float> Jd;
    for (int32_t b = 0; b < n_instances; ++b)
      Jd.insert(Jd.end(), descs[b].J_dense, descs[b].J_dense + (int64_t)descs[b].n * descs[b].n);
    ok = upload(&h->d_Jdense, Jd) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&h->d_tile_args, sizeof(TileArgs)) == cudaSuccess &&
       cudaMalloc(&h->d_seeds, sizeof(uint64_t) * n_instances) == cudaSuccess &&
       cudaMalloc(&h->d_stats, sizeof(unsigned long long) * 8) == cudaSuccess &&
       cudaMalloc(&h->d_queue, sizeof(int32_t) * 4) == cudaSuccess &&
       cudaMallocHost(&h->h_stats_pinned, sizeof(unsigned long long) * 8) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_handle(h);
    return ISING_ERR_OOM;
  }
  *out = h;
  return ISING_OK;
}

ising_status ising_energy(ising_handle *h, const int8_t *spins_dev, int32_t replicas, double *energy_dev,
                          int32_t *energy_i32_dev, cudaStream_t stream) {
  const NvtxRange nvtx_range("ising_energy");
  if (!h || !spins_dev || !energy_dev || replicas < 1) return ISING_ERR_INVALID_ARG;
  if (h->latched != ISING_OK) {
    ising_status l = h->latched;
    h->latched = ISING_OK;
    return l;
  }
  if (energy_i32_dev && (h->dtype != ISING_I8 || h->abs_energy_bound > 0x7fffffffLL))
    return ISING_ERR_UNSUPPORTED;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  cudaError_t e = launch_energy(h, spins_dev, replicas, energy_dev, energy_i32_dev, stream);
  if (cur != h->device) cudaSetDevice(cur);
  return e == cudaSuccess ? ISING_OK : ISING_ERR_CUDA;
}

int32_t ising_plan_kernel(ising_handle *h, int32_t replicas, const ising_search_params *p) {
  if (!h || replicas < 1) return -(int32_t)ISING_ERR_INVALID_ARG;
  ising_status st = validate_params(p);
  if (st != ISING_OK) return -(int32_t)st;
  return resolve_kernel(h, replicas, p);
}

ising_status ising_local_search(ising_handle *h, const uint64_t *seeds, int32_t replicas,
                                const ising_search_params *p, int8_t *spins_dev, double *energy_dev,
                                int32_t *energy_i32_dev, int32_t *minima_dev, ising_stats *stats,
                                cudaStream_t stream) {
  const NvtxRange nvtx_range("ising_local_search");
  if (!h || !seeds || replicas < 1 || !spins_dev || !energy_dev) return ISING_ERR_INVALID_ARG;
  ising_status st = validate_params(p);
  if (st != ISING_OK) return st;
  if (h->latched != ISING_OK) {
    ising_status l = h->latched;
    h->latched = ISING_OK;
    return l;
  }
  if (energy_i32_dev && (h->dtype != ISING_I8 || h->abs_energy_bound > 0x7fffffffLL))
    return ISING_ERR_UNSUPPORTED;
  if ((int64_t)replicas * h->total_spins > (int64_t)1 << 40) return ISING_ERR_UNSUPPORTED;
  const int32_t kernel = resolve_kernel(h, replicas, p);
  if (kernel < 0) return (ising_status)(-kernel);
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  st = ISING_OK;
  h->launches = 0;
  do {
    if (cudaMemcpyAsync(h->d_seeds, seeds, sizeof(uint64_t) * h->n_inst, cudaMemcpyHostToDevice, stream) !=
            cudaSuccess ||
        cudaMemsetAsync(h->d_stats, 0, sizeof(unsigned long long) * 8, stream) != cudaSuccess) {
      st = ISING_ERR_CUDA;
      break;
    }
    if (fault_is("launch")) {  // injected: as if the family's launch had failed
      st = ISING_ERR_CUDA;
      break;
    }
    switch (kernel) {
      case ISING_KERNEL_TILE:
        st = run_tile(h, h->dtype == ISING_F32 ? 1 : 0, replicas, p, spins_dev, energy_dev, energy_i32_dev,
                      minima_dev, stream);
        break;
      case ISING_KERNEL_MSC:
        st = run_tile(h, (h->all_lattice && p->schedule == ISING_SCHED_COLOUR) ? 3 : 2, replicas, p, spins_dev,
                      energy_dev, energy_i32_dev, minima_dev, stream);
        break;
      case ISING_KERNEL_SWEEP:
        if (launch_sweep(h, p, replicas, spins_dev, energy_dev, energy_i32_dev, minima_dev, seeds, stream) !=
            cudaSuccess)
          st = ISING_ERR_CUDA;
        break;
      case ISING_KERNEL_DENSE_TC: {
        const cudaError_t e = launch_dense(h, p, replicas, spins_dev, energy_dev, energy_i32_dev, minima_dev, seeds,
                                           stream);
        if (e == cudaErrorLaunchTimeout) st = ISING_ERR_TIMEOUT;  // a bounded device wait gave up
        else if (e != cudaSuccess) st = ISING_ERR_CUDA;
        break;
      }
      case ISING_KERNEL_PLAIN:
        kt_begin(h, "plain_path", stream);
        if (launch_plain(h, p, replicas, spins_dev, energy_dev, energy_i32_dev, minima_dev, seeds, stream) !=
            cudaSuccess)
          st = ISING_ERR_CUDA;
        kt_end(h, stream);
        break;
      default:
        st = ISING_ERR_UNSUPPORTED;
        break;
    }
  } while (0);
  if (st == ISING_OK && stats) {
    if (cudaMemcpyAsync(h->h_stats_pinned, h->d_stats, sizeof(unsigned long long) * 6, cudaMemcpyDeviceToHost,
                        stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
      st = ISING_ERR_CUDA;
    } else {
      stats->flip_evals = h->h_stats_pinned[0];
      stats->flips = h->h_stats_pinned[1];
      stats->minima = h->h_stats_pinned[2];
      stats->descents = h->h_stats_pinned[3];
      stats->sweeps = h->h_stats_pinned[4];
      stats->launches = h->launches;
      // the families that skip visits count the evaluated ones; the others
      // compute every gain they visit
      const bool skips = kernel == ISING_KERNEL_TILE || kernel == ISING_KERNEL_MSC || kernel == ISING_KERNEL_SWEEP;
      stats->evaluated = skips ? h->h_stats_pinned[5] : h->h_stats_pinned[0];
    }
  }
  if (cur != h->device) cudaSetDevice(cur);
  return st;
}

ising_status ising_autotune(ising_handle *h, int32_t replicas, const ising_search_params *p, int32_t *chosen,
                            cudaStream_t stream) {
  const NvtxRange nvtx_range("ising_autotune");
  if (!h || !p || replicas < 1) return ISING_ERR_INVALID_ARG;
  ising_status st = validate_params(p);
  if (st != ISING_OK) return st;
  const std::string key = tune_key(h, replicas, p);
  // a cached decision for this GPU and instance class?
  int32_t cached = tune_cache_lookup(key);
  if (cached > 0) {
    ising_search_params q = *p;
    q.kernel = (ising_kernel)cached;
    if (resolve_kernel(h, replicas, &q) == cached) {
      h->tuned[replicas] = cached;
      if (chosen) *chosen = cached;
      return ISING_OK;
    }
  }
  // time every eligible family on this handle with these parameters
  const int32_t families[] = {ISING_KERNEL_MSC, ISING_KERNEL_TILE, ISING_KERNEL_SWEEP, ISING_KERNEL_DENSE_TC};
  int8_t *spins = nullptr;
  double *E = nullptr;
  int32_t *mins = nullptr;
  if (cudaMalloc(&spins, (size_t)replicas * h->total_spins) != cudaSuccess ||
      cudaMalloc(&E, sizeof(double) * replicas * h->n_inst) != cudaSuccess ||
      cudaMalloc(&mins, sizeof(int32_t) * replicas * h->n_inst) != cudaSuccess) {
    cudaFree(spins);
    cudaFree(E);
    cudaFree(mins);
    return ISING_ERR_OOM;
  }
  std::vector<uint64_t> seeds(h->n_inst);
  for (int32_t b = 0; b < h->n_inst; ++b) seeds[b] = 0x9E3779B97F4A7C15ull * (uint64_t)(b + 1);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int32_t best_k = -1;
  float best_ms = 0.0f;
  h->tuned.erase(replicas);
  for (int32_t fam : families) {
    ising_search_params q = *p;
    q.kernel = (ising_kernel)fam;
    if (resolve_kernel(h, replicas, &q) != fam) continue;
    ising_stats s1;
    if (ising_local_search(h, seeds.data(), replicas, &q, spins, E, nullptr, mins, &s1, stream) != ISING_OK) continue;
    cudaEventRecord(e0, stream);
    ising_status r = ising_local_search(h, seeds.data(), replicas, &q, spins, E, nullptr, mins, nullptr, stream);
    cudaEventRecord(e1, stream);
    if (r != ISING_OK || cudaEventSynchronize(e1) != cudaSuccess) continue;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best_k < 0 || ms < best_ms) {
      best_k = fam;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(spins);
  cudaFree(E);
  cudaFree(mins);
  if (best_k < 0) return ISING_ERR_UNSUPPORTED;
  h->tuned[replicas] = best_k;
  tune_cache_store(key, best_k);
  if (chosen) *chosen = best_k;
  return ISING_OK;
}

ising_status ising_destroy(ising_handle *h) {
  free_handle(h);
  return ISING_OK;
}

ising_status ising_fm_search(ising_handle *h, const uint64_t *seeds, int32_t replicas, const ising_fm_params *p,
                             int8_t *spins_dev, double *energy_dev, int32_t *passes_dev, ising_stats *stats,
                             cudaStream_t stream) {
  const NvtxRange nvtx_range("ising_fm_search");
  if (!h || !seeds || !p || replicas < 1 || p->restarts < 1 || p->max_passes < 0 || p->starts < 0 ||
      p->starts > 2 || p->reg_kernel < -1 || p->reg_kernel > 1 || !spins_dev || !energy_dev)
    return ISING_ERR_INVALID_ARG;
  if (h->latched != ISING_OK) {
    ising_status l = h->latched;
    h->latched = ISING_OK;
    return l;
  }
  if (h->nmax > fm_max_spins()) return ISING_ERR_UNSUPPORTED;
  if ((int64_t)replicas * h->n_inst > 0x7fffffffLL) return ISING_ERR_UNSUPPORTED;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  ising_status st = ISING_OK;
  h->launches = 0;
  if (fault_is("launch")) {
    st = ISING_ERR_CUDA;
  } else if (cudaMemcpyAsync(h->d_seeds, seeds, sizeof(uint64_t) * h->n_inst, cudaMemcpyHostToDevice, stream) !=
                 cudaSuccess ||
             cudaMemsetAsync(h->d_stats, 0, sizeof(unsigned long long) * 8, stream) != cudaSuccess) {
    st = ISING_ERR_CUDA;
  } else {
    kt_begin(h, "fm_kernel", stream);
    if (launch_fm(h, replicas, p, spins_dev, energy_dev, passes_dev, stream) != cudaSuccess)
      st = ISING_ERR_CUDA;
    kt_end(h, stream);
  }
  if (st == ISING_OK && stats) {
    if (cudaMemcpyAsync(h->h_stats_pinned, h->d_stats, sizeof(unsigned long long) * 5, cudaMemcpyDeviceToHost,
                        stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
      st = ISING_ERR_CUDA;
    } else {
      stats->flip_evals = h->h_stats_pinned[0];
      stats->flips = h->h_stats_pinned[1];
      stats->minima = h->h_stats_pinned[2];
      stats->descents = h->h_stats_pinned[3];
      stats->sweeps = h->h_stats_pinned[4];
      stats->launches = h->launches;
      stats->evaluated = h->h_stats_pinned[0];
    }
  }
  if (cur != h->device) cudaSetDevice(cur);
  return st;
}

ising_status ising_set_timing(ising_handle *h, int32_t enable) {
  if (!h) return ISING_ERR_INVALID_ARG;
  if (enable && h->kt_used && cudaEventSynchronize(h->ktimers[h->kt_used - 1].b) != cudaSuccess)
    return ISING_ERR_CUDA;
  h->timing = enable != 0;
  if (enable) h->kt_used = 0;
  return ISING_OK;
}

int32_t ising_kernel_times(ising_handle *h, ising_kernel_time *out, int32_t cap) {
  if (!h || cap < 0 || (cap > 0 && !out)) return -(int32_t)ISING_ERR_INVALID_ARG;
  std::vector<ising_kernel_time> acc;
  for (size_t i = 0; i < h->kt_used; ++i) {
    const auto &t = h->ktimers[i];
    float ms = 0.0f;
    if (cudaEventSynchronize(t.b) != cudaSuccess || cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess)
      return -(int32_t)ISING_ERR_CUDA;
    size_t k = 0;
    while (k < acc.size() && std::strcmp(acc[k].name, t.name) != 0) ++k;
    if (k == acc.size()) acc.push_back(ising_kernel_time{t.name, 0.0, 0});
    acc[k].ms += (double)ms;
    acc[k].launches += 1;
  }
  for (size_t k = 0; k < acc.size() && (int32_t)k < cap; ++k) out[k] = acc[k];
  return (int32_t)acc.size();
}

const char *ising_status_string(ising_status s) {
  switch (s) {
    case ISING_OK: return "ok";
    case ISING_ERR_INVALID_ARG: return "invalid argument";
    case ISING_ERR_ASYMMETRIC: return "coupling matrix is not symmetric";
    case ISING_ERR_SELF_LOOP: return "coupling matrix has a self loop";
    case ISING_ERR_BAD_HYPEREDGE: return "malformed hyper-edge";
    case ISING_ERR_BAD_COLOURING: return "colouring is not proper for the conflict graph";
    case ISING_ERR_UNSUPPORTED: return "unsupported instance/kernel combination";
    case ISING_ERR_OOM: return "out of memory";
    case ISING_ERR_CUDA: return "CUDA runtime error";
    case ISING_ERR_TIMEOUT: return "device-side wait timed out";
    case ISING_ERR_DEVICE: return "device-side check failed";
  }
  return "unknown status";
}

}  // extern "C"
