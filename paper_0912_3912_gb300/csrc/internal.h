// internal.h — device-side instance layout, kernel argument blocks and the
// handle shared by the host API and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "ising.h"

namespace isg {

constexpr int kTileThreads = 256;   // threads per tile CTA (8 warps)
constexpr int kSweepThreads = 256;  // threads per CTA of the large-instance sweeps

// One instance as the kernels see it.  Spin, edge and class arrays of all
// instances are concatenated; these are each instance's offsets into them.
struct InstDesc {
  int32_t n;          // spins
  int32_t ncls;       // colour classes
  int64_t spin_off;   // first spin (global index) = offset into h, order, row
  int64_t cls_off;    // offset into the class-pointer array (ncls + 1 entries)
  int64_t hyper_off;  // first hyper-edge (global id)
  int32_t n_hyper;    // hyper-edges of this instance
  int32_t max_deg;    // largest CSR row length
  int32_t lat_L;      // side of a recognised periodic hypercubic lattice, else 0
  int32_t lat_d;      // its dimension (2 or 3), else 0
  // FP32 couplings: biased exponent of the smallest nonzero |J|, |h|, |J_e|
  // when the energy can be summed exactly in 64-bit fixed point with that
  // unit (see xe_term), else -1 (FP64 sums instead)
  int32_t ebase;
  // Exactness of FP64 arithmetic on the instance's fields, gains and energies:
  // 1 = every such value is an integer multiple of one unit (2^(ebase - 150)
  //     for FP32 couplings, 1 for int8) below 2^53 in magnitude;
  // 2 = (FP32) each spin's field values are multiples of that spin's refresh
  //     unit (DevGraph::runit) below 2^53 units; energies are not covered;
  // 0 = neither.
  int32_t fx53;
  // Bits of the largest energy term in fixed-point units: |term| < 2^ebits
  // (int8: 7; FP32 with ebase >= 0: 24 + emax - ebase; else -1).
  int32_t ebits;
};

// Everything a kernel needs to read an instance set.
struct DevGraph {
  const InstDesc *inst;
  const uint32_t *row;      // [total_spins + 1] global offsets into col/J
  const int32_t *col;       // local neighbour index
  const void *J;            // int8_t or float
  const void *h;            // [total_spins] int8_t or float (zeros when absent)
  const uint32_t *inc_ptr;  // [total_spins + 1] offsets into inc_edge
  const int32_t *inc_edge;  // global hyper-edge ids containing the spin, ascending
  const int2 *inc_oth;      // per incidence: the edge's two other members (local) when it
                            // has exactly three, else (-1, -1)
  const uint32_t *hptr;     // [total_edges + 1] offsets into hmem
  const int32_t *hmem;      // local member indices
  const void *hJ;           // [total_edges] int8_t or float
  const int32_t *order;     // [total_spins] local spins sorted by (colour, index)
  const int32_t *cls;       // class pointers per instance (ncls + 1 each)
  // Periodic lattices, per colour-order position v (global index spin_off + v):
  //   meta bits 0-5   entry k of the site's CSR row wraps around the boundary
  //        bits 8-25  direction of entry k (3 bits each: 0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z)
  //        bits 26-31 entry k has a negative coupling
  //   Jpos[k * nsp + spin_off + v] = coupling of entry k (int8_t or float)
  const uint32_t *meta;
  const void *Jpos;
  //   latinfo[spin_off + v]: bit d = the neighbour in direction d (0 +x, 1 -x,
  //   2 +y, 3 -y, 4 +z, 5 -z) wraps around; bit 8 + d = its coupling is negative
  const uint16_t *latinfo;
  //   Jfwd[a * nsp + spin_off + j]: coupling (int8_t or float) of the bond from
  //   site j to its +a neighbour (a = 0 x, 1 y, 2 z; wrapping), by site index:
  //   the lattice's bonds once each
  const void *Jfwd;
  // FP32 instances: per spin, the unit (smallest biased exponent) of an exact
  // fixed-point refresh, or -1 when that spin's refresh needs FP64 (see xr_exact)
  const int16_t *runit;
  int64_t nsp;              // total spins (stride of Jpos)
  int32_t dtype;            // ISING_I8 / ISING_F32
};

// Per-call arguments of the tile kernels (kept in device memory so that a
// captured graph can be replayed with new outputs and seeds).
struct TileArgs {
  DevGraph g;
  const int2 *tiles;        // (instance, 32-replica group), largest instances first
  int32_t n_tiles;
  int32_t *queue;           // work-queue counter, zeroed before each launch
  int32_t R, max_sweeps, restarts, budget, refresh, sequential;
  const uint64_t *seeds;    // [n_inst]
  float *F;                 // [grid][nmax][32] FP32 fields (float lane path)
  int32_t fsm_cap;          // instances up to this size keep their fields in shared memory
  uint32_t *bw;             // [grid][nmax] best-state words
  int32_t nmax;
  int8_t *spins;            // out [inst][replica][spin]
  double *energy;           // out [inst][replica]
  int32_t *energy_i32;      // out or null
  int32_t *minima;          // out or null
  unsigned long long *stats;  // [5] accumulated work counters
};

// Per-handle state of one launcher family (device buffers, graphs, streams
// kept across calls).  The handle owns one per family that has run on it; the
// family's *_free function releases its resources at ising_destroy.
struct FamilyState {
  virtual ~FamilyState() = default;
};

struct PlanKey {
  int32_t R, kernel, schedule;
  bool operator<(const PlanKey &o) const {
    return std::tie(R, kernel, schedule) < std::tie(o.R, o.kernel, o.schedule);
  }
};

}  // namespace isg

struct ising_handle {
  int device = 0;
  int sm_count = 0;
  int32_t n_inst = 0;
  int32_t dtype = 0;
  bool dense = false;       // instances given as dense matrices
  bool msc_ok = false;      // every coupling +/-1, every field in {-1,0,+1}, no hyper-edges
  bool has_hyper = false;
  int32_t nmax = 0;
  int64_t total_spins = 0, total_nnz = 0, total_edges = 0, total_members = 0;
  int64_t abs_energy_bound = 0;  // sum |J| + |h| + |J_e| (integer instances)
  std::vector<isg::InstDesc> inst;
  std::vector<int32_t> h_cls;  // host copy of the class pointers

  // device copies
  isg::InstDesc *d_inst = nullptr;
  uint32_t *d_row = nullptr;
  int32_t *d_col = nullptr;
  void *d_J = nullptr;
  void *d_h = nullptr;
  uint32_t *d_inc_ptr = nullptr;
  int32_t *d_inc_edge = nullptr;
  int2 *d_inc_oth = nullptr;
  uint32_t *d_hptr = nullptr;
  int32_t *d_hmem = nullptr;
  void *d_hJ = nullptr;
  int32_t *d_order = nullptr;
  int32_t *d_cls = nullptr;
  float *d_Jdense = nullptr;
  uint32_t *d_meta = nullptr;
  uint16_t *d_latinfo = nullptr;
  int16_t *d_runit = nullptr;
  bool all_lattice = false;  // every instance is a recognised periodic lattice
  bool lat_parity = false;   // ... coloured by site parity: class c = {x + y + z = c mod 2}
  void *d_Jpos = nullptr;
  void *d_Jfwd = nullptr;
  bool any_lattice = false;

  // scratch and per-call state, grown on demand
  void *d_scratch = nullptr;
  size_t scratch_bytes = 0;
  isg::TileArgs *d_tile_args = nullptr;
  uint64_t *d_seeds = nullptr;
  unsigned long long *d_stats = nullptr;
  int32_t *d_queue = nullptr;
  int2 *d_tiles = nullptr;
  int32_t tiles_R = -1;
  int32_t n_tiles = 0;
  unsigned long long *h_stats_pinned = nullptr;
  // energy work list (per replica count) and partial sums
  int32_t en_R = -1, en_nwork = 0;
  int4 *d_en_work = nullptr;
  int32_t *d_en_first = nullptr;
  double *d_en_partd = nullptr;
  long long *d_en_parti = nullptr;

  // tuned kernel family per replica count (autotuner cache)
  std::map<int32_t, int32_t> tuned;
  // the tile path's launch sequence (queue reset + persistent kernel) captured
  // once per (mode, grid, shared memory) and replayed
  cudaGraphExec_t tile_exec = nullptr;
  int32_t tile_exec_key[3] = {-1, -1, -1};
  ising_status latched = ISING_OK;
  uint64_t launches = 0;  // kernel launches enqueued by the current call
  // Optional device timing (ising_set_timing): CUDA events recorded on the
  // call's stream around each main kernel launch (or graph of launches).
  struct KTimer {
    const char *name;
    cudaEvent_t a, b;
  };
  bool timing = false;
  std::vector<KTimer> ktimers;
  size_t kt_used = 0;
  // launcher state, created by each family's first call on this handle
  std::unique_ptr<isg::FamilyState> dense_st, fm_st, plain_st, sweep_st;
  isg::DevGraph graph() const;
};

namespace isg {
// The launcher state of type T held in `slot` of a handle, created on first
// use.  Calls on one handle do not overlap (the ABI's rule), so no lock is
// needed; different handles share nothing.
template <typename T>
T &family_state(std::unique_ptr<FamilyState> &slot) {
  if (!slot) slot.reset(new T());
  return static_cast<T &>(*slot);
}
// device timing around a launch (no-ops unless timing is on); name: a static string
void kt_begin(ising_handle *h, const char *name, cudaStream_t s);
void kt_end(ising_handle *h, cudaStream_t s);
// launchers (tile.cu / energy.cu / plain.cu / sweep.cu / dense.cu)
cudaError_t launch_tile(ising_handle *h, int mode, int grid, size_t smem, cudaStream_t s);
size_t tile_smem_bytes(int mode, int nmax);
int tile_fsm_cap(int nmax, size_t budget);
int tile_max_ctas_per_sm(int mode, size_t smem);
cudaError_t launch_energy(ising_handle *h, const int8_t *spins, int32_t R, double *E,
                          int32_t *E32, cudaStream_t s);
void energy_plan_free(ising_handle *h);
size_t msc_cluster_smem(int csz);
cudaError_t launch_msc_cluster(ising_handle *h, int n_tiles, int P, int csz_max, int D, cudaStream_t s);
// the pass-based search (fm.cu)
int fm_max_spins();
cudaError_t launch_fm(ising_handle *h, int32_t R, const ising_fm_params *p, int8_t *spins, double *E,
                      int32_t *passes, cudaStream_t s);
void fm_free(ising_handle *h);
int msc_cluster_max_active(ising_handle *h, int n_tiles, int P, int csz_max, int D);
}  // namespace isg
