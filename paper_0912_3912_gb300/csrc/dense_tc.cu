// dense_tc.cu — the dense (Sherrington-Kirkpatrick) path on 5th-generation
// tensor cores, hand-written with tcgen05, TMA and thread-block clusters.
//
// Method: the paper's sequential single-spin descent (Sec. IV) on a complete
// graph, where every colour class is one spin.  Spins are decided in blocks of
// 128 consecutive indices.  The fields of a block for 128 replicas are
//     F[r][i] = sum_j S[r][j] J[i][j],   i in the block, j = 0..n-1,
// a GEMM with K = n, computed as S.J_hi^T + S.J_lo^T (J = J_hi + J_lo, both
// BF16; spins +/-1 exact in BF16) with FP32 accumulation in tensor memory.  The
// block's spins are then decided one after another, each field corrected in
// FP32 for the earlier flips inside the block (+2 J_ij s_j): the paper's
// incremental gain update restricted to the block.
//
// Work split: a cluster of 4 CTAs owns 128 replicas for the first sweeps of a
// round (one descent of every replica): the replicas start from their Philox
// states together and sweep in lockstep.  CTA q multiplies the K-slice
// j in [q n/4, (q+1) n/4) into its own tensor-memory accumulator; every CTA
// stores the rows of its partial block that belong to CTA q straight into CTA
// q's receive buffer (distributed shared memory), and CTA q sums the four in a
// fixed order and decides replicas 32q..32q+31.  The spin operand
// comes from tensor memory: CTA q keeps the spin bits of all 128 replicas over
// its K-slice in shared memory, and four warps expand each 64-spin chunk to
// BF16 +/-1 and store it to tensor memory (tcgen05.st), so that only the
// coupling tiles pass through shared memory (TMA loads, 128-byte swizzled
// K-major) and the MMAs read one shared-memory operand instead of two.
// Thread 0 of each CTA issues the loads and the MMAs through a 3-stage mbarrier
// pipeline.  The deciding warps read and write their replicas' bits of a block
// in the owning CTA's shared memory (distributed shared memory).  A last pass
// without decisions exports the full field vectors of the replicas still
// descending, which dense_push.cu continues one replica at a time: the first
// sweeps flip most spins (a GEMM per block is then cheap per flip), the later
// ones few, and their number varies widely between replicas.  Every mbarrier wait is bounded; a CTA whose wait gives up
// records ISING_ERR_TIMEOUT, keeps the cluster's barrier sequence and skips its
// remaining work, and the cluster ends together at the next sweep.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cfloat>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "dense.cuh"
#include "device_common.cuh"
#include "tc.cuh"

namespace isg {

namespace {

constexpr int kTM = 128;        // replicas per cluster (MMA M)
constexpr int kTB = 128;        // spins per block (MMA N)
constexpr int kKC = 64;         // K per TMA chunk (128 bytes of BF16)
constexpr int kClus = 4;        // CTAs per cluster (split K)
constexpr int kThreads = 1024;  // one warp per decided replica (32 per CTA)
constexpr int kFl = kTB + 1;    // padded row of the block fields [replica][spin]
constexpr int kTileBytes = kTB * kKC * 2;                 // 16 KB, one coupling tile
constexpr int kStages = 3;                                // operand pipeline depth
constexpr int kStageBytes = 2 * kTileBytes;               // B_hi, B_lo
constexpr int kRxBytes = kClus * kTB * 32 * 4;            // 64 KB, received partials [source][spin][replica]
constexpr int kJblkBytes = kTB * kTB * 4;                 // 64 KB, the block's couplings in FP32
constexpr int kFlocBytes = 32 * kFl * 4;                  // this CTA's replicas' block fields
constexpr int kAcc = kTB;                                 // tensor-memory columns of the accumulator
constexpr int kACols = kKC / 2;                           // columns of one spin chunk (two BF16 per column)
constexpr int kTmemCols = 256;                            // accumulator + kStages spin chunks
constexpr int kGen0 = 4;                                  // warps kGen0..kGen0+3 write the spin chunks
constexpr int kMaxN = 16384;
// Shared memory: the stages (once a block's MMAs have completed they hold its
// FP32 couplings until the next block's loads), the receive buffer (the
// decided replicas' summed fields replace the partials once read), the spin
// bits [n / 128 words][128 replicas] of the CTA's K-slice, alignment slack.
// The receive buffer lies outside the stages: other CTAs write into it while
// this CTA's MMAs may still read its stages.
constexpr int smem_bytes(int n) { return kStages * kStageBytes + kRxBytes + 4 * n + 1024; }
static_assert(kJblkBytes <= kStages * kStageBytes, "couplings must fit the stages");
static_assert(kFlocBytes <= kRxBytes, "fields must fit the receive buffer");
static_assert(smem_bytes(kMaxN) + 2048 <= 227 * 1024, "shared memory per CTA (2 KB for the static part)");
static_assert(kAcc + kStages * kACols <= kTmemCols, "tensor-memory columns");
static_assert(kGen0 >= 1 && kGen0 + 4 <= kThreads / 32, "spin-chunk warps: not warp 0 (thread 0 issues)");
static_assert(kThreads == kTB * 8 && kThreads > 512, "phase-3 and staging thread maps");

struct TcArgs {
  int32_t n, R, Rp, b;             // spins (padded to a multiple of 256), replicas, padded replicas, instance
  int32_t n_eval;                  // the instance's own spins (work counters)
  int32_t max_sweeps, budget;      // sweep cap per descent, sweep budget over descents (<= 0: none)
  int32_t sweeps_a;                // decision sweeps of a round on tensor cores before the export
  uint64_t seed;
  const float *J;                  // [n][n] FP32 (in-block corrections)
  const float *h;                  // [n] FP32 fields of the spins (zeros allowed)
  __nv_bfloat16 *S;                // [Rp][n] spins +/-1
  float *Fx;                       // [R][n] exported fields (h included) of replicas still descending
  DenseRep *rep;                   // [R] per-replica state, read at entry and written back
  unsigned long long *stats;
  int32_t *error;                  // set to ISING_ERR_TIMEOUT when a wait gives up
  int32_t stall_test;              // nonzero: CTA 0 waits, with a short limit, on a barrier nothing
                                   // completes (exercises the failure path in tests)
};

// Philox start R(b, r, k) of replica r, written as BF16 +/-1 into S[r][:];
// warp-cooperative, lane l handles the 128-spin blocks l, l + 32, ...
__device__ __forceinline__ void write_start_warp(const TcArgs &A, int r, int k, int lane) {
  __nv_bfloat16 *row = A.S + (size_t)r * A.n;
  for (int w = lane; w * 128 < A.n; w += 32) {
    const uint4 x = start_bits(A.seed, (uint32_t)w, (uint32_t)r, (uint32_t)k, (uint32_t)A.b);
    for (int t = 0; t < 128 && w * 128 + t < A.n; ++t)
      row[w * 128 + t] = __float2bfloat16_rn(((word_of(x, t / 32) >> (t % 32)) & 1u) ? 1.0f : -1.0f);
  }
}

// Spins 2c and 2c + 1 of a 32-spin word (bit = 1: +1) as two BF16 +/-1 in one
// 32-bit tensor-memory column (the lower K index in the low half).
__device__ __forceinline__ uint32_t pm1_pair(uint32_t w, int c) {
  return 0xBF80BF80u ^ (((w >> (2 * c)) & 1u) << 15) ^ (((w >> (2 * c + 1)) & 1u) << 31);
}

// Bounded wait of the spin-chunk warps; gives up at once when thread 0 has
// failed (its MMAs, which complete the barrier, will not come).
__device__ __forceinline__ bool gen_wait(uint64_t *bar, uint32_t parity, const volatile int32_t *abort) {
  const uint64_t t0 = tc::global_ns();
  for (;;) {
    for (int it = 0; it < 64; ++it)
      if (tc::mbar_try_wait(bar, parity)) return true;
    if (*abort || tc::global_ns() - t0 > 1000000000ull) return false;
  }
}

// One round's first sweeps on tensor cores.  Every replica taking part starts
// its descent (restart k) from its Philox state and sweeps in lockstep with the
// cluster's other replicas for up to sweeps_a sweeps; a final pass then computes
// every block's fields once more without decisions, giving the energy of each
// replica's state and, for replicas still descending, their full field vectors
// (exported to Fx for the per-replica continuation).
__global__ void __cluster_dims__(kClus, 1, 1) __launch_bounds__(kThreads, 1)
    dense_tc_kernel(const __grid_constant__ CUtensorMap mapJhi, const __grid_constant__ CUtensorMap mapJlo, TcArgs A) {
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte alignment as an offset into the shared array, so that the
  // compiler keeps the shared address space of every pointer below
  uint8_t *smem = smem_raw + ((1024u - (tc::smem_addr(smem_raw) & 1023u)) & 1023u);
  uint8_t *stage = smem;                                              // kStages x (Bhi, Blo)
  float *Jblk = reinterpret_cast<float *>(smem);                      // in the stages: [128][128]
  float *Rx = reinterpret_cast<float *>(smem + kStages * kStageBytes);  // [source CTA][spin][replica]
  float *Floc = Rx;                                                   // after the sum: [32 replicas][kFl]
  // spin bits of the cluster's 128 replicas over this CTA's K-slice: word w
  // (spins kbase + 32 w .. + 31, bit t = spin kbase + 32 w + t, 1 = +1) of
  // replica r0 + row at kbits[w * 128 + row]
  uint32_t *kbits = reinterpret_cast<uint32_t *>(smem + kStages * kStageBytes + kRxBytes);

  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], afull_bar[kStages], done_bar, drain_bar,
      stall_bar;
  __shared__ volatile int32_t s_abort;  // thread 0 failed: the spin-chunk warps stop waiting
  __shared__ uint32_t tmem_base_s;
  __shared__ int32_t s_flag[2];   // cluster-visible: [0] my replicas still busy, [1] my failure
  __shared__ int32_t s_ctrl[4];   // broadcast inside the CTA
  __shared__ int32_t s_act[32], s_nfl[32], s_run[32];
  __shared__ double s_en[32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t q = tc::cluster_rank();
  const int tile = blockIdx.x / kClus;
  const int r0 = tile * kTM;                 // first replica of the cluster
  const int rq = r0 + 32 * (int)q;           // first replica this CTA decides
  const int n = A.n, nblk = n / kTB, kslice = n / kClus;
  const int kchunks = kslice / kKC, kbase = (int)q * kslice;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kTM, kTB);

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&empty_bar[s], 1);
      tc::mbar_init(&afull_bar[s], 4);  // one arrival per spin-chunk warp
    }
    tc::mbar_init(&done_bar, 1);
    tc::mbar_init(&drain_bar, 1);
    tc::mbar_init(&stall_bar, 1);
    tc::fence_barrier_init();
    tc::prefetch_tmap(&mapJhi);
    tc::prefetch_tmap(&mapJlo);
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base_s, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  // per-replica state: thread t of warp 0 owns replica rq + t
  const int my_r = rq + lane;
  const bool real = warp == 0 && my_r < A.R;
  // the fields of DenseRep this kernel changes (static shared memory is nearly
  // all taken by the stages, partials and spin bits)
  struct TcRep {
    int32_t active, conv, total, d, flips, round;
    double E;
  };
  __shared__ TcRep s_rep[32];  // warp 0, lane l: replica rq + l
  TcRep &st = s_rep[lane];
  if (warp == 0) {
    st.active = st.conv = st.total = st.d = st.flips = st.round = 0;
    st.E = 0.0;
    s_run[lane] = s_nfl[lane] = 0;
    if (real) {
      const DenseRep g = A.rep[my_r];
      st.active = g.active;
      st.conv = g.conv;
      st.total = g.total;
      st.d = g.d;
      st.round = g.round;
      st.E = g.E;
      s_run[lane] = g.round;
      s_nfl[lane] = g.k;
    }
  }
  unsigned long long c_evals = 0, c_flips = 0, c_sweeps = 0;
  __syncthreads();
  if (rq + warp < A.R && s_run[warp]) write_start_warp(A, rq + warp, s_nfl[warp], lane);
  // the start bits of every replica of the cluster taking part in the round,
  // over this CTA's K-slice (item e: replica r0 + e % 128, word e / 128; the
  // slice need not start on a 128-spin block)
  for (int e = tid; e < kTM * (kslice / 32); e += kThreads) {
    const int row = e & (kTM - 1), w = e / kTM, r = r0 + row, g = kbase / 32 + w;
    if (r < A.R && A.rep[r].round) {
      const uint4 x = start_bits(A.seed, (uint32_t)(g / 4), (uint32_t)r, (uint32_t)A.rep[r].k, (uint32_t)A.b);
      kbits[w * kTM + row] = word_of(x, g & 3);
    }
  }
  bool failed = false;
  uint32_t ph_full[kStages], ph_empty[kStages], ph_a[kStages], ph_done = 0;
  int tma_pending[kStages], mma_pending = 0;
#pragma unroll
  for (int st2 = 0; st2 < kStages; ++st2) ph_full[st2] = ph_empty[st2] = ph_a[st2] = 0, tma_pending[st2] = 0;
  uint32_t g_used = 0, g_ph = 0;  // spin-chunk warps: stages written before, parity of their next completion
  tc::cluster_sync();

  for (int sw = 0; sw <= A.sweeps_a; ++sw) {
    // ---- cluster-wide control: is anybody active?  did anybody fail?
    if (tid == 0) s_flag[0] = 0, s_flag[1] = failed ? 1 : 0;
    __syncthreads();
    if (warp == 0) {
      const int busy = __any_sync(0xffffffffu, st.active != 0);
      if (lane == 0) s_flag[0] = busy;
    }
    __syncthreads();
    tc::cluster_sync();
    if (tid == 0) {
      int busy = 0, bad = 0;
      for (uint32_t c = 0; c < kClus; ++c) {
        busy |= (int)tc::ld_cluster_u32(tc::map_shared(&s_flag[0], c));
        bad |= (int)tc::ld_cluster_u32(tc::map_shared(&s_flag[1], c));
      }
      s_ctrl[0] = busy;
      s_ctrl[1] = bad;
    }
    tc::cluster_sync();  // nobody rewrites s_flag before every CTA has read it
    const int any_busy = s_ctrl[0], any_bad = s_ctrl[1];
    if (any_bad) break;
    if (sw == 0 && !any_busy) break;  // no replica of the cluster takes part in this round
    // the export pass: fields and energies of the current states, no decisions
    const bool export_pass = !any_busy || sw == A.sweeps_a;
    double e_lane = 0.0;  // export pass: this lane's part of its warp's replica energy sum
    // ---- one sweep (or the export pass) over the blocks
    for (int blk = 0; blk < nblk; ++blk) {
      const int b0 = blk * kTB;
      // Phase 1: partial fields of the block over this CTA's K-slice.  Thread 0
      // keeps kStages chunks in flight: after issuing chunk kc's MMAs it refills
      // the stage of chunk kc-1 once those MMAs have read it, so the tensor pipe
      // always has the next chunk queued.  The spin-chunk warps write chunk kc's
      // spins to the tensor-memory columns of its stage once the MMAs of the
      // stage's previous chunk have completed.
      if (tid == 0 && !failed) {
        auto load = [&](int s, int kn) {
          uint8_t *st_ = stage + s * kStageBytes;
          tc::mbar_arrive_expect_tx(&full_bar[s], kStageBytes);
          tc::tma_load_2d(st_, &mapJhi, &full_bar[s], kbase + kn * kKC, b0);
          tc::tma_load_2d(st_ + kTileBytes, &mapJlo, &full_bar[s], kbase + kn * kKC, b0);
          tma_pending[s] = 1;
        };
        for (int s = 0; s < kStages && s < kchunks; ++s) load(s, s);
        if (A.stall_test && blockIdx.x == 0 && sw == 0 && blk == 0 && !tc::mbar_wait(&stall_bar, 0, 20000))
          failed = true;  // nothing arrives on stall_bar: the wait gives up after 20 us
        int waited = 0;  // chunks whose MMA completion (empty barrier) has been consumed
        for (int kc = 0; kc < kchunks && !failed; ++kc) {
          const int s = kc % kStages;
          if (!tc::mbar_wait(&full_bar[s], ph_full[s])) {
            failed = true;
            break;
          }
          ph_full[s] ^= 1u;
          tma_pending[s] = 0;
          if (!tc::mbar_wait(&afull_bar[s], ph_a[s])) {
            failed = true;
            break;
          }
          ph_a[s] ^= 1u;
          tc::tc_fence_after();
          uint8_t *st_ = stage + s * kStageBytes;
          const uint64_t dh = tc::smem_desc_k_sw128(st_);
          const uint64_t dl = tc::smem_desc_k_sw128(st_ + kTileBytes);
          const uint32_t ta = tmem + (uint32_t)(kAcc + s * kACols);
#pragma unroll
          for (int kk = 0; kk < kKC / 16; ++kk)
            tc::mma_bf16_ts(tmem, ta + 8 * kk, dh + 2 * kk, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
#pragma unroll
          for (int kk = 0; kk < kKC / 16; ++kk) tc::mma_bf16_ts(tmem, ta + 8 * kk, dl + 2 * kk, idesc, 1u);
          tc::mma_commit(&empty_bar[s]);
          mma_pending = 1;
          if (kc >= 1) {
            const int pc = kc - 1, sp = pc % kStages;
            if (!tc::mbar_wait(&empty_bar[sp], ph_empty[sp])) {
              failed = true;
              break;
            }
            ph_empty[sp] ^= 1u;
            waited = kc;
            if (pc + kStages < kchunks) load(sp, pc + kStages);
          }
        }
        if (!failed) {
          tc::mma_commit(&done_bar);
          // consume the MMA completions not waited for above
          for (int c = waited; c < kchunks && !failed; ++c) {
            const int sp = c % kStages;
            if (!tc::mbar_wait(&empty_bar[sp], ph_empty[sp])) failed = true;
            ph_empty[sp] ^= 1u;
          }
        }
        if (failed) s_abort = 1;
      } else if (warp >= kGen0 && warp < kGen0 + 4 && !failed) {
        // spin-chunk warp: tensor-memory lanes 32 lq .. + 31 = replicas r0 + 32 lq + lane
        const int lq = warp - kGen0, row = 32 * lq + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)kAcc;
        for (int kc = 0; kc < kchunks; ++kc) {
          const int s = kc % kStages;
          if ((g_used >> s) & 1u) {
            if (!gen_wait(&empty_bar[s], (g_ph >> s) & 1u, &s_abort)) {
              failed = true;
              break;
            }
            g_ph ^= 1u << s;
          }
          g_used |= 1u << s;
          const uint32_t w0 = kbits[(2 * kc) * kTM + row], w1 = kbits[(2 * kc + 1) * kTM + row];
          uint32_t v[32];
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            v[c] = pm1_pair(w0, c);
            v[16 + c] = pm1_pair(w1, c);
          }
          tc::tc_fence_after();
          tc::tmem_st32(trow + (uint32_t)(s * kACols), v);
          tc::tc_fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&afull_bar[s]);
        }
      }
      failed = __syncthreads_or(failed) != 0;
      // Phase 2: accumulator -> the deciding CTAs' receive buffers; meanwhile
      // the other warps stage the block's couplings in FP32 (the stages are free
      // once the MMAs have completed)
      {
        const bool ok = failed ? true : tc::mbar_wait(&done_bar, ph_done);
        failed = __syncthreads_or(failed || !ok) != 0;
        tc::tc_fence_after();
        if (tid == 0 && !failed) mma_pending = 0;
      }
      ph_done ^= 1u;
      if (!failed && warp < 16) {
        // warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its lane quarter:
        // replicas of CTA w % 4) and accumulator columns 32 (w / 4) .. + 31, and
        // stores them to slot q of that CTA's receive buffer
        const int lq = warp & 3, cc = warp >> 2;
        uint32_t v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(cc * 32), v);
        const uint32_t dst = tc::map_shared(Rx + ((int)q * kTB + cc * 32) * 32 + lane, (uint32_t)lq);
#pragma unroll
        for (int k = 0; k < 32; ++k) tc::st_cluster_u32(dst + 128u * k, v[k]);
      } else if (!failed && !export_pass) {
        for (int e = tid - 512; e < kTB * kTB / 4; e += kThreads - 512) {
          const int i = e / (kTB / 4), c4 = e % (kTB / 4);
          reinterpret_cast<float4 *>(Jblk)[e] =
              *reinterpret_cast<const float4 *>(A.J + (size_t)(b0 + i) * n + b0 + 4 * c4);
        }
      }
      tc::tc_fence_before();
      __syncthreads();
      tc::cluster_sync();  // every CTA's partials have arrived
      // Phase 3: sum the four partials (fixed order) and add h for this CTA's 32
      // replicas; the sums replace the partials in the receive buffer
      {
        const int i = tid >> 3, c4 = tid & 7;  // kThreads = kTB x 8
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!failed) {
          for (int c = 0; c < kClus; ++c) {
            const float4 p = *reinterpret_cast<const float4 *>(Rx + (c * kTB + i) * 32 + 4 * c4);
            acc.x += p.x;
            acc.y += p.y;
            acc.z += p.z;
            acc.w += p.w;
          }
          const float hv = __ldg(A.h + b0 + i);
          acc.x += hv;
          acc.y += hv;
          acc.z += hv;
          acc.w += hv;
        }
        __syncthreads();
        if (!failed) {
          Floc[(4 * c4 + 0) * kFl + i] = acc.x;
          Floc[(4 * c4 + 1) * kFl + i] = acc.y;
          Floc[(4 * c4 + 2) * kFl + i] = acc.z;
          Floc[(4 * c4 + 3) * kFl + i] = acc.w;
        }
      }
      // Phase 4: sequential decisions (or the export).  Warp w decides replica
      // rq + w; lane l keeps the fields of spins 32q + l (q = 0..3) in
      // registers.  Spins are decided in index order; between two flips no field
      // changes, so the warp ballots every current decision of a quarter and
      // jumps to the first flipping spin at or after the current one, flips it,
      // adds 2 J_ij s_j to the fields of the later spins (in flip order, the same
      // FP32 order as visiting them one by one) and continues after it.
      if (warp == 0) s_act[lane] = (my_r < A.R && !failed) ? st.active : 0;
      __syncthreads();
      {
        const int rr = rq + warp;
        const bool valid_r = rr < A.R && !failed;
        // word j of the block's bits of replica rr lives in the CTA whose K-slice
        // holds spins b0 + 32 j .. + 31 (a K-slice may end inside a block); lane
        // j < 4 fetches it
        const int gw = (b0 >> 5) + (lane & 3), qb = (32 * gw) / kslice;
        const uint32_t baddr = tc::map_shared(kbits + (gw - qb * (kslice >> 5)) * kTM + 32 * (int)q + warp, (uint32_t)qb);
        const uint32_t mine = (valid_r && lane < 4) ? tc::ld_cluster_u32(baddr) : 0u;
        uint32_t wq[4];  // the block's 128 spins of replica rr (1 = +1)
        float f[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          wq[qq] = __shfl_sync(0xffffffffu, mine, qq);
          f[qq] = valid_r ? Floc[warp * kFl + 32 * qq + lane] : 0.0f;
        }
        if (export_pass) {
          // E = -1/2 sum_i s_i (f_i + h_i), f including h: FP64 sums per lane over
          // the blocks (one warp reduction after the last block); FP64 issues
          // slowly, so a warp whose four h values are all zero adds s_i f_i
          // (exact in FP32) with one conversion and one FP64 add each
          float hq[4];
          bool hz = true;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            hq[qq] = __ldg(A.h + b0 + 32 * qq + lane);
            hz = hz && hq[qq] == 0.0f;
          }
          if (__all_sync(0xffffffffu, hz)) {
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) e_lane += (double)(((wq[qq] >> lane) & 1u) ? f[qq] : -f[qq]);
          } else {
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const double v = (double)f[qq] + (double)hq[qq];
              e_lane += ((wq[qq] >> lane) & 1u) ? v : -v;
            }
          }
          if (valid_r && s_act[warp]) {
            float *dst = A.Fx + (size_t)rr * n + b0;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) dst[32 * qq + lane] = f[qq];
          }
        } else {
          const bool act = valid_r && s_act[warp] != 0;
          const uint32_t w_old[4] = {wq[0], wq[1], wq[2], wq[3]};
          if (act) {
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              uint32_t from = 0xffffffffu;  // lanes not yet decided in this quarter
              for (;;) {
                // spin 32 qq + lane flips iff its field is nonzero with the sign
                // of the spin (+1 and f < 0, or -1 and f > 0): the field's sign
                // bit xor the spin bit is clear and the rest nonzero
                const int32_t t = (int32_t)(__float_as_uint(f[qq]) ^ (((wq[qq] >> lane) & 1u) << 31));
                const uint32_t m = __ballot_sync(0xffffffffu, t > 0) & from;
                if (!m) break;
                const int li = __ffs(m) - 1;
                const float c = ((wq[qq] >> li) & 1u) ? -2.0f : 2.0f;  // 2 s_i with the new spin
                wq[qq] ^= 1u << li;
                from = 0xfffffffeu << li;
                // J symmetric: row i = column i.  c J is exact, so one FMA rounds
                // like adding c J; later spins of this quarter, then the later quarters
                const float *Jrow = Jblk + (32 * qq + li) * kTB + lane;
                const float jq = Jrow[32 * qq];
                if (lane > li) f[qq] = __fmaf_rn(c, jq, f[qq]);
#pragma unroll
                for (int q2 = qq + 1; q2 < 4; ++q2) f[q2] = __fmaf_rn(c, Jrow[32 * q2], f[q2]);
              }
            }
          }
          uint32_t fl[4];
          int nfl = 0;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            fl[qq] = wq[qq] ^ w_old[qq];
            nfl += __popc(fl[qq]);
          }
          if (nfl) {
            if (lane < 4)
              tc::st_cluster_u32(baddr, lane == 0 ? wq[0] : lane == 1 ? wq[1] : lane == 2 ? wq[2] : wq[3]);
            __nv_bfloat16 *row = A.S + (size_t)rr * n + b0;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq)
              if ((fl[qq] >> lane) & 1u) row[32 * qq + lane] = __float2bfloat16_rn(((wq[qq] >> lane) & 1u) ? 1.0f : -1.0f);
          }
          if (lane == 0) s_nfl[warp] = act ? nfl : 0;
        }
      }
      __syncthreads();
      if (warp == 0 && my_r < A.R && !failed && !export_pass) {
        st.flips += s_nfl[lane];
        c_flips += (unsigned long long)s_nfl[lane];
      }
      // generic-proxy writes to the stages (the couplings) are ordered before
      // the next block's TMA writes
      tc::fence_proxy_async_shared();
      __syncthreads();
      tc::cluster_sync();  // new spin bits visible to every CTA's next block
    }
    // (a CTA that failed keeps the cluster's barrier sequence; the control step
    // of the next sweep ends the cluster together)
    if (export_pass) {
      const double e = warp_sum(e_lane);
      if (lane == 0) s_en[warp] = e;
      __syncthreads();
      if (real && st.round) st.E = -0.5 * s_en[lane];
      break;
    }
    // ---- end of sweep: per-replica bookkeeping (warp 0)
    if (real && st.active) {
      st.total += 1;
      st.d += 1;
      c_evals += (unsigned long long)A.n_eval;
      ++c_sweeps;
      const bool conv = st.flips == 0;
      st.flips = 0;
      if (conv || st.d >= A.max_sweeps || (A.budget > 0 && st.total >= A.budget)) {
        st.active = 0;
        st.conv = conv ? 1 : 0;
      }
    }
  }

  if (real) {
    DenseRep &g = A.rep[my_r];
    g.active = st.active;
    g.conv = st.conv;
    g.total = st.total;
    g.d = st.d;
    g.flips = 0;
    g.E = st.E;
    if (c_sweeps) {
      atomicAdd(A.stats + 0, c_evals);
      atomicAdd(A.stats + 1, c_flips);
      atomicAdd(A.stats + 4, c_sweeps);
    }
  }
  if (failed && tid == 0) {
    atomicExch(A.error, (int32_t)ISING_ERR_TIMEOUT);
    // let copies and MMAs still in flight land before the CTA releases its memory
    for (int s = 0; s < kStages; ++s)
      if (tma_pending[s]) tc::mbar_wait(&full_bar[s], ph_full[s]);
    if (mma_pending) {  // a barrier of its own: done_bar's phase may not match after a failure
      tc::mma_commit(&drain_bar);
      tc::mbar_wait(&drain_bar, 0);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

// ---------------------------------------------------------------- host side
// Any n up to kMaxN: smaller or ragged instances run zero-padded to a multiple
// of 256 (padded spins have no couplings and no field, so they never flip and
// add nothing to an energy).
bool dense_tc_eligible(int n) { return n >= 1 && n <= kMaxN; }
int dense_tc_padded(int n) { return (n + 255) / 256 * 256; }

// A 2-D BF16 tensor map (row-major, `inner` elements per row, `outer` rows)
// for TMA tile loads of box_inner x box_outer with 128-byte swizzling.
cudaError_t tc_encode_2d(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                         uint32_t box_outer) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {inner * 2};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// One round's tensor-core sweeps (see dense_tc_kernel).  n a multiple of 256
// (n_eval <= n the instance's own spins); S: [Rp][n] BF16 spins (Rp a multiple
// of 128), Jhi/Jlo [n][n] BF16, J [n][n] FP32, h [n] FP32, Fx [R][n] FP32
// exported fields, rep [R] per-replica state.
cudaError_t dense_tc_run(int n, int n_eval, int R, int Rp, int b, uint64_t seed, const float *J, const float *h,
                         const __nv_bfloat16 *Jhi, const __nv_bfloat16 *Jlo, __nv_bfloat16 *S, float *Fx,
                         DenseRep *rep, int sweeps_a, unsigned long long *stats, int32_t *error,
                         const ising_search_params *p, cudaStream_t s) {
  if (n % 256 != 0 || n > kMaxN || n_eval > n || Rp % kTM != 0) return cudaErrorInvalidValue;
  CUtensorMap mH, mL;
  cudaError_t e;
  if ((e = tc_encode_2d(&mH, Jhi, (uint64_t)n, (uint64_t)n, kKC, kTB)) != cudaSuccess) return e;
  if ((e = tc_encode_2d(&mL, Jlo, (uint64_t)n, (uint64_t)n, kKC, kTB)) != cudaSuccess) return e;
  TcArgs A;
  A.n = n;
  A.n_eval = n_eval;
  A.R = R;
  A.Rp = Rp;
  A.b = b;
  A.max_sweeps = p->max_sweeps;
  A.budget = p->sweep_budget;
  A.sweeps_a = sweeps_a;
  A.seed = seed;
  A.J = J;
  A.h = h;
  A.S = S;
  A.Fx = Fx;
  A.rep = rep;
  A.stats = stats;
  A.error = error;
  {
    const char *f = std::getenv("ISING_FAULT");
    A.stall_test = (f && std::strcmp(f, "device_timeout") == 0) ? 1 : 0;
  }
  const int grid = (Rp / kTM) * kClus;
  if ((e = cudaFuncSetAttribute(dense_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(kMaxN))) !=
      cudaSuccess)
    return e;
  dense_tc_kernel<<<grid, kThreads, smem_bytes(n), s>>>(mH, mL, A);
  return cudaGetLastError();
}

}  // namespace isg
