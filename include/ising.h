/*
 * ising.h — C ABI of the GB300 local-search library for Ising spin glasses.
 *
 * Method: García & Markov, "High-performance Energy Minimization in Spin-glasses
 * with Applications to Adiabatic Quantum Computing" (arXiv:0912.3912).
 *   - Energy with pair couplings and fields: Sec. II, Eq. 1.
 *   - Energy with k-spin hyper-couplings: Sec. VI, Eq. 6.
 *   - Gain of a single-spin move, random starts, passes, restarts: Sec. IV
 *     (Fig. 3 and the text around it).
 *   - Incremental ("efficient") gain updates after a move: Sec. IV.
 *
 * The library runs single-spin-flip descent to a 1-flip local minimum, with
 * counter-based random restarts, over many replicas of many instances at once,
 * on one GPU.  Every buffer argument is a plain pointer; nothing here depends on
 * PyTorch.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  Spins are +1/-1.  An instance has n spins, a symmetric CSR coupling graph
 *  (J_ij = J_ji, no self loops, no repeated column in a row), optional fields h_i,
 *  and optional hyper-edges e (>= 2 distinct members) with strengths J_e.
 *
 *  Energy (Eq. 1 extended by Eq. 6), each unordered pair counted once:
 *      E(s) = - sum_{i<j, (i,j) in CSR} J_ij s_i s_j
 *             - sum_e J_e prod_{k in e} s_k  -  sum_i h_i s_i
 *  Local field of spin i:
 *      f_i = h_i + sum_j J_ij s_j + sum_{e contains i} J_e prod_{k in e, k != i} s_k
 *  Flipping spin i changes the energy by dE_i = 2 s_i f_i; the paper's gain is
 *  -dE_i (positive gain = lower energy).  A descent flips a spin iff dE_i < 0.
 *
 *  Threads: calls on different handles may run concurrently on different host
 *  threads; calls on one handle must not overlap.
 *
 *  Schedules.  A sweep visits every spin once.
 *   - ISING_SCHED_COLOUR: colour classes c = 0..C-1 in ascending order; all
 *     spins of a class decide against the same state, then flip together.  A
 *     class is an independent set of the conflict graph (CSR edges plus every
 *     pair inside one hyper-edge), so this equals visiting the class's spins
 *     one after another in any order.
 *   - ISING_SCHED_SEQUENTIAL: spins 0..n-1 in index order, each deciding on
 *     the current state (the paper's one-move-at-a-time order).
 *
 *  Descent and restarts (per replica r of instance b):
 *   descent k = 0,1,... starts from the random configuration R(b, r, k) below
 *   and sweeps until a sweep makes no flip (converged: a 1-flip local minimum)
 *   or max_sweeps sweeps were made (capped).  The replica runs `restarts`
 *   descents, or stops earlier when its total sweep count reaches
 *   sweep_budget (> 0).  Its result is the lowest-energy final state among its
 *   converged descents, the earliest one on ties; if none converged, the final
 *   state of its last descent.
 *
 *  Random starts R(b, r, k) (Sec. IV: uniform random configuration): Philox4x32-10
 *  (Salmon, Moraes, Dror, Shaw, SC'11) with key = (low 32 bits of seeds[b],
 *  high 32 bits of seeds[b]) and counter = (w, r, k, b).  Spin i of the start is
 *  +1 iff bit (i mod 128) of the 128-bit output for w = i / 128 is 1, where bit t
 *  of the output is bit (t mod 32) of output word t / 32.
 *
 *  Floating-point couplings (ISING_F32).  Local fields are kept in FP32 and
 *  updated incrementally: at each visit of spin j, for every CSR neighbour i
 *  (in j's row order) that flipped since j's previous visit, f_j += 2 J_ji s_i;
 *  then for every hyper-edge e containing j (in ascending edge order) in which an
 *  odd number of the other members flipped since that visit,
 *  f_j += 2 J_e prod_{k in e, k != j} s_k (FP32 additions, round to nearest).
 *  At descent sweeps d with d % refresh_every == 0 (and always at d == 0) the
 *  visit instead recomputes f_j from scratch in FP64, in the same order, and
 *  rounds it to FP32.  The flip decision is s_j * f_j < 0 in FP32.  Energies
 *  are computed from scratch in FP64.  Integer couplings (ISING_I8) use exact
 *  int32 fields and energies.
 *
 *  Layouts.  Spin outputs and inputs are int8 (+1/-1), ordered
 *  [instance][replica][spin]; instance b's block starts at
 *  replicas * (n_0 + ... + n_{b-1}).  Energies are [instance][replica].
 *
 *  Ownership.  The caller owns every buffer passed in.  ising_create copies the
 *  instances to the device; the handle owns those copies, the colourings, the
 *  work plans and the scratch memory it allocates.  Device-pointer arguments
 *  must be allocated on the device that was current at ising_create.  Calls are
 *  ordered on the stream passed in (NULL = the legacy default stream).
 *
 *  Errors.  Argument and instance errors are returned synchronously and leave
 *  no partial state (a failed ising_create returns no handle).  A device-side
 *  check that fails (for instance a wait that gave up) is latched in the
 *  handle and returned by the next call on it.
 */
#ifndef ISING_GB300_H
#define ISING_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cudaStream_t;

typedef enum {
  ISING_OK = 0,
  ISING_ERR_INVALID_ARG = 1,   /* NULL where a pointer is required, sizes out of range  */
  ISING_ERR_ASYMMETRIC = 2,    /* CSR not symmetric (structure or values)               */
  ISING_ERR_SELF_LOOP = 3,     /* CSR row i lists column i                              */
  ISING_ERR_BAD_HYPEREDGE = 4, /* < 2 members, repeated member, member out of range     */
  ISING_ERR_BAD_COLOURING = 5, /* colour out of range or two conflicting spins share it */
  ISING_ERR_UNSUPPORTED = 6,   /* instance/kernel combination this build cannot run     */
  ISING_ERR_OOM = 7,           /* device or host allocation failed                      */
  ISING_ERR_CUDA = 8,          /* a CUDA runtime call failed                            */
  ISING_ERR_TIMEOUT = 9,       /* a device-side bounded wait ran out                    */
  ISING_ERR_DEVICE = 10        /* a device-side consistency check failed                */
} ising_status;

/* Value type of an instance's couplings, fields and hyper-edge strengths.
 * ISING_F64 instances (wide coefficients, e.g. the factoring instances of
 * Sec. VI) run the pass-based search, plain descent (kernel family PLAIN)
 * and ising_energy; every field, gain and energy is the FP64 value of the
 * sequential definition: fields h, the CSR row in stored order, then the
 * hyper-edges ascending, recomputed at every visit in descent; energies as a
 * compensated (Neumaier) FP64 sum of the terms in the order pairs of row i
 * (j > i, stored order) and field i for i = 0..n-1, then the hyper-edges.
 * Other families return ISING_ERR_UNSUPPORTED for them.                     */
typedef enum { ISING_I8 = 0, ISING_F32 = 1, ISING_F64 = 2 } ising_dtype;

typedef enum { ISING_SCHED_COLOUR = 0, ISING_SCHED_SEQUENTIAL = 1 } ising_schedule;

/* Kernel families.  AUTO lets the planner (and its tuning cache) choose. */
typedef enum {
  ISING_KERNEL_AUTO = 0,
  ISING_KERNEL_TILE = 1,     /* one CTA per (instance, 32-replica group), lane = replica,
                                persistent work queue over all tiles                    */
  ISING_KERNEL_MSC = 2,      /* multi-spin coded tile: 32 replicas as bits of a word;
                                needs J in {-1,+1}, h in {-1,0,+1}, no hyper-edges      */
  ISING_KERNEL_SWEEP = 3,    /* large instances: one launch per colour class over the
                                whole GPU; chunks of sweeps captured once in a CUDA
                                graph and replayed until every replica is done          */
  ISING_KERNEL_DENSE_TC = 4, /* dense couplings (J_dense, no hyper-edges), sequential
                                schedule: a descent's first sweeps with block fields as
                                a tcgen05 GEMM (BF16 hi+lo), the rest as per-replica
                                incremental gain updates (any dense instance: at most
                                16384 spins).  Decisions can differ from the FP64
                                definition only for fields within ~1e-5 of zero          */
  ISING_KERNEL_PLAIN = 5     /* plain comparator: one launch per instance and colour
                                class, one thread per (spin, replica), the same field
                                semantics, no bit packing, no skipping, no graph        */
} ising_kernel;

/* One instance.  All pointers are HOST pointers; they are read during
 * ising_create only.  J, h and hyper_J hold int8_t for ISING_I8, float for
 * ISING_F32 and double for ISING_F64.  Exactly one of (row_ptr, col, J) and
 * J_dense (ISING_F32 only) is given.                                           */
typedef struct {
  int32_t n;                    /* number of spins, >= 1                            */
  const int64_t *row_ptr;       /* [n+1], row_ptr[0] = 0, non-decreasing            */
  const int32_t *col;           /* [row_ptr[n]] neighbour indices                   */
  const void *J;                /* [row_ptr[n]] couplings, symmetric                */
  const float *J_dense;         /* [n*n] row-major, symmetric, zero diagonal
                                   (ISING_F32 only); NULL for CSR instances          */
  const void *h;                /* [n] fields, or NULL for h = 0                    */
  int32_t n_hyper;              /* number of hyper-edges, >= 0                      */
  const int64_t *hyper_ptr;     /* [n_hyper+1] offsets into hyper_members           */
  const int32_t *hyper_members; /* members of each hyper-edge                       */
  const void *hyper_J;          /* [n_hyper] strengths J_e                          */
  const int32_t *colour;        /* [n] colour class per spin, or NULL: the library
                                   colours the conflict graph greedily in index
                                   order (smallest colour unused by earlier
                                   conflicting spins)                               */
  ising_dtype dtype;
} ising_instance_desc;

/* Variant of the dense family (ISING_KERNEL_DENSE_TC). */
typedef enum {
  ISING_DENSE_OWN = 0,     /* the library's own kernels (n <= 4096)                  */
  ISING_DENSE_LIBRARY = 1  /* comparator: 128-spin block decisions with the block
                              fields from cuBLAS BF16 GEMMs (hi+lo), any n            */
} ising_dense_variant;

/* Search parameters.  The last three fields choose between implementations of
 * one family; none changes what a search computes beyond the rounding noted
 * for the dense family.  Zero-initialised, they take the library's defaults.   */
typedef struct {
  int32_t max_sweeps;    /* >= 1, cap on sweeps per descent                          */
  int32_t restarts;      /* >= 1, descents per replica                               */
  int32_t sweep_budget;  /* 0 = no budget; else total sweeps per replica             */
  int32_t refresh_every; /* ISING_F32: FP64 field refresh period in descent sweeps;
                            0 = only at the first sweep of a descent                 */
  ising_schedule schedule;
  ising_kernel kernel;
  int32_t dense_variant;       /* ising_dense_variant (dense family only)            */
  int32_t dense_tensor_sweeps; /* ISING_DENSE_OWN: sweeps of each descent decided on
                                  tensor cores before the per-replica continuation;
                                  0 = default (3), < 0 = none (identical results
                                  up to the dense family's rounding)                 */
  int32_t cluster_ctas;        /* multi-spin-coded periodic lattices: CTAs per
                                  cluster; 0 = automatic, 1 = no clusters, 2/4/8 =
                                  only that size where eligible, else none (same
                                  results either way)                                */
} ising_search_params;

/* Work counters of one ising_local_search call, summed over all replicas:
 * flip_evals = spins visited (one gain computed and decided per visit),
 * flips = accepted moves, minima = converged descents, descents = descents run,
 * sweeps = sweeps run.  They depend only on the method's semantics, not on the
 * kernel that ran it.  launches = this library's kernel launches the call
 * enqueued (kernel nodes of replayed graphs included; library GEMMs not).
 * evaluated = (spin, replica) visits whose gain the kernels actually computed:
 * families TILE, MSC and SWEEP skip a visit when no neighbour of the spin (and
 * no member of its hyper-edges) flipped since its previous visit, because its
 * gain and its decision (no flip) are then unchanged (Sec. IV, incremental gain
 * updates); the count depends on the kernel and its work layout, and equals
 * flip_evals for the families that never skip.
 * When stats is non-NULL the call waits for the search to finish.              */
typedef struct {
  uint64_t flip_evals, flips, minima, descents, sweeps, launches, evaluated;
} ising_stats;

typedef struct ising_handle ising_handle;

/* Validate and upload n_instances instances (all of one dtype).  An instance
 * is the paper's problem statement (Sec. II): spins s_i = +/-1 on the nodes of
 * a coupling graph with couplings J_ij and fields h_i, whose energy is Eq. 1,
 * extended by the k-spin hyper-couplings J_e of Eq. 6 (Sec. VI).  Checks:
 * sizes and pointers (ISING_ERR_INVALID_ARG, also for non-finite FP32 values),
 * J_ij = J_ji with matching structure (ISING_ERR_ASYMMETRIC), no self loop
 * (ISING_ERR_SELF_LOOP), hyper-edges of >= 2 distinct in-range members
 * (ISING_ERR_BAD_HYPEREDGE), a given colouring valid for the conflict graph
 * (ISING_ERR_BAD_COLOURING).  On success *out owns device copies (the host
 * arrays may be freed); on failure *out is NULL and nothing stays allocated.  */
ising_status ising_create(const ising_instance_desc *descs, int32_t n_instances,
                          ising_handle **out);

/* Energies (Eq. 1 / Eq. 6) of caller-supplied configurations.
 * spins_dev: device int8 +/-1, [instance][replica][spin] with `replicas`
 * replicas per instance.  energy_dev: device double [instance][replica]
 * (required).  energy_i32_dev: device int32 [instance][replica] or NULL;
 * ISING_I8 handles only.                                                       */
ising_status ising_energy(ising_handle *h, const int8_t *spins_dev, int32_t replicas,
                          double *energy_dev, int32_t *energy_i32_dev, cudaStream_t stream);

/* Descent with restarts for `replicas` replicas of every instance.
 * seeds: HOST uint64 [n_instances].  spins_dev: device int8 out,
 * [instance][replica][spin].  energy_dev: device double out [instance][replica].
 * energy_i32_dev, minima_dev (device int32 [instance][replica], converged
 * descents per replica) may be NULL.  stats (host) may be NULL; when given, the
 * call waits for the stream to finish and fills it.                           */
ising_status ising_local_search(ising_handle *h, const uint64_t *seeds, int32_t replicas,
                                const ising_search_params *p, int8_t *spins_dev,
                                double *energy_dev, int32_t *energy_i32_dev,
                                int32_t *minima_dev, ising_stats *stats,
                                cudaStream_t stream);

/* The kernel family the planner would use for these arguments (after
 * resolving ISING_KERNEL_AUTO), or a negative ising_status on invalid input.   */
int32_t ising_plan_kernel(ising_handle *h, int32_t replicas, const ising_search_params *p);

/* Time every eligible kernel family on this handle (on `stream`, synchronising
 * it) and record the fastest per instance class in the tuning cache; later
 * ISING_KERNEL_AUTO calls use it.  Writes the chosen family to *chosen.        */
ising_status ising_autotune(ising_handle *h, int32_t replicas, const ising_search_params *p,
                            int32_t *chosen, cudaStream_t stream);

/* Allocation-free energy evaluation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory - for example a
 * framework whose pool allocator owns the whole device, or code that must not
 * trigger the device-wide synchronisation a cudaMalloc implies - and so can
 * use neither ising_create nor ising_energy's on-demand scratch.  It returns
 * the same energies as ising_energy for instances with pair couplings and
 * fields only (no hyper-edges): minus the sum over each coupled pair, counted
 * once, of J_ij s_i s_j, minus the sum of h_i s_i.  Inputs are the caller's own
 * DEVICE buffers: row_ptr_dev int64 [n+1], col_dev int32 and J_dev (int8_t or
 * float per dtype) [row_ptr[n]], a symmetric CSR as for ising_create that is
 * not re-validated here (all three required: an instance without couplings
 * still passes valid device pointers), h_dev [n] or NULL (no fields),
 * spins_dev int8 [replicas][n]; energy_dev double [replicas] out.  All buffers
 * and `stream` belong to the current device.  It allocates nothing: its
 * scratch is a fixed array of ISING_NOALLOC_MAX_PARTIALS doubles (512 KiB)
 * that every device loading the library holds until the process exits, so it
 * returns ISING_ERR_UNSUPPORTED when ceil(n / 4096) * replicas exceeds that
 * limit, and ISING_ERR_INVALID_ARG for a NULL required pointer or a size
 * below 1.  Outside stream capture every call looks up that array's address
 * on the current device, so a device reset or a recreated context does not
 * invalidate it; a call made while `stream` is capturing reuses the address
 * of the last uncaptured call on that device, so at least one uncaptured call
 * on the device (and none since a reset) must come before any capture, else
 * the call returns ISING_ERR_CUDA.  All calls share the array: calls that
 * overlap on the GPU race and must be ordered by the caller.                   */
#define ISING_NOALLOC_MAX_PARTIALS 65536
ising_status ising_energy_noalloc(int32_t n, const int64_t *row_ptr_dev, const int32_t *col_dev,
                                  const void *J_dev, const void *h_dev, ising_dtype dtype,
                                  const int8_t *spins_dev, int32_t replicas, double *energy_dev,
                                  cudaStream_t stream);

/* Parameters of the pass-based search. */
typedef struct {
  int32_t restarts;    /* >= 1, random starts per replica                          */
  int32_t max_passes;  /* >= 0, cap on passes per start; 0 = no cap                */
  int32_t starts;      /* 0 = automatic; 1 = a replica's starts one after another
                          in one warp; 2 = one start per warp, the best chosen
                          afterwards (same results either way)                    */
  int32_t reg_kernel;  /* instances of at most 512 spins in the one-unit integer
                          form: 0 = automatic (registers when the searches fit one
                          wave), 1 = always the register-resident kernel, -1 =
                          always the shared-memory kernel (same results)          */
} ising_fm_params;

/* The paper's pass-based search with hill climbing (Sec. IV, Fig. 3), for
 * instances of at most 4096 spins (else ISING_ERR_UNSUPPORTED).  Per replica,
 * p->restarts starts (Philox, counter layout as for ising_local_search, restart
 * index k = 0 .. p->restarts-1); from each start, passes: every spin moves once
 * per pass in best-gain order (largest -2 s_i f_i among the spins not yet
 * moved, ties to the lowest index; moves with negative gain included), the
 * pass is cut back to its earliest strictly lowest-energy prefix, and passes
 * repeat while one lowers the energy strictly (float couplings: by more than
 * 1e-9 (1 + |E|)); p->max_passes > 0 caps the passes per start (0: no cap).  Gains
 * and energies are the FP64 values of that definition (fields summed as h,
 * then the CSR row in stored order, then the hyper-edges ascending); where FP64
 * is exact on an instance the kernels compute them in integers, with the same
 * results.  Per replica the result is the lowest-energy start (ties keep the
 * earlier).  The work is ordered on `stream` (internal streams are forked from
 * it and joined back before the call's last launch).  The handle keeps its
 * scratch (item lists; with few replicas, every start's result, at most 1 GiB)
 * until ising_destroy.
 * spins_dev, energy_dev: as for ising_local_search; passes_dev: device int32
 * [instance][replica] passes summed over the starts, or NULL.  stats (nullable;
 * the call then waits): descents = starts, sweeps = passes, flips and
 * flip_evals = moves applied (n per pass), minima = 0.                        */
ising_status ising_fm_search(ising_handle *h, const uint64_t *seeds, int32_t replicas, const ising_fm_params *p,
                             int8_t *spins_dev, double *energy_dev, int32_t *passes_dev, ising_stats *stats,
                             cudaStream_t stream);

/* Device timing of the kernels a search runs, for measurement.
 * ising_set_timing(h, 1) opens a timing window (clearing the previous one);
 * while it is open every ising_local_search call records a pair of CUDA events
 * on its stream around each of its main kernel launches (a family's main
 * kernel, or a graph of them: "tile_kernel", "msc_cluster_kernel",
 * "sweep_chunk", "dense_tc_kernel", "dense_push_kernel", "dense_energy_tc",
 * "plain_path", "fm_kernel").  ising_set_timing(h, 0) stops recording.
 * ising_kernel_times waits for the recorded events and writes up to cap
 * entries {name, total ms, launches} summed over the window, in order of first
 * launch; it returns the number of distinct names (which may exceed cap), or
 * a negative ising_status.  name points to a static string of the library.    */
typedef struct {
  const char *name;
  double ms;
  int32_t launches;
} ising_kernel_time;
ising_status ising_set_timing(ising_handle *h, int32_t enable);
int32_t ising_kernel_times(ising_handle *h, ising_kernel_time *out, int32_t cap);

/* Measurement helper, not an operation of the method: the issue rate of 32-bit
 * three-input logic operations (lop3) on the calling thread's current GPU, in
 * lane-operations per second (one lane-op = one 32-bit logic op of one thread),
 * from a self-timed kernel of register-only logic chains at full occupancy
 * (best of three launches of about 10 ms).  This rate bounds the multi-spin-
 * coded kernels, whose gains are word-wide logic on 32 replicas at once.
 * *lane_ops_per_s (host) receives the rate, 0 on failure.  Blocks until done;
 * ISING_ERR_INVALID_ARG for NULL, ISING_ERR_CUDA on a CUDA error.           */
ising_status ising_logic_peak(double *lane_ops_per_s);

/* Measurement helper, not an operation of the method: replica-bit logic
 * operations per second on word_bits-wide words (32 or 64), from chains of
 * two-input XORs of that width (PTX xor.b32 / xor.b64) on registers at full
 * occupancy, counted as XORs x word_bits (one replica per bit, as in
 * multi-spin coding; best of three
 * launches of about 10 ms).  Compares the two word widths multi-spin coding
 * could use.  *bit_ops_per_s (host) receives the rate, 0 on failure.  Blocks
 * until done; ISING_ERR_INVALID_ARG for NULL or another width, ISING_ERR_CUDA
 * on a CUDA error.                                                           */
ising_status ising_logic_bits_rate(int32_t word_bits, double *bit_ops_per_s);

/* Free everything the handle owns.  ising_destroy(NULL) returns ISING_OK.      */
ising_status ising_destroy(ising_handle *h);

const char *ising_status_string(ising_status s);

#ifdef __cplusplus
}
#endif
#endif /* ISING_GB300_H */
