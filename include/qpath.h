/*
 * qpath.h -- C ABI of libqpath, a GB300 (sm_103a) many-replica Metropolis
 * annealer for the one-hot UAV path QUBO of "GPU-Accelerated Quantum
 * Annealing-Inspired UAV Path Planning for Smart Agriculture".
 *
 * The paper's pipeline (Algorithm 1) is: travel-cost matrix from the grid
 * (Section II) -> one-hot variables x_{t,i} -> H_visit + H_time (Eqs. 4, 5) ->
 * H_dist (Eq. 3) -> H_QUBO (Eq. 6) -> a GPU sampler -> the path read off the
 * best state.  This library is that pipeline with its own sampler:
 *   qp_build_qubo / qp_build_from_dense   the QUBO (Section II, Eqs. 3-6)
 *   qp_anneal / qp_anneal_ex / _batch     many independent Metropolis chains
 *                                         (the role of the paper's parallel
 *                                         annealing engine, Section IV-A)
 *   qp_decode_path / qp_decode_batch      the path reconstruction step of
 *                                         Algorithm 1
 *
 * Conventions shared by every call
 *   Variables.  k = t*C + i, t = step, i = cell id; C free cells numbered in
 *     row-major grid order; n = C*C.  The start cell s is clamped: x_{0,s} = 1,
 *     the rest of row 0 and of column s are 0 and never proposed.
 *   Energy.  E(x) = B*sum_{t<C-1} sum_{i,j} d_ij x_{t,i} x_{t+1,j}
 *                 + A*sum_i (1 - sum_t x_{t,i})^2 + A*sum_t (1 - sum_i x_{t,i})^2
 *     (Eqs. 3-6 with every penalty range over 0..C-1), an exact int64.  A
 *     multiplies the penalties (the paper's lambda_p), B the distance term.
 *   Distances.  d_ij = round(scale * sqrt(dr^2 + dc^2)) in exact integers.
 *   Random numbers.  Philox4x32-10, key (seed_lo, seed_hi), counter
 *     (k>>2, sweep, replica, 0x51505448); the draw of k is output word k&3.
 *   Schedule.  T_s = T0*(T1/T0)^(s/(n_sweeps-1)) (T0 if n_sweeps == 1).
 *     Proposal k in sweep s is accepted iff dE <= 0, or dE < len_s and
 *     u < floor(2^32 exp(-dE/T_s)); len_s is the first dE whose threshold is 0.
 *     Tables are built on the host in double precision, once per device and
 *     schedule, and cached (the least recently used dropped first beyond
 *     4 GiB of tables; a batch keeps its schedule's tables for its life).
 *   Sweeps.  Sweep s proposes every free k once, in increasing k.
 *   Best energy.  Minimum of E over the ends of the sweeps run at which every
 *     row and column sum is 1 (no test for a QUBO without path structure);
 *     INT64_MAX if there was none.
 *   Pointers.  Every buffer is owned by the caller and may be host or device
 *     memory (told apart with cudaPointerGetAttributes).  When every output of
 *     a call is device memory the call is asynchronous on `cuda_stream`
 *     (a cudaStream_t, NULL = legacy default stream); otherwise it returns
 *     after the results are in the caller's buffers.
 *   Errors.  Every call returns a status and never aborts; qp_last_error()
 *     gives a message for the calling thread.  Handles are not thread-safe:
 *     use one handle per host thread, or serialise calls on it; asynchronous
 *     calls on one handle must not overlap on the GPU either (different
 *     streams included), since they share the handle's device buffers.
 */
#ifndef QPATH_H
#define QPATH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QP_OK = 0,
  QP_EINVAL = 1,       /* bad argument                                     */
  QP_ENOMEM = 2,       /* host or device allocation failed                 */
  QP_ERANGE = 3,       /* a value does not fit the integer types used      */
  QP_ECUDA = 4,        /* a CUDA call failed                               */
  QP_ETIMEOUT = 5,     /* a bounded device wait gave up                    */
  QP_EINFEASIBLE = 6   /* decode: the state is not a one-hot permutation   */
} qp_status;

/* Every call that fails returns its status before launching any kernel on a
 * buffer it could not allocate, and leaves the handle usable.  Failure
 * injection for tests: with the environment variable QPATH_FAIL_ALLOC = N the
 * library's next N device allocations succeed and every later one fails
 * (QP_ENOMEM), until the variable changes or is removed. */

typedef struct qp_handle qp_handle;

/* A grid field (Section II).  free_mask[r*cols + c] = 1 marks a cell to
 * visit; NULL means every cell.  start is the grid index of the start cell and
 * must be free. */
typedef struct {
  int32_t rows, cols;
  const uint8_t *free_mask;
  int32_t start;
} qp_field;

/* Geometric schedule over n_sweeps sweeps; a call runs sweeps
 * [sweep_begin, sweep_end), which makes a run resumable: running [0, S) equals
 * running [0, m) and then [m, S) from the states it returned. */
typedef struct {
  int32_t n_sweeps;
  double T0, T1;
  int32_t sweep_begin, sweep_end;
} qp_schedule;

/* qp_build_qubo flags */
enum { QP_DENSE = 1, QP_STRUCTURED = 2, QP_DIST_I16 = 4 };
/* qp_anneal_opts.kernel.  STRUCTURED uses the row-parallel kernel for fields
 * of up to 512 cells and the general one above; STRUCTURED_ROWS forces the
 * row-parallel kernel (up to 512 cells), STRUCTURED_FLAT the general structured
 * kernel (up to 4096 cells), STRUCTURED_GROUP the grouped kernel that anneals 4
 * replicas per warp up to 64 cells and 2 up to 128 (faster than the
 * row-parallel kernel at low temperature, slower at high temperature).  Above
 * 256 cells the row-parallel kernel keeps each replica's spins in global
 * memory (more replicas resident per SM); STRUCTURED_ROWS_SHARED forces the
 * variant with the spins in shared memory.  All give the same results. */
enum {
  QP_KERNEL_AUTO = 0,
  QP_KERNEL_DENSE = 1,
  QP_KERNEL_STRUCTURED = 2,
  QP_KERNEL_STRUCTURED_FLAT = 3,
  QP_KERNEL_STRUCTURED_ROWS = 4,
  QP_KERNEL_STRUCTURED_GROUP = 5,
  QP_KERNEL_STRUCTURED_ROWS_SHARED = 6
};

/* qp_anneal_opts.flags.  QP_ANNEAL_SKIP_SETTLED lets the row-parallel kernel
 * (fields of up to 512 cells, also in qp_batch_*) skip a sweep whose outcome
 * is already known: once a sweep of a replica met no proposal with dE < len
 * (none accepted outright, none needing a draw), its state cannot change in
 * any later sweep whose table is no longer (len non-increasing, as on a
 * cooling schedule), so those sweeps are not evaluated.  Results are
 * identical bit for bit; only the time changes.  Other kernels ignore it. */
enum { QP_ANNEAL_SKIP_SETTLED = 1 };

typedef struct {
  int32_t kernel;            /* QP_KERNEL_*; AUTO = structured when built     */
  int32_t replicas_per_cta;  /* warps (= replicas) per CTA; 0 = chosen to keep
                                the most chains resident at once (occupancy) */
  int32_t replica_offset;    /* global index of replica 0 (its RNG stream)    */
  int64_t *accepts_out;      /* optional [R]: accepted flips per replica      */
  int32_t flags;             /* QP_ANNEAL_* bits                              */
} qp_anneal_opts;

/* Section II and Eqs. 3-6 (Algorithm 1, first five steps): build the path
 * QUBO of a field.  A <= 0 selects A = 2*max d (penalty above any one step).
 * B >= 1 weights the distance term; scale > 0 (100 = centi-units).
 * flags: QP_STRUCTURED keeps the C x C distance matrix on the device (the
 * structured sweep's input; int16 when QP_DIST_I16 is set or every entry
 * fits); QP_DENSE also stores the n x n matrix S of the dense form (int16 on
 * the device when every entry fits).  flags == 0 means QP_STRUCTURED.
 * Errors: QP_EINVAL (bad field, start not free, fewer than 2 cells),
 * QP_ERANGE (|dE| bound or d beyond int32), QP_ENOMEM, QP_ECUDA.
 * *out receives a handle owned by the caller (free with qp_destroy). */
qp_status qp_build_qubo(const qp_field *field, int32_t A, int32_t B, int32_t scale,
                        int32_t flags, qp_handle **out);

/* A generic QUBO in dense form: E(x) = sum_k S_kk x_k + sum_{k<l} S_kl x_k x_l
 * + c0 with S symmetric (n x n int32, row-major, host memory).  frozen (n
 * bytes, NULL = none) marks variables that are never proposed; they take
 * frozen_val (NULL = 0).  The dense form of Eq. 6 is one such QUBO.
 * Errors: QP_EINVAL (n < 1, S not symmetric), QP_ERANGE (a row's absolute sum
 * beyond int32), QP_ENOMEM, QP_ECUDA. */
/* The extended objective (Section V names battery capacity and the pesticide
 * amount as the next objectives and gives no formula; the reading here): the
 * distance term of Eq. 3 with one weight per leg,
 *   E(x) = sum_{t<C-1} w_t sum_{i,j} d_ij x_{t,i} x_{t+1,j} + the penalties,
 * where w_t stands for the mass carried on the leg from step t to t+1 (a fixed
 * amount sprayed per cell, flight energy taken proportional to mass times
 * distance).  leg_weights: n_legs = C - 1 non-negative int32, host memory,
 * copied.  A <= 0 selects A = 2 * max w * max d.  The handle holds the dense
 * form (QP_DENSE) and the distance matrix; it anneals with QP_KERNEL_DENSE
 * (QP_KERNEL_AUTO picks it), decodes like any field handle (qp_decode_path,
 * qp_decode_batch: the length reported is the unweighted one) and works with
 * qp_ws_walk.  The structured-form calls refuse it (QP_EINVAL): the structured
 * kernels of qp_anneal_ex, qp_anneal_noalloc, qp_anneal_pt, qp_anneal_timed,
 * the batch and the repair (whose 2-opt shortens the unweighted length).
 * Errors as qp_build_qubo; QP_EINVAL also for NULL or device weights, a wrong
 * count or a negative weight. */
qp_status qp_build_qubo_weighted(const qp_field *field, int32_t A, const int32_t *leg_weights, int32_t n_legs,
                                 int32_t scale, qp_handle **out);

qp_status qp_build_from_dense(const int32_t *S, int64_t n, const uint8_t *frozen,
                              const uint8_t *frozen_val, int64_t c0, qp_handle **out);

/* Sizes of a handle: n variables, C cells (0 for a generic QUBO), c0, max d
 * (0 for a generic QUBO), and the penalty weight A actually used. Any output
 * pointer may be NULL. */
qp_status qp_qubo_info(const qp_handle *h, int64_t *n_vars, int32_t *n_cells, int64_t *c0,
                       int32_t *max_d, int32_t *A_used);

/* The dense form S (n x n int32, caller-owned host buffer) of the handle. */
qp_status qp_export_dense(const qp_handle *h, int32_t *S_out);

/* The distance matrix d (C x C int32, caller-owned host buffer). QP_EINVAL
 * for a generic QUBO. */
qp_status qp_export_dist(const qp_handle *h, int32_t *d_out);

/* The acceptance thresholds of sweep `sweep` of `sched`: out[0] = 0xFFFFFFFF,
 * out[dE] = floor(2^32 exp(-dE/T_s)) for 1 <= dE < len.  *len_out = len.
 * QP_ERANGE if cap < len (len is still written). out may be NULL. */
qp_status qp_thresholds(const qp_schedule *sched, int32_t sweep, uint32_t *out, int32_t cap,
                        int32_t *len_out);

/* Anneal `replicas` independent chains of the handle's QUBO over the sweeps
 * [sweep_begin, sweep_end) of `sched` (the sampler step of Algorithm 1).
 * init_states: R*n bytes (0/1, t-major) or NULL for the all-zero start; the
 *   clamp / frozen values are applied on top.
 * states_out: R*n bytes, the final states.  energies_out: R int64 final E.
 * best_out: R int64 best feasible E (NULL allowed).
 * Same as qp_anneal_ex with every option at its default. */
qp_status qp_anneal(qp_handle *h, int32_t replicas, const qp_schedule *sched, uint64_t seed,
                    const uint8_t *init_states, uint8_t *states_out, int64_t *energies_out,
                    int64_t *best_out, void *cuda_stream);

/* qp_anneal with options (opts may be NULL).  The kernel choice changes the
 * speed, never the result: both kernels follow the same sequential sweep.
 * The dense kernel brings each accepted flip's row of S into shared memory
 * by a bulk copy when the buffers fit; a copy that has not completed after
 * ~0.5 s ends its replica with energy INT64_MIN, and a synchronous call
 * (some output in host memory) then returns QP_ETIMEOUT. */
qp_status qp_anneal_ex(qp_handle *h, int32_t replicas, const qp_schedule *sched,
                       uint64_t seed, const uint8_t *init_states, uint8_t *states_out,
                       int64_t *energies_out, int64_t *best_out, const qp_anneal_opts *opts,
                       void *cuda_stream);

/* The structured anneal of qp_anneal_ex (same kernel as QP_KERNEL_STRUCTURED_FLAT,
 * same results) without any allocation, for callers that cannot allocate
 * device memory while they run: software that reserves all of its memory at
 * start-up, code under an external memory manager that owns the GPU's memory,
 * or a loop that cannot afford an allocation's latency.  The paper has no
 * counterpart; this is a deployment entry point.
 * The per-replica working state lives in a fixed 16 MiB array in the library's
 * own device memory: R * (ceil(C*C/32) + 1, rounded up to 4) * 4 bytes must
 * fit, else QP_ERANGE.  CUDA loads the array's module lazily and allocates the
 * array then; qp_build_qubo does that for the handle's device (it is the
 * call that allocates), so this call needs a handle built by qp_build_qubo
 * and, from then on, the device holds the 16 MiB until the process exits.
 * Every buffer (init_states, states_out, energies_out, best_out) must be
 * device memory (QP_EINVAL otherwise); init_states and best_out may be NULL.
 * The schedule's threshold tables must already exist on the device: one
 * earlier qp_anneal/qp_anneal_ex call with the same n_sweeps, T0 and T1 builds
 * them, and they stay cached unless more than 4 GiB of other schedules' tables
 * were built since (QP_EINVAL otherwise).  Each call looks up the array's
 * device address afresh (cudaGetSymbolAddress), so nothing stale survives a
 * device reset.  Every call shares the one array, and each kernel rewrites
 * the part it uses before reading it, so nothing carries over between calls;
 * calls that overlap on the GPU (other streams, other threads) race on it and
 * must be serialised by the caller.  Asynchronous on cuda_stream. */
qp_status qp_anneal_noalloc(qp_handle *h, int32_t replicas, const qp_schedule *sched, uint64_t seed,
                            const uint8_t *init_states, uint8_t *states_out, int64_t *energies_out,
                            int64_t *best_out, int32_t replica_offset, void *cuda_stream);

/* Many fields of uneven size annealed in one persistent launch (the same
 * sampler as qp_anneal, batched over problems).  Field f runs `replicas`
 * chains with replica indices 0..replicas-1 and seed + f, so its results equal
 * qp_anneal(hs[f], replicas, sched, seed + f, NULL, ...) bit for bit.  Every
 * handle must come from qp_build_qubo with int16 distances (QP_ERANGE
 * otherwise; fields up to 512 cells); outputs are caller-owned device buffers
 * (states_out[f]: replicas*C_f^2 bytes, energies_out[f] and best_out[f]:
 * replicas int64; best_out or any best_out[f] may be NULL).
 * qp_batch_create builds the field table and the work order (largest fields
 * first), and captures a CUDA graph of {reset the work-queue head, launch the
 * persistent kernel}; qp_batch_run replays it on a stream (asynchronous);
 * qp_batch_destroy frees it.  The handles and output buffers must outlive the
 * batch.  Taking work is one atomic add per (field, replica): no device wait.
 * opts (NULL = defaults): replicas_per_cta (warps per CTA) and ctas (grid
 * size, 0 = as many as fit on the GPU at once), which the autotuner picks,
 * and flags: QP_ANNEAL_SKIP_SETTLED (same results) and QP_BATCH_D_SHARED, the
 * staging choice (same results): a CTA takes replicas_per_cta replicas of one
 * field at a time and stages that field's int16 distance matrix in shared
 * memory, instead of each warp taking one (field, replica) and reading d
 * from L2.  QP_EINVAL for other flags. */
enum { QP_BATCH_D_SHARED = 2 };
typedef struct qp_batch qp_batch;
typedef struct {
  int32_t replicas_per_cta;
  int32_t ctas;
  int32_t flags;  /* QP_ANNEAL_SKIP_SETTLED | QP_BATCH_D_SHARED, or 0 */
} qp_batch_opts;
qp_status qp_batch_create(qp_handle *const *hs, int32_t count, int32_t replicas, const qp_schedule *sched,
                          uint64_t seed, uint8_t *const *states_out, int64_t *const *energies_out,
                          int64_t *const *best_out, const qp_batch_opts *opts, qp_batch **out);
qp_status qp_batch_run(qp_batch *batch, void *cuda_stream);
/* The configuration a batch was built with (any pointer may be NULL). */
qp_status qp_batch_info(const qp_batch *batch, int32_t *replicas_per_cta, int32_t *ctas, int32_t *units);
void qp_batch_destroy(qp_batch *batch);

/* One-shot batch: create, run on cuda_stream, wait, destroy. */
qp_status qp_anneal_batch(qp_handle *const *hs, int32_t count, int32_t replicas, const qp_schedule *sched,
                          uint64_t seed, uint8_t *const *states_out, int64_t *const *energies_out,
                          int64_t *const *best_out, void *cuda_stream);

/* Algorithm 1 last step: the flight path of one state (n bytes, host or
 * device).  path_out[t] = cell id flown at step t (C int32, host), *length_out
 * = sum_t d(path[t], path[t+1]) (host).  QP_EINFEASIBLE if a row or column
 * sum is not 1 (outputs untouched). */
qp_status qp_decode_path(const qp_handle *h, const uint8_t *state, int32_t *path_out,
                         int64_t *length_out);

/* Decode R states on the device: paths_out [R*C] int32, lengths_out [R] int64
 * (-1 where the state is infeasible).  Pointers host or device. */
qp_status qp_decode_batch(const qp_handle *h, int32_t replicas, const uint8_t *states,
                          int32_t *paths_out, int64_t *lengths_out, void *cuda_stream);

/* Repair R states into flight paths on the device (one warp per state), so
 * that every state yields the feasible path the reconstruction step of
 * Algorithm 1 hands back, then shorten each path by 2-opt.  The paper does
 * not say how an infeasible sample is turned into a path; this is the rule:
 *   Greedy fix.  path[0] = s; for t = 1 .. C-1 the candidates are the cells
 *     not yet on the path with x_{t,i} = 1, or every cell not yet on the path
 *     if there is none; path[t] = the candidate nearest to path[t-1] (smallest
 *     d, ties to the smaller id).  A feasible state (every row and column sum
 *     1, x_{0,s} = 1) gives exactly its decoded path.
 *   2-opt.  Move (i, j), 1 <= i < j <= C-1, reverses path[i..j].  A pass
 *     scans i = 1 .. C-2 and, for each, j = i+1 .. C-1 in order, applying a
 *     move as soon as it makes the path strictly shorter and going on with
 *     the next j on the changed path.  Passes repeat while the previous one
 *     moved, at most max_passes of them (0: no 2-opt; < 0: until no move
 *     helps, which always ends since each move shortens an integer length).
 * states: R*n bytes (host or device).  paths_out: R*C int32; lengths_out: R
 * int64 (sum of d along the path); status_out: R int32 (NULL allowed):
 * 0 = feasible and kept as decoded, 1 = feasible and shortened by 2-opt,
 * 2 = infeasible, repaired.  Outputs host or device; asynchronous on
 * cuda_stream when every pointer is device memory.  QP_EINVAL for a generic
 * QUBO. */
qp_status qp_repair_batch(const qp_handle *h, int32_t replicas, const uint8_t *states, int32_t max_passes,
                          int32_t *paths_out, int64_t *lengths_out, int32_t *status_out, void *cuda_stream);

/* qp_repair_batch for one state (host or device) into host outputs. */
qp_status qp_repair_path(const qp_handle *h, const uint8_t *state, int32_t max_passes, int32_t *path_out,
                         int64_t *length_out, int32_t *status_out);

/* The sampler under a wall-clock budget: the solver time limit L of
 * Algorithm 1 (100 ms in the paper's evaluation, Section IV-C).  Runs the
 * geometric schedule (n_sweeps, T0, T1; sweep_begin/sweep_end are ignored)
 * on `replicas` chains, repairs every final state (qp_repair_batch with
 * max_passes) and returns the shortest path.
 *   Probes first run 9 sweeps of `replicas` chains at the constant
 *   temperature T0, then 9 at T1 from the first probe's states, and time
 *   sweeps 1..8 of each; the time per sweep is taken as the mean of the hot
 *   (slowest) and cold (fastest) rates, and the probes' chains are
 *   discarded.  If n_sweeps sweeps at that rate fit in what is left,
 *   every round runs the whole schedule; otherwise a shorter schedule with the
 *   same T0, T1 and n' sweeps runs instead, n' = the budget's share of sweeps
 *   rounded down to m*2^e (8 <= m < 16) so that such schedules repeat and
 *   their threshold tables are reused.  Round k anneals fresh chains with
 *   replica indices k*R .. k*R+R-1; a round starts while the previous round's
 *   duration still fits in the budget (round 0 always runs).
 * The sweeps run with QP_ANNEAL_SKIP_SETTLED (same results, less time).
 * Given info->n_sweeps and info->rounds the result is reproducible: it equals
 * qp_anneal_ex over sweeps [0, n_sweeps) with replica_offset k*R for each
 * round k, qp_repair_batch of each round's states, and the shortest path
 * (ties to the smaller replica index).  The budget is a target, not a bound:
 * round 0 always completes, and the first call on a schedule also builds its
 * threshold tables on the host (inside round 0).  path_out: C int32 (host);
 * *length_out: its length; state_out: n bytes of the winning replica's final
 * state (host, NULL allowed); info (NULL allowed) as below.  Synchronous. */
typedef struct {
  int32_t n_sweeps;    /* sweeps of the schedule that ran in every round */
  int32_t rounds;      /* rounds of `replicas` chains */
  int32_t replica;     /* replica index of the returned path */
  int32_t status;      /* its repair status (0, 1, 2 as in qp_repair_batch) */
  int64_t n_feasible;  /* final states over all rounds that were feasible */
  int64_t energy;      /* final energy E of the returned replica's state */
  double probe_ms;     /* wall time up to the end of the probe */
  double elapsed_ms;   /* wall time of the whole call */
} qp_timed_info;
qp_status qp_anneal_timed(qp_handle *h, int32_t replicas, const qp_schedule *sched, uint64_t seed,
                          double time_limit_ms, int32_t max_passes, int32_t *path_out, int64_t *length_out,
                          uint8_t *state_out, qp_timed_info *info, void *cuda_stream);

/* Replica exchange (parallel tempering) over the replica batch.  The paper
 * runs many chains of its sampler in parallel (Sections III-C, IV-A) and
 * does not say whether they interact; this is the standard way to let them.
 * G groups of M chains; chain r = g*M + m starts at level m of the ladder
 * T_m = T_lo (T_hi/T_lo)^(m/(M-1)) (m = 0 coldest; the geometric schedule
 * formula over M "sweeps").  Round e = 0 .. exchanges-1: every chain runs
 * sweeps [e*I, (e+1)*I) (I = sweeps_per_exchange; the sweep index feeds the
 * random counters as in qp_anneal) at the fixed temperature of its level,
 * then the pairs of levels (m, m+1), m = e mod 2, m+2, ..., of every group
 * try to trade: with a the chain at m and b the chain at m+1 and
 * X = E_b - E_a, the trade is accepted iff X <= 0 or (X < len and
 * u < thr[X]), thr = the threshold table at the effective temperature
 * T_m T_{m+1} / (T_{m+1} - T_m) (so the probability is
 * min(1, exp((1/T_m - 1/T_{m+1})(E_a - E_b)))), u = word 0 of
 * Philox4x32-10 at counter (m, e, g, 0x50545843).  A trade swaps the two
 * chains' levels; states stay with their chains.
 * init_states: G*M*n bytes or NULL (all-zero start).  Outputs (host or
 * device): states_out G*M*n final states and energies_out G*M final E, by
 * chain; best_out G*M (NULL allowed) the best feasible E of each chain at
 * any sweep end; levels_out G*M int32 (NULL allowed) each chain's final
 * level; swaps_out G*(M-1) int64 (NULL allowed) accepted trades of each
 * pair of levels.  Fields of up to 512 cells use the row kernel, larger ones
 * the flat kernel.  Asynchronous on cuda_stream when every output is device
 * memory; calls on one handle must not overlap (they share its buffers).
 * QP_ERANGE if two levels are so close that the exchange temperature
 * exceeds 1e8. */
typedef struct {
  int32_t levels;              /* M >= 2 */
  double T_lo, T_hi;           /* 0 < T_lo < T_hi */
  int32_t sweeps_per_exchange; /* I >= 1 */
  int32_t exchanges;           /* rounds >= 1; I * rounds sweeps in all */
} qp_pt_schedule;
qp_status qp_anneal_pt(qp_handle *h, int32_t groups, const qp_pt_schedule *pt, uint64_t seed,
                       const uint8_t *init_states, uint8_t *states_out, int64_t *energies_out,
                       int64_t *best_out, int32_t *levels_out, int64_t *swaps_out, void *cuda_stream);

/* ---- Learned warm start (no counterpart in the paper: a seed generator for
 * the sampler).  A per-cell MLP maps 16 features of a free cell to logits over
 * its step t in the flight path (t < 256): Linear(16,256)+ReLU,
 * Linear(256,256)+ReLU x 2, Linear(256,256).  bf16 weights and activations,
 * fp32 accumulation on the tensor cores (tcgen05), fp32 master weights and
 * Adam moments.  Trained with softmax cross-entropy over the steps t < C of
 * the cell's field, on paths the annealer itself found. */
typedef struct qp_ws qp_ws;

/* A model with He-uniform weights drawn from `seed` (zero biases). */
qp_status qp_ws_create(uint64_t seed, qp_ws **out);
void qp_ws_destroy(qp_ws *ws);
/* Number of parameters; the flat layout of get/set is W1[256][16], b1[256],
 * W2[256][256], b2, W3[256][256], b3, W4[256][256], b4 (fp32). */
int64_t qp_ws_param_count(void);
qp_status qp_ws_get_params(qp_ws *ws, float *params_out);
qp_status qp_ws_set_params(qp_ws *ws, const float *params);

/* The 16 features of every free cell of a field, in cell-id order (row-major
 * free cells): x/15, y/15, blocked fraction of the 8 neighbours (obstacles or
 * outside), start x/15, start y/15, W/16, H/16, C/256, (x-start x)/15,
 * (y-start y)/15, x/(W-1), y/(H-1), free fraction of the 5x5 block, y mod 2,
 * 1, 0.  feats_out: C*16 floats (host) or NULL to get only *n_cells. */
qp_status qp_ws_features(const qp_field *field, float *feats_out, int32_t *n_cells);

/* Logits for M cells: feats (M*16 fp32, host), logits_out (M*256 fp32, host or
 * device).  QP_ETIMEOUT if a tensor-core wait gave up. */
qp_status qp_ws_forward(qp_ws *ws, const float *feats, int32_t M, float *logits_out, void *cuda_stream);

/* How the forward pass (of qp_ws_forward, _grads, _train_step, _infer) runs:
 * QP_WS_FORWARD_FUSED (the default) is one launch for all four layers, each
 * 128-cell tile's activations kept in shared memory between layers;
 * QP_WS_FORWARD_LAYERED is one tensor-core GEMM launch per layer, the
 * activations through global memory.  Both issue the same MMAs in the same
 * order, so their logits are bit-identical.  QP_EINVAL for another mode. */
enum { QP_WS_FORWARD_FUSED = 0, QP_WS_FORWARD_LAYERED = 1 };
qp_status qp_ws_set_forward_mode(qp_ws *ws, int32_t mode);

/* Gradients of the mean cross-entropy over M cells without updating: labels
 * (M int32: the cell's step, -1 = ignore), steps (M int32: the cell's field
 * size C, logits t >= C are masked).  grads_out (param_count floats, host, may
 * be NULL) in the get/set layout; *loss_out = mean loss (may be NULL). */
qp_status qp_ws_grads(qp_ws *ws, const float *feats, const int32_t *labels, const int32_t *steps, int32_t M,
                      float *grads_out, float *loss_out, void *cuda_stream);

/* One training step: gradients as in qp_ws_grads, then Adam (Kingma & Ba,
 * ICLR 2015: bias-corrected first and second moments; beta1 0.9f, beta2
 * 0.999f, eps 1e-8f as fp32 constants, step count from 1) with learning rate
 * lr, in fp32 on the master weights; the bf16 weights and their transposes are
 * rewritten from the updated masters (round to nearest even). */
qp_status qp_ws_train_step(qp_ws *ws, const float *feats, const int32_t *labels, const int32_t *steps, int32_t M,
                           float lr, float *loss_out, void *cuda_stream);

/* Read-back of the model for checking it (no counterpart in the paper).
 * qp_ws_get_state: one fp32 tensor set in the flat get/set layout -- the
 * master parameters (QP_WS_STATE_PARAMS), Adam's first and second moments
 * (QP_WS_STATE_ADAM_M, _ADAM_V; zero before the first step) or the gradients
 * of the last qp_ws_grads / qp_ws_train_step call (QP_WS_STATE_GRADS: the
 * very gradients its Adam step applied).  out: param_count floats (host).
 * qp_ws_get_buffer: raw contents of a device buffer, rows 0..rows-1 of the
 * last forward / backward pass (bf16 as uint16 bits, row-major, 16 columns
 * for QP_WS_BUF_X0, 256 otherwise; QP_WS_BUF_Z is fp32): the input features
 * X0, the hidden activations H1..H3 (written by passes that keep them:
 * qp_ws_grads, qp_ws_train_step, or any pass in the layered mode), the logits
 * Z, their gradient dZ and the back-propagated dH1..dH3 (the gradients at
 * H1..H3 after the ReLU mask).  QP_WS_BUF_W_BF16 + l and QP_WS_BUF_WT_BF16 +
 * l (l = 0..3) give layer l's bf16 weight [out x in] and its transpose
 * [in x out] (rows ignored).  QP_EINVAL for an unknown buffer or rows beyond
 * the buffers' capacity (the largest M so far, rounded up to 128); rows past
 * the last pass's M hold no defined values.  Both wait for the device. */
enum { QP_WS_STATE_PARAMS = 0, QP_WS_STATE_ADAM_M = 1, QP_WS_STATE_ADAM_V = 2, QP_WS_STATE_GRADS = 3 };
qp_status qp_ws_get_state(qp_ws *ws, int32_t which, float *out);
enum {
  QP_WS_BUF_X0 = 0, QP_WS_BUF_H1 = 1, QP_WS_BUF_H2 = 2, QP_WS_BUF_H3 = 3, QP_WS_BUF_Z = 4, QP_WS_BUF_DZ = 5,
  QP_WS_BUF_DH1 = 6, QP_WS_BUF_DH2 = 7, QP_WS_BUF_DH3 = 8, QP_WS_BUF_W_BF16 = 16, QP_WS_BUF_WT_BF16 = 32
};
qp_status qp_ws_get_buffer(qp_ws *ws, int32_t which, int32_t rows, void *out);

/* Logits of one field's C cells (row stride ld >= C, host) -> a feasible
 * one-hot state (C*C bytes, t-major) and its path: the start cell takes step
 * 0, then the largest remaining logit over unassigned cells and free steps
 * fixes one (cell, step) pair at a time (ties: smaller cell, then smaller
 * step).  Either output may be NULL. */
qp_status qp_ws_decode(const float *logits, int32_t ld, int32_t C, int32_t start_cell, uint8_t *state_out,
                       int32_t *path_out);

/* Logits of one field's C cells -> a feasible state by a guided walk: from
 * the start cell, each step goes to the nearest unvisited cell (d: the C x C
 * distance matrix, host, e.g. from qp_export_dist); among equally near cells
 * the one with the smallest expected step E_j = sum_t softmax(logits_j)_t t
 * (t < C) wins, then the smaller cell id.  Either output may be NULL. */
qp_status qp_ws_decode_walk(const float *logits, int32_t ld, int32_t C, int32_t start_cell, const int32_t *d,
                            uint8_t *state_out, int32_t *path_out);

/* The whole inference step of the warm start for one field: its features
 * (qp_ws_features), the network's logits (qp_ws_forward) and a feasible seed
 * decoded from them -- the guided walk (qp_ws_decode_walk) when d (the
 * field's C x C distance matrix, host, e.g. qp_export_dist) is given, greedy
 * matching (qp_ws_decode) when d is NULL.  state_out: C*C bytes, path_out: C
 * int32 (host; either may be NULL).  QP_ERANGE above 256 cells. */
qp_status qp_ws_infer(qp_ws *ws, const qp_field *field, const int32_t *d, uint8_t *state_out, int32_t *path_out,
                      void *cuda_stream);

/* Device decode of the warm start (no counterpart in the paper).
 * qp_ws_expected_steps: E_m = sum_{t < T_m} t softmax(logits_m)_t over the
 * first T_m = steps[m] logits of row m (T_m clamped to [1, min(256, ld)]), in
 * fp32, for M rows of row stride ld.  logits (M*ld fp32), steps (M int32) and
 * E_out (M fp32) are device buffers (QP_EINVAL otherwise).  Asynchronous.
 * qp_ws_walk: a feasible one-hot seed of the handle's field by a walk: step 0
 * is the start cell; each later step goes to a cell not yet visited, chosen
 * among the unvisited cells within `slack` (same units as d, >= 0) of the
 * nearest unvisited distance from the current cell, as the smallest (score,
 * distance, cell id) when score (C fp32, finite, -0 counts as +0) is given,
 * else the smallest (distance, cell id).  slack = 0 with score = the expected
 * steps is qp_ws_decode_walk; no score is the plain nearest-cell walk.
 * Outputs (device, each may be NULL, not both state and path): state_out C*C
 * bytes (zeroed, then one 1 per step), path_out C int32, length_out one int64
 * (the path's length in d units).  Needs a handle from qp_build_qubo (QP_EINVAL
 * otherwise); QP_ERANGE for more than 4096 cells or max d >= 2^20; host
 * buffers are refused (QP_EINVAL).  One warp runs the field; asynchronous. */
qp_status qp_ws_expected_steps(const float *logits, int32_t ld, int32_t M, const int32_t *steps, float *E_out,
                               void *cuda_stream);
qp_status qp_ws_walk(qp_handle *h, const float *score, int32_t slack, uint8_t *state_out, int32_t *path_out,
                     int64_t *length_out, void *cuda_stream);
/* qp_ws_greedy: qp_ws_decode on the device.  logits (C rows of stride ld >= C,
 * fp32, finite), state_out (C*C bytes, zeroed then one 1 per step) and
 * path_out (C int32) are device buffers (either output may be NULL, not
 * both); 1 <= C <= 256, 0 <= start_cell < C (QP_EINVAL otherwise, and for
 * host buffers or buffers smaller than the call needs).  Step 0 is the start
 * cell; then the largest logit over the unassigned cells and the free steps
 * 1..C-1 fixes one (cell, step) pair at a time, ties to the smaller cell,
 * then the smaller step.  One CTA; asynchronous on the stream. */
qp_status qp_ws_greedy(const float *logits, int32_t ld, int32_t C, int32_t start_cell, uint8_t *state_out,
                       int32_t *path_out, void *cuda_stream);

/* Self-test of the bounded wait that guards the library's asynchronous copies
 * (no counterpart in the paper): one warp waits on an mbarrier phase that
 * nothing completes.  *timed_out = 1 when the wait gave up after its bound
 * (~0.5 s of SM clock) instead of hanging; *waited_ms (NULL allowed) = how
 * long it waited, from the SM clock.  The context stays usable. */
qp_status qp_selftest_wait(int32_t *timed_out, double *waited_ms);

/* Device bounds checks (no counterpart in the paper; the substitute for a
 * memory checker).  The checked build of the library (compiled with
 * QP_DEVICE_CHECKS=1) tests, before the access, every index of the sweep and
 * repair kernels' threshold-table, distance-row, spin-word, row-of-S and
 * hot-cell reads and writes; a failed check records (site << 24) | (index mod
 * 2^24) and the access goes to element 0 instead, so it cannot leave its
 * array.  *enabled = 1 in the checked build, 0 in the release build (which
 * compiles no checks).  *first_failure = the first failure since the last
 * call, 0 = none; the call clears it.  Sites: 1 threshold table, 2 distance
 * row, 3 spin word, 4 row of S, 5 repair distance, 6 hot-cell list.
 * QP_ECUDA if the record could not be read from the device. */
qp_status qp_device_checks(int32_t *enabled, uint32_t *first_failure);

/* Free a handle and its device memory (NULL is ignored). */
void qp_destroy(qp_handle *h);

/* Message of the calling thread's last failed call ("" if none). */
const char *qp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QPATH_H */
