// Internal types shared by the host library (qp_host.cpp) and the kernels.
// Not part of the public ABI (include/qpath.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <mutex>
#include <string>

#include "qpath.h"

namespace qp {

constexpr uint32_t kRngTag = 0x51505448u;  // counter word 3 of every sweep draw
constexpr int kMaxCells = 4096;            // C limit (n = C^2 fits int32 comfortably)
constexpr int kMaxWarpsPerCta = 16;

// Thresholds of one schedule on one device: thr[off[s] + dE] for 0 <= dE < len[s].
struct DeviceSchedule {
  const uint32_t *thr = nullptr;
  const int64_t *off = nullptr;
  const int32_t *len = nullptr;
  const float *c = nullptr;  // log2(e) / T_s, rounded to float
  int32_t n_sweeps = 0;
  int32_t max_len = 0;
  int64_t total = 0;
};

// Arguments of the structured sweep (one warp = one replica).
struct StructArgs {
  int32_t C, Cp, start, A, B;
  const void *d;             // C x Cp, int16 or int32
  int32_t R, rep_offset;
  int32_t sweep_begin, sweep_end;
  uint32_t key0, key1;
  const uint32_t *thr;
  const int64_t *thr_off;
  const int32_t *thr_len;
  const float *thr_c;
  const uint8_t *init;       // R x n or null
  uint8_t *states_out;       // R x n
  int64_t *E_out, *best_out, *acc_out;  // best/acc may be null
  uint32_t *gstate;          // R x nw_pad words when the state lives in global memory
  int32_t nw_pad;
  // Replica exchange: the table row replica r (local index) uses in every
  // sweep of the launch (its ladder level); null = row s for sweep s.
  const int32_t *level;
  // QP_ANNEAL_SKIP_SETTLED: skip sweeps that provably change nothing
  int32_t skip_settled;
};

// Arguments of the dense sweep (one warp = one replica).
struct DenseArgs {
  int64_t n;
  int32_t np;                // padded row stride of S (multiple of 8)
  const void *S;             // n x np, int16 or int32
  int64_t c0;
  int32_t C;                 // path structure (0 = generic)
  const uint32_t *frozen_bits, *fval_bits;  // nw words each
  int32_t R, rep_offset;
  int32_t sweep_begin, sweep_end;
  uint32_t key0, key1;
  const uint32_t *thr;
  const int64_t *thr_off;
  const int32_t *thr_len;
  const float *thr_c;
  const uint8_t *init;
  uint8_t *states_out;
  int64_t *E_out, *best_out, *acc_out;
  int32_t *hbuf;             // R x np int32 when h lives in global memory
  int32_t *err;              // set to 1 when a bulk row copy did not complete (nullable)
};

struct LaunchInfo {
  int warps_per_cta = 0;
  int blocks = 0;
  size_t smem = 0;
  const char *variant = "";
};

// Kernel launchers (qp_kernels.cu).  Return cudaSuccess or the launch error.
cudaError_t launch_structured(const StructArgs &a, bool d_i16, int warps_per_cta, bool want_state_smem,
                              cudaStream_t st, LaunchInfo *info);
size_t structured_gstate_words(int C);  // nw_pad for the global-state layout
bool structured_state_fits_smem(int C, bool d_i16, int warps_per_cta);
// Row-parallel structured kernel (qp_sweep_rows.cu), fields of up to 512 cells.
bool rows_supported(int C, bool d_i16, int warps_per_cta);
// Replicas per CTA for the row kernel that keep the most chains resident on
// the GPU at once (R replicas in all); memoised per device and shape.
int rows_auto_warps(int C, bool d_i16, int R);
// The row kernel with the spins in global memory (fields of 257..512 cells):
// words of one replica's row bitsets, support, occupancy choice, launch
// (a.gstate: R x rows_g_words(C) words).  A launch with more chains than fit
// on the GPU at once runs persistent over (replica, sweep segment) units.
size_t rows_g_words(int C);
bool rows_g_supported(int C, bool d_i16, int warps_per_cta);
int rows_g_auto_warps(int C, bool d_i16, int R);
// counter (1 int), progress (R ints) and err (1 int) must be zero at launch;
// carry: 2R int64 the kernel uses between segments of a chain.
cudaError_t launch_rows_g(const StructArgs &a, bool d_i16, int warps_per_cta, int *counter, int *progress,
                          long long *carry, int *err, cudaStream_t st, LaunchInfo *info);
cudaError_t launch_rows(const StructArgs &a, bool d_i16, int warps_per_cta, cudaStream_t st,
                        LaunchInfo *info);
// Batched persistent launch (qp_sweep_rows.cu): fields[] per field, units[]
// = (field, replica) in processing order, counter = the work-queue head (zeroed
// before each launch).  All fields must use int16 distances.
bool batch_supported(int Cmax, int warps_per_cta);
cudaError_t batch_prepare(int Cmax, int warps_per_cta, int *blocks_per_sm);
cudaError_t launch_batch(const StructArgs *fields, const int2 *units, int n_units, int *counter, int Cmax,
                         int warps_per_cta, int blocks, cudaStream_t st);
// The batched launch with each field's d staged in shared memory (units of W
// replicas of one field per CTA).
bool batch_staged_supported(int Cmax, int warps_per_cta);
cudaError_t batch_staged_prepare(int Cmax, int warps_per_cta, int *blocks_per_sm);
cudaError_t launch_batch_staged(const StructArgs *fields, const int2 *units, int n_units, int *counter, int Cmax,
                                int warps_per_cta, int blocks, cudaStream_t st);
// Grouped structured kernel (qp_sweep_group.cu): 4 replicas per warp for
// C <= 64, 2 for C <= 128.
int group_size_for(int C);
bool group_supported(int C, bool d_i16, int warps_per_cta);
cudaError_t launch_group(const StructArgs &a, bool d_i16, int warps_per_cta, cudaStream_t st, LaunchInfo *info);
cudaError_t launch_dense(const DenseArgs &a, bool s_i16, int warps_per_cta, cudaStream_t st,
                         LaunchInfo *info);
bool dense_h_fits_smem(int64_t n, int C, int warps_per_cta);
// w: per-leg weights (device, C-1 int32) in place of B, or null
cudaError_t launch_build_dense(void *S, bool s_i16, int32_t np, int32_t C, const int32_t *d32,
                               int32_t A, int32_t B, cudaStream_t st, const int32_t *w = nullptr);
cudaError_t launch_decode(const uint8_t *states, int32_t R, int32_t C, const int32_t *d32,
                          int32_t *paths, int64_t *lengths, cudaStream_t st);

// Read-only views used by the allocation-free entry point (qp_noalloc.cu);
// none of these allocate.
// Repair of R states into paths (greedy fix + 2-opt), one warp per replica.
size_t repair_smem_per_warp(int32_t C);
cudaError_t launch_repair(const uint8_t *states, int32_t R, int32_t C, int32_t start, const int32_t *d32,
                          int32_t max_passes, int32_t *paths, int64_t *lengths, int32_t *status,
                          cudaStream_t st);

// Replica exchange round (qp_pt.cu).
struct PtArgs {
  int32_t G, M, phase, round;
  const int64_t *E;          // R final energies of the last block of sweeps
  const int64_t *best_seg;   // R best feasible energies of that block (null: skip the fold)
  int64_t *best;             // R running minimum
  int32_t *owner;            // G x M: chain at each level
  int32_t *level;            // R: level of each chain
  int64_t *swaps;            // G x (M-1) accepted trades per pair
  const uint32_t *thr;       // exchange tables, row m at off[m], len[m] entries
  const int64_t *off;
  const int32_t *len;
  uint32_t key0, key1;
};
cudaError_t launch_pt_exchange(const PtArgs &a, cudaStream_t st);

struct StructView {
  int dev;
  int32_t C, Cp, start, A, B, max_d;
  const void *d;
  bool d_i16;
  const int32_t *d32;  // C x C int32 on the device
  bool weighted;       // leg weights on the distance term (the structured kernels do not apply them)
};
bool handle_struct_view(const qp_handle *h, StructView *out);  // false for a generic QUBO
// false if not cached on this device; *keep (may be NULL) holds the tables alive
bool schedule_lookup(const qp_schedule &sc, DeviceSchedule *out, std::shared_ptr<const void> *keep);
qp_status set_error(qp_status s, const char *msg);
void clear_error();  // empties this thread's qp_last_error message
bool device_pointer(const void *p);
// True when the caller's device buffer [p, p + bytes) lies inside the one
// allocation that holds p (cuMemGetAddressRange), or when the driver cannot
// tell (p not in its allocation tables).  A pooling allocator's buffer lies
// inside a larger block, so only overruns past that block are caught.
bool device_range_fits(const void *p, size_t bytes);

// Makes the current device load the module that holds qp_anneal_noalloc's
// fixed scratch array (the driver allocates the array at that moment; CUDA
// loads modules lazily).  qp_build_qubo calls it, where allocating is
// allowed, so that the allocation-free entry point never triggers the load.
// Failure is not reported here: qp_anneal_noalloc reports it on its call.
void noalloc_preload();

// Every device allocation of the library.  Fault injection for tests: when
// the environment variable QPATH_FAIL_ALLOC holds N, the next N allocations
// (counted from the moment the value was first seen) succeed and every later
// one fails with cudaErrorMemoryAllocation, until the value changes.
cudaError_t dev_malloc(void **p, size_t bytes);

// Device bounds checks of the checked build (QP_DEVICE_CHECKS=1): each
// returns, and clears, the first failed check of its translation unit's
// kernels, (site << 24) | index, 0 = none; always 0 in the release build.
namespace chk {
uint32_t kernels();
uint32_t rows();
uint32_t group();
uint32_t repair();
int32_t enabled();
}  // namespace chk

// Held around every "set the kernel's dynamic shared-memory limit, then
// launch (or query the occupancy)" pair whose size depends on the call, so
// that calls from several host threads cannot launch under another call's
// smaller limit.
std::mutex &launch_mutex();

}  // namespace qp
