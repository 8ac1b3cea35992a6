// Host-side internals of libqpath shared by qp_host.cpp (build, anneal,
// decode), qp_batch.cpp (batched launch), qp_path.cpp (repair, time budget)
// and qp_pt_host.cpp (replica exchange): error reporting, device buffers, the
// schedule tables and the handle.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "qp_internal.h"

namespace qp {
namespace host {

// Message of the calling thread's last failed call (qp_last_error).
extern thread_local std::string g_err;

// Record a printf-style message and return s.
qp_status fail(qp_status s, const char *fmt, ...);

// A caller's device buffer smaller than the call needs is refused before any
// launch (QP_EINVAL) when the driver can see it.
#define QP_DEV_FITS(p, bytes, what)                                                            \
  do {                                                                                          \
    if ((p) && ::qp::host::is_device_ptr(p) && !::qp::device_range_fits((p), (bytes)))          \
      return ::qp::host::fail(QP_EINVAL, "%s: the device buffer is smaller than the %zu bytes " \
                              "the call needs", (what), (size_t)(bytes));                       \
  } while (0)

#define QP_CU(call)                                                                    \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? QP_ENOMEM : QP_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                  \
  } while (0)

#define QP_TRY(expr)              \
  do {                            \
    qp_status s_ = (expr);        \
    if (s_ != QP_OK) return s_;   \
  } while (0)

bool is_device_ptr(const void *p);

// A device allocation owned by a handle, grown on demand.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  qp_status ensure(size_t want) {
    if (want <= bytes) return QP_OK;
    release();
    cudaError_t e = dev_malloc(&p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return fail(QP_ENOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    bytes = want;
    return QP_OK;
  }
  template <typename T>
  T *as() const { return static_cast<T *>(p); }
};

// Make `dev` current for the scope (restores the caller's device).
struct DevSet {
  int prev = -1;
  explicit DevSet(int dev) {
    int cur = 0;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev) {
      prev = cur;
      cudaSetDevice(dev);
    }
  }
  ~DevSet() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Key of the per-device table caches (schedules, replica-exchange ladders).
struct SchedKey {
  int dev;
  int32_t n;
  uint64_t t0, t1;
  bool operator<(const SchedKey &o) const {
    return std::tie(dev, n, t0, t1) < std::tie(o.dev, o.n, o.t0, o.t1);
  }
};

double temperature(const qp_schedule &sc, int s);
// thr[dE] = floor(2^32 exp(-dE/T)) for dE >= 1 until it reaches 0; thr[0] unused.
void build_thresholds(double T, std::vector<uint32_t> &out);
qp_status check_schedule(const qp_schedule *sc);
// Device tables of a schedule (all n_sweeps sweeps), built once per device and
// cached (least recently used dropped first beyond 4 GiB of tables).  *keep
// (may be NULL) holds the tables alive while the caller needs them.
qp_status device_schedule(const qp_schedule &sc, DeviceSchedule *out, std::shared_ptr<const void> *keep);

}  // namespace host
}  // namespace qp

// The handle behind the ABI's opaque qp_handle.
struct qp_handle {
  int dev = 0;
  bool path = false;       // built from a field (structured terms available)
  bool weighted = false;   // per-leg weights on the distance term: the dense form only
  int32_t C = 0, start = 0, A = 0, B = 0, max_d = 0;
  int64_t n = 0, c0 = 0;
  std::vector<int32_t> d;  // C x C (host)
  // device data
  qp::host::DevBuf d_dev;            // C x Cp, int16 or int32
  bool d_i16 = false;
  int32_t Cp = 0;
  qp::host::DevBuf d32_dev;          // C x C int32 (decode, dense build)
  qp::host::DevBuf S_dev;            // n x np, int16 or int32
  bool has_dense = false, S_i16 = false;
  int32_t np = 0;
  qp::host::DevBuf frozen_bits, fval_bits;
  std::vector<uint8_t> frozen_host, fval_host;  // generic QUBOs
  // scratch
  qp::host::DevBuf rg_aux, rg_carry;  // the segmented row kernel: counter, progress flags, carried best/acc
  qp::host::DevBuf gstate, hbuf, in_stage, st_stage, e_stage, b_stage, a_stage, p_stage, l_stage, r_stage;
  qp::host::DevBuf kernel_err;  // int32 flag: a bulk row copy of the dense sweep did not complete
  qp::host::DevBuf t_states[2], t_E, t_paths, t_len, t_stat;  // qp_anneal_timed
  qp::host::DevBuf pt_states[2], pt_E, pt_bseg, pt_best, pt_level, pt_owner, pt_swaps;  // qp_anneal_pt
};

namespace qp {
namespace host {
// The structured sweep of a.R replicas: the row kernel when allowed and the
// field fits it, else the flat kernel.
// W = replicas per CTA, 0 = chosen from the occupancy (row kernel) or 4 (flat kernel)
qp_status launch_structured_auto(qp_handle *h, StructArgs &a, int W, bool allow_rows, cudaStream_t st,
                                 LaunchInfo *info, bool rows_shared_spins = false);
}  // namespace host
}  // namespace qp
