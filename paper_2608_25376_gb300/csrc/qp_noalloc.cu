// qp_anneal_noalloc: the structured anneal for callers that must not allocate
// device memory while they run -- flight or control software that reserves
// all of its memory at start-up, code running under an external memory
// manager that owns the GPU's memory, or a loop that cannot afford an
// allocation's latency.  Every other entry point may allocate (handles, staging
// buffers, the per-replica working state of large fields); this one uses a
// fixed scratch array in the library's own device memory instead.
//
// The scratch is a file-scope __device__ array of kStaticScratchBytes (16 MiB).
// CUDA loads a module lazily, on the first use of one of its kernels or
// symbols, and the driver allocates the array then; from that moment the
// device holds it until the process exits.  qp_build_qubo triggers the load
// (noalloc_preload, with the handle's device current), so a call here, which
// needs such a handle, finds the array already in place.  Host code cannot
// use the array's name as a device address (it names a host-side stand-in):
// every call looks the address up with cudaGetSymbolAddress, with the
// handle's device current (no cached pointer can outlive a device reset).
#include "qp_internal.h"

namespace qp {
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;

__device__ __align__(256) uint32_t g_static_scratch[kStaticScratchBytes / 4];

// Device address of the scratch array on the current device.
cudaError_t scratch_address(uint32_t **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<uint32_t *>(p);
  return cudaSuccess;
}

}  // namespace

void noalloc_preload() {
  uint32_t *p = nullptr;
  if (scratch_address(&p) != cudaSuccess) cudaGetLastError();
}

}  // namespace qp

extern "C" qp_status qp_anneal_noalloc(qp_handle *h, int32_t R, const qp_schedule *sc, uint64_t seed,
                                       const uint8_t *init, uint8_t *states_out, int64_t *energies_out,
                                       int64_t *best_out, int32_t replica_offset, void *stream_) {
  using namespace qp;
  clear_error();
  StructView v;
  if (!h || !handle_struct_view(h, &v)) return set_error(QP_EINVAL, "qp_anneal_noalloc needs a handle built by qp_build_qubo");
  if (v.weighted) return set_error(QP_EINVAL, "qp_anneal_noalloc: the structured form is unweighted: a handle with leg weights anneals with the dense kernel only");
  if (!sc || !states_out || !energies_out || R < 1 || replica_offset < 0 ||
      (int64_t)replica_offset + R > INT32_MAX)
    return set_error(QP_EINVAL, "qp_anneal_noalloc: bad argument");
  if (sc->n_sweeps < 1 || sc->sweep_begin < 0 || sc->sweep_end < sc->sweep_begin || sc->sweep_end > sc->n_sweeps)
    return set_error(QP_EINVAL, "qp_anneal_noalloc: need 0 <= sweep_begin <= sweep_end <= n_sweeps");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return set_error(QP_ECUDA, "qp_anneal_noalloc: cudaGetDevice failed");
  if (prev != v.dev && cudaSetDevice(v.dev) != cudaSuccess)
    return set_error(QP_ECUDA, "qp_anneal_noalloc: cudaSetDevice failed");
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev != dev) cudaSetDevice(prev);
    }
  } restore{prev, v.dev};

  if (!device_pointer(states_out) || !device_pointer(energies_out) || (best_out && !device_pointer(best_out)) ||
      (init && !device_pointer(init)))
    return set_error(QP_EINVAL, "qp_anneal_noalloc: every buffer must be device memory");
  const size_t n = (size_t)v.C * v.C;
  if (!device_range_fits(states_out, (size_t)R * n) || !device_range_fits(energies_out, (size_t)R * 8) ||
      (best_out && !device_range_fits(best_out, (size_t)R * 8)) || (init && !device_range_fits(init, (size_t)R * n)))
    return set_error(QP_EINVAL, "qp_anneal_noalloc: a device buffer is smaller than the call needs");
  DeviceSchedule sched;
  std::shared_ptr<const void> sched_keep;  // the tables stay alive until the launch is queued
  if (!schedule_lookup(*sc, &sched, &sched_keep))
    return set_error(QP_EINVAL,
                     "qp_anneal_noalloc: the schedule's threshold tables do not exist on this device yet; "
                     "make one qp_anneal/qp_anneal_ex call with the same n_sweeps, T0, T1 first");
  const size_t words = structured_gstate_words(v.C);
  if ((size_t)R * words * 4 > kStaticScratchBytes)
    return set_error(QP_ERANGE,
                     "qp_anneal_noalloc: replicas x per-replica state exceed the 16 MiB static scratch "
                     "(R * (ceil(C*C/32) + 1, rounded up to 4) * 4 bytes)");
  uint32_t *scratch = nullptr;
  const cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return set_error(QP_ECUDA, cudaGetErrorString(e));

  StructArgs a{};
  a.C = v.C; a.Cp = v.Cp; a.start = v.start; a.A = v.A; a.B = v.B;
  a.d = v.d;
  a.R = R; a.rep_offset = replica_offset;
  a.sweep_begin = sc->sweep_begin; a.sweep_end = sc->sweep_end;
  a.key0 = (uint32_t)seed; a.key1 = (uint32_t)(seed >> 32);
  a.thr = sched.thr; a.thr_off = sched.off; a.thr_len = sched.len; a.thr_c = sched.c;
  a.init = init; a.states_out = states_out; a.E_out = energies_out; a.best_out = best_out; a.acc_out = nullptr;
  a.gstate = scratch;
  a.nw_pad = (int32_t)words;
  const cudaError_t le = launch_structured(a, v.d_i16, 4, /*want_state_smem=*/false,
                                           static_cast<cudaStream_t>(stream_), nullptr);
  if (le != cudaSuccess) return set_error(QP_ECUDA, cudaGetErrorString(le));
  return QP_OK;
}
