// Host side of the batched anneal: the field table and the work order of
// (field, replica) units, the CUDA graph of {reset the queue head, launch the
// persistent kernel}, and the one-shot helper.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "qp_host.h"

using namespace qp;
using namespace qp::host;

// --------------------------------------------------------------------------- batched anneal
struct qp_batch {
  int dev = 0;
  int count = 0, R = 0, Cmax = 0, W = 0, blocks = 0, n_units = 0;
  bool staged = false;
  DevBuf fields, units, counter;
  std::shared_ptr<const void> sched_keep;  // the schedule's tables, referenced by the captured graph
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~qp_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
  }
};

extern "C" qp_status qp_batch_create(qp_handle *const *hs, int32_t count, int32_t R, const qp_schedule *sc,
                                     uint64_t seed, uint8_t *const *states_out, int64_t *const *energies_out,
                                     int64_t *const *best_out, const qp_batch_opts *opts, qp_batch **out) {
  g_err.clear();
  if (!hs || !out || !states_out || !energies_out) return fail(QP_EINVAL, "NULL argument");
  *out = nullptr;
  if (count < 1 || R < 1) return fail(QP_EINVAL, "need count >= 1 and replicas >= 1");
  if ((int64_t)count * R > INT32_MAX) return fail(QP_ERANGE, "count x replicas beyond int32");
  QP_TRY(check_schedule(sc));
  qp_batch_opts o{};
  if (opts) o = *opts;
  auto b = std::make_unique<qp_batch>();
  QP_CU(cudaGetDevice(&b->dev));
  int Cmax = 0;
  for (int f = 0; f < count; ++f) {
    const qp_handle *h = hs[f];
    if (!h || !h->path) return fail(QP_EINVAL, "field %d: a batch needs handles built by qp_build_qubo", f);
    if (h->weighted) return fail(QP_EINVAL, "field %d: the batch sweep is unweighted (a handle with leg weights)", f);
    if (h->dev != b->dev) return fail(QP_EINVAL, "field %d lives on another device", f);
    if (!h->d_i16) return fail(QP_ERANGE, "field %d: a batch needs int16 distances", f);
    if (!is_device_ptr(states_out[f]) || !is_device_ptr(energies_out[f]) ||
        (best_out && best_out[f] && !is_device_ptr(best_out[f])))
      return fail(QP_EINVAL, "field %d: batch outputs must be device memory", f);
    QP_DEV_FITS(states_out[f], (size_t)R * h->n, "states_out[f]");
    QP_DEV_FITS(energies_out[f], (size_t)R * 8, "energies_out[f]");
    if (best_out) QP_DEV_FITS(best_out[f], (size_t)R * 8, "best_out[f]");
    Cmax = std::max(Cmax, (int)h->C);
  }
  if (o.flags & ~(QP_ANNEAL_SKIP_SETTLED | QP_BATCH_D_SHARED)) return fail(QP_EINVAL, "unknown batch flags");
  const bool staged = (o.flags & QP_BATCH_D_SHARED) != 0;
  auto fits = [&](int w) { return staged ? batch_staged_supported(Cmax, w) : batch_supported(Cmax, w); };
  int W = o.replicas_per_cta > 0 ? o.replicas_per_cta : 4;
  while (W > 1 && !fits(W)) --W;
  if (!fits(W)) return fail(QP_ERANGE, "largest field (%d cells) too large for the batch kernel", Cmax);
  DeviceSchedule sched;
  QP_TRY(device_schedule(*sc, &sched, &b->sched_keep));
  std::vector<StructArgs> fa(count);
  for (int f = 0; f < count; ++f) {
    const qp_handle *h = hs[f];
    StructArgs &a = fa[f];
    a = StructArgs{};
    a.C = h->C; a.Cp = h->Cp; a.start = h->start; a.A = h->A; a.B = h->B;
    a.d = h->d_dev.p;
    a.R = R; a.rep_offset = 0;
    a.sweep_begin = sc->sweep_begin; a.sweep_end = sc->sweep_end;
    const uint64_t sf = seed + (uint64_t)f;
    a.key0 = (uint32_t)sf; a.key1 = (uint32_t)(sf >> 32);
    a.thr = sched.thr; a.thr_off = sched.off; a.thr_len = sched.len; a.thr_c = sched.c;
    a.init = nullptr;
    a.states_out = states_out[f]; a.E_out = energies_out[f];
    a.best_out = best_out ? best_out[f] : nullptr;
    a.acc_out = nullptr;
    a.skip_settled = (o.flags & QP_ANNEAL_SKIP_SETTLED) ? 1 : 0;
  }
  // work units, largest fields first
  std::vector<int> order(count);
  for (int f = 0; f < count; ++f) order[f] = f;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hs[x]->C > hs[y]->C; });
  // a unit: one (field, replica) for a warp, or W replicas of one field for a
  // CTA when d is staged in shared memory
  std::vector<int2> units;
  units.reserve((size_t)count * R);
  for (int f : order)
    for (int r = 0; r < R; r += staged ? W : 1) units.push_back(make_int2(f, r));
  QP_TRY(b->fields.ensure(fa.size() * sizeof(StructArgs)));
  QP_TRY(b->units.ensure(units.size() * sizeof(int2)));
  QP_TRY(b->counter.ensure(sizeof(int)));
  QP_CU(cudaMemcpy(b->fields.p, fa.data(), fa.size() * sizeof(StructArgs), cudaMemcpyHostToDevice));
  QP_CU(cudaMemcpy(b->units.p, units.data(), units.size() * sizeof(int2), cudaMemcpyHostToDevice));
  int per_sm = 0, sms = 0;
  QP_CU(staged ? batch_staged_prepare(Cmax, W, &per_sm) : batch_prepare(Cmax, W, &per_sm));
  QP_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev));
  if (per_sm < 1) return fail(QP_ERANGE, "batch kernel does not fit on an SM");
  const int want = o.ctas > 0 ? o.ctas : per_sm * sms;
  b->blocks = std::min(want, staged ? (int)units.size() : (int)((units.size() + W - 1) / W));
  b->staged = staged;
  b->count = count; b->R = R; b->Cmax = Cmax; b->W = W; b->n_units = (int)units.size();
  // one graph: reset the queue head, run the persistent kernel
  QP_CU(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  QP_CU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e1 = cudaMemsetAsync(b->counter.p, 0, sizeof(int), b->cap);
  cudaError_t e2 = e1;
  if (e1 == cudaSuccess)
    e2 = staged ? launch_batch_staged(b->fields.as<StructArgs>(), b->units.as<int2>(), b->n_units,
                                      b->counter.as<int>(), Cmax, W, b->blocks, b->cap)
                : launch_batch(b->fields.as<StructArgs>(), b->units.as<int2>(), b->n_units, b->counter.as<int>(),
                               Cmax, W, b->blocks, b->cap);
  cudaError_t e3 = cudaStreamEndCapture(b->cap, &b->graph);
  if (e2 != cudaSuccess) return fail(QP_ECUDA, "capturing the batch graph: %s", cudaGetErrorString(e2));
  if (e3 != cudaSuccess) return fail(QP_ECUDA, "capturing the batch graph: %s", cudaGetErrorString(e3));
  QP_CU(cudaGraphInstantiate(&b->exec, b->graph, 0));
  *out = b.release();
  return QP_OK;
}

extern "C" qp_status qp_batch_run(qp_batch *b, void *stream) {
  g_err.clear();
  if (!b) return fail(QP_EINVAL, "batch is NULL");
  DevSet ds(b->dev);
  QP_CU(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
  return QP_OK;
}

extern "C" qp_status qp_batch_info(const qp_batch *b, int32_t *replicas_per_cta, int32_t *ctas, int32_t *units) {
  if (!b) return fail(QP_EINVAL, "batch is NULL");
  if (replicas_per_cta) *replicas_per_cta = b->W;
  if (ctas) *ctas = b->blocks;
  if (units) *units = b->n_units;
  return QP_OK;
}

extern "C" void qp_batch_destroy(qp_batch *b) {
  if (!b) return;
  DevSet ds(b->dev);
  delete b;
}

extern "C" qp_status qp_anneal_batch(qp_handle *const *hs, int32_t count, int32_t R, const qp_schedule *sc,
                                     uint64_t seed, uint8_t *const *states_out, int64_t *const *energies_out,
                                     int64_t *const *best_out, void *stream) {
  qp_batch *b = nullptr;
  QP_TRY(qp_batch_create(hs, count, R, sc, seed, states_out, energies_out, best_out, nullptr, &b));
  const qp_status s = qp_batch_run(b, stream);
  if (s == QP_OK) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    qp_batch_destroy(b);
    if (e != cudaSuccess) return fail(QP_ECUDA, "batch: %s", cudaGetErrorString(e));
    return QP_OK;
  }
  qp_batch_destroy(b);
  return s;
}
