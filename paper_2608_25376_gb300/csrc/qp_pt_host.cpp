// Host side of replica exchange (qp_anneal_pt): the ladder's exchange tables
// (one Metropolis table per pair of neighbouring levels, at their effective
// temperature) and the loop of sweep blocks and exchange rounds.
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

// --------------------------------------------------------------------------- replica exchange
namespace {

struct XchgEntry {
  DevBuf thr, off, len;
};
std::mutex g_xchg_mu;
std::map<SchedKey, std::unique_ptr<XchgEntry>> g_xchg;

// Exchange tables of a ladder: row m (m < M-1) holds the Metropolis
// thresholds at T_m T_{m+1} / (T_{m+1} - T_m); built once per device.
qp_status exchange_tables(const qp_schedule &ladder, const uint32_t **thr, const int64_t **off,
                          const int32_t **len) {
  int dev = 0;
  QP_CU(cudaGetDevice(&dev));
  SchedKey key{dev, ladder.n_sweeps, 0, 0};
  std::memcpy(&key.t0, &ladder.T0, 8);
  std::memcpy(&key.t1, &ladder.T1, 8);
  std::lock_guard<std::mutex> lk(g_xchg_mu);
  auto it = g_xchg.find(key);
  if (it == g_xchg.end()) {
    const int M = ladder.n_sweeps;
    std::vector<int64_t> o(M - 1);
    std::vector<int32_t> l(M - 1);
    std::vector<uint32_t> all, tab;
    for (int m = 0; m + 1 < M; ++m) {
      const double Tm = temperature(ladder, m), Tn = temperature(ladder, m + 1);
      const double Te = Tm * Tn / (Tn - Tm);
      if (!(Te > 0.0) || !std::isfinite(Te) || Te > 1e8)
        return fail(QP_ERANGE, "ladder levels %d and %d are too close (exchange temperature %g)", m, m + 1, Te);
      build_thresholds(Te, tab);
      o[m] = (int64_t)all.size();
      l[m] = (int32_t)tab.size();
      all.insert(all.end(), tab.begin(), tab.end());
    }
    auto e = std::make_unique<XchgEntry>();
    QP_TRY(e->thr.ensure(all.size() * 4));
    QP_TRY(e->off.ensure(o.size() * 8));
    QP_TRY(e->len.ensure(l.size() * 4));
    QP_CU(cudaMemcpy(e->thr.p, all.data(), all.size() * 4, cudaMemcpyHostToDevice));
    QP_CU(cudaMemcpy(e->off.p, o.data(), o.size() * 8, cudaMemcpyHostToDevice));
    QP_CU(cudaMemcpy(e->len.p, l.data(), l.size() * 4, cudaMemcpyHostToDevice));
    it = g_xchg.emplace(key, std::move(e)).first;
  }
  *thr = it->second->thr.as<uint32_t>();
  *off = it->second->off.as<int64_t>();
  *len = it->second->len.as<int32_t>();
  return QP_OK;
}

}  // namespace

extern "C" qp_status qp_anneal_pt(qp_handle *h, int32_t G, const qp_pt_schedule *pt, uint64_t seed,
                                  const uint8_t *init, uint8_t *states_out, int64_t *energies_out,
                                  int64_t *best_out, int32_t *levels_out, int64_t *swaps_out, void *stream_) {
  g_err.clear();
  if (!h || !pt || !states_out || !energies_out || G < 1) return fail(QP_EINVAL, "bad argument");
  if (!h->path) return fail(QP_EINVAL, "replica exchange needs a handle built by qp_build_qubo");
  if (h->weighted) return fail(QP_EINVAL, "replica exchange: the structured form is unweighted: a handle with leg weights anneals with the dense kernel only");
  const int M = pt->levels, I = pt->sweeps_per_exchange, X = pt->exchanges;
  if (M < 2 || I < 1 || X < 1) return fail(QP_EINVAL, "need levels >= 2, sweeps_per_exchange >= 1, exchanges >= 1");
  if (!(pt->T_lo > 0.0) || !(pt->T_hi > pt->T_lo) || !std::isfinite(pt->T_hi))
    return fail(QP_EINVAL, "need 0 < T_lo < T_hi (finite)");
  if ((int64_t)G * M > INT32_MAX / 2) return fail(QP_ERANGE, "too many chains");
  if ((int64_t)I * X > INT32_MAX) return fail(QP_ERANGE, "too many sweeps");
  qp_schedule ladder{M, pt->T_lo, pt->T_hi, 0, M};
  QP_TRY(check_schedule(&ladder));
  const int32_t R = G * M;
  DevSet ds(h->dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  DeviceSchedule lt;
  std::shared_ptr<const void> ladder_keep;  // the ladder's tables stay alive through the rounds
  QP_TRY(device_schedule(ladder, &lt, &ladder_keep));
  const uint32_t *xthr = nullptr;
  const int64_t *xoff = nullptr;
  const int32_t *xlen = nullptr;
  QP_TRY(exchange_tables(ladder, &xthr, &xoff, &xlen));
  const size_t n = (size_t)h->n;
  QP_DEV_FITS(init, (size_t)R * n, "init_states");
  QP_DEV_FITS(states_out, (size_t)R * n, "states_out");
  QP_DEV_FITS(energies_out, (size_t)R * 8, "energies_out");
  QP_DEV_FITS(best_out, (size_t)R * 8, "best_out");
  QP_DEV_FITS(levels_out, (size_t)R * 4, "levels_out");
  QP_DEV_FITS(swaps_out, (size_t)G * (M - 1) * 8, "swaps_out");
  QP_TRY(h->pt_states[0].ensure((size_t)R * n));
  QP_TRY(h->pt_states[1].ensure((size_t)R * n));
  QP_TRY(h->pt_E.ensure((size_t)R * 8));
  QP_TRY(h->pt_bseg.ensure((size_t)R * 8));
  QP_TRY(h->pt_best.ensure((size_t)R * 8));
  QP_TRY(h->pt_level.ensure((size_t)R * 4));
  QP_TRY(h->pt_owner.ensure((size_t)R * 4));
  QP_TRY(h->pt_swaps.ensure((size_t)G * (M - 1) * 8));
  {
    std::vector<int32_t> lev(R), own(R);
    std::vector<int64_t> best(R, INT64_MAX);
    for (int r = 0; r < R; ++r) {
      lev[r] = r % M;
      own[r] = r;
    }
    QP_CU(cudaMemcpyAsync(h->pt_level.p, lev.data(), (size_t)R * 4, cudaMemcpyHostToDevice, st));
    QP_CU(cudaMemcpyAsync(h->pt_owner.p, own.data(), (size_t)R * 4, cudaMemcpyHostToDevice, st));
    QP_CU(cudaMemcpyAsync(h->pt_best.p, best.data(), (size_t)R * 8, cudaMemcpyHostToDevice, st));
    QP_CU(cudaMemsetAsync(h->pt_swaps.p, 0, (size_t)G * (M - 1) * 8, st));
    QP_CU(cudaStreamSynchronize(st));  // the host vectors go out of scope
  }
  const uint8_t *init_d = init;
  if (init && !is_device_ptr(init)) {
    QP_TRY(h->in_stage.ensure((size_t)R * n));
    QP_CU(cudaMemcpyAsync(h->in_stage.p, init, (size_t)R * n, cudaMemcpyHostToDevice, st));
    init_d = h->in_stage.as<uint8_t>();
  }
  uint8_t *cur = h->pt_states[0].as<uint8_t>(), *nxt = h->pt_states[1].as<uint8_t>();
  StructArgs a{};
  a.C = h->C; a.Cp = h->Cp; a.start = h->start; a.A = h->A; a.B = h->B;
  a.d = h->d_dev.p;
  a.R = R; a.rep_offset = 0;
  a.key0 = (uint32_t)seed; a.key1 = (uint32_t)(seed >> 32);
  a.thr = lt.thr; a.thr_off = lt.off; a.thr_len = lt.len; a.thr_c = lt.c;
  a.E_out = h->pt_E.as<int64_t>(); a.best_out = h->pt_bseg.as<int64_t>(); a.acc_out = nullptr;
  a.level = h->pt_level.as<int32_t>();
  PtArgs x{};
  x.G = G; x.M = M;
  x.E = h->pt_E.as<int64_t>(); x.best_seg = h->pt_bseg.as<int64_t>(); x.best = h->pt_best.as<int64_t>();
  x.owner = h->pt_owner.as<int32_t>(); x.level = h->pt_level.as<int32_t>(); x.swaps = h->pt_swaps.as<int64_t>();
  x.thr = xthr; x.off = xoff; x.len = xlen;
  x.key0 = a.key0; x.key1 = a.key1;
  LaunchInfo info;
  for (int e = 0; e < X; ++e) {
    a.sweep_begin = e * I;
    a.sweep_end = (e + 1) * I;
    a.init = e == 0 ? init_d : cur;
    a.states_out = nxt;
    QP_TRY(launch_structured_auto(h, a, 0, true, st, &info));
    x.phase = e & 1;
    x.round = e;
    QP_CU(launch_pt_exchange(x, st));
    std::swap(cur, nxt);
  }
  bool host_out = false;
  auto put = [&](void *dst, const void *src, size_t bytes) -> qp_status {
    if (!dst) return QP_OK;
    host_out = host_out || !is_device_ptr(dst);
    QP_CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    return QP_OK;
  };
  QP_TRY(put(states_out, cur, (size_t)R * n));
  QP_TRY(put(energies_out, h->pt_E.p, (size_t)R * 8));
  QP_TRY(put(best_out, h->pt_best.p, (size_t)R * 8));
  QP_TRY(put(levels_out, h->pt_level.p, (size_t)R * 4));
  QP_TRY(put(swaps_out, h->pt_swaps.p, (size_t)G * (M - 1) * 8));
  if (host_out || (init && init_d != init)) QP_CU(cudaStreamSynchronize(st));
  return QP_OK;
}

