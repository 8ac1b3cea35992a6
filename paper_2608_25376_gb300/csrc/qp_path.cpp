// Host side of the path-level calls: repair of annealed states into flight
// paths (qp_repair_batch, qp_repair_path) and the sampler under a wall-clock
// budget (qp_anneal_timed).
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

extern "C" qp_status qp_repair_batch(const qp_handle *hc, int32_t R, const uint8_t *states, int32_t max_passes,
                                     int32_t *paths_out, int64_t *lengths_out, int32_t *status_out,
                                     void *stream_) {
  g_err.clear();
  qp_handle *h = const_cast<qp_handle *>(hc);
  if (!h || !states || !paths_out || !lengths_out || R < 1) return fail(QP_EINVAL, "bad argument");
  if (!h->path) return fail(QP_EINVAL, "a generic QUBO has no path");
  if (h->weighted) return fail(QP_EINVAL, "the repair's 2-opt shortens the unweighted length: not for a handle with leg weights");
  DevSet ds(h->dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  const size_t n = (size_t)h->n;
  QP_DEV_FITS(states, (size_t)R * n, "states");
  QP_DEV_FITS(paths_out, (size_t)R * h->C * 4, "paths_out");
  QP_DEV_FITS(lengths_out, (size_t)R * 8, "lengths_out");
  QP_DEV_FITS(status_out, (size_t)R * 4, "status_out");
  const uint8_t *sd = states;
  bool sync = false;
  if (!is_device_ptr(states)) {
    QP_TRY(h->in_stage.ensure((size_t)R * n));
    QP_CU(cudaMemcpyAsync(h->in_stage.p, states, (size_t)R * n, cudaMemcpyHostToDevice, st));
    sd = h->in_stage.as<uint8_t>();
    sync = true;
  }
  int32_t *pd = paths_out, *rd = status_out;
  int64_t *ld = lengths_out;
  const bool ph = !is_device_ptr(paths_out), lh = !is_device_ptr(lengths_out);
  const bool rh = status_out && !is_device_ptr(status_out);
  if (ph) { QP_TRY(h->p_stage.ensure((size_t)R * h->C * 4)); pd = h->p_stage.as<int32_t>(); }
  if (lh) { QP_TRY(h->l_stage.ensure((size_t)R * 8)); ld = h->l_stage.as<int64_t>(); }
  if (!status_out || rh) { QP_TRY(h->r_stage.ensure((size_t)R * 4)); rd = h->r_stage.as<int32_t>(); }
  QP_CU(launch_repair(sd, R, h->C, h->start, h->d32_dev.as<int32_t>(), max_passes, pd, ld, rd, st));
  if (ph) QP_CU(cudaMemcpyAsync(paths_out, pd, (size_t)R * h->C * 4, cudaMemcpyDeviceToHost, st));
  if (lh) QP_CU(cudaMemcpyAsync(lengths_out, ld, (size_t)R * 8, cudaMemcpyDeviceToHost, st));
  if (rh) QP_CU(cudaMemcpyAsync(status_out, rd, (size_t)R * 4, cudaMemcpyDeviceToHost, st));
  if (sync || ph || lh || rh) QP_CU(cudaStreamSynchronize(st));
  return QP_OK;
}

extern "C" qp_status qp_repair_path(const qp_handle *h, const uint8_t *state, int32_t max_passes,
                                    int32_t *path_out, int64_t *length_out, int32_t *status_out) {
  if (!path_out || !length_out || is_device_ptr(path_out) || is_device_ptr(length_out) ||
      (status_out && is_device_ptr(status_out)))
    return fail(QP_EINVAL, "qp_repair_path: outputs must be host memory");
  int32_t status = 0;
  QP_TRY(qp_repair_batch(h, 1, state, max_passes, path_out, length_out, &status, nullptr));
  if (status_out) *status_out = status;
  return QP_OK;
}

namespace {

double ms_since(const std::chrono::steady_clock::time_point &t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// n rounded down to m * 2^e with 8 <= m < 16 (n itself below 16), so that
// budget-fitted schedules come from a short list and their tables are reused.
int32_t quantize_sweeps(int64_t n) {
  if (n < 16) return (int32_t)std::max<int64_t>(1, n);
  int e = 0;
  while ((n >> e) >= 16) ++e;
  return (int32_t)((n >> e) << e);
}

}  // namespace

extern "C" qp_status qp_anneal_timed(qp_handle *h, int32_t R, const qp_schedule *sc, uint64_t seed,
                                     double time_limit_ms, int32_t max_passes, int32_t *path_out,
                                     int64_t *length_out, uint8_t *state_out, qp_timed_info *info,
                                     void *stream_) {
  const auto t0 = std::chrono::steady_clock::now();
  g_err.clear();
  if (!h || !sc || !path_out || !length_out || R < 1) return fail(QP_EINVAL, "bad argument");
  if (!h->path) return fail(QP_EINVAL, "qp_anneal_timed needs a handle built by qp_build_qubo");
  if (h->weighted) return fail(QP_EINVAL, "qp_anneal_timed: the structured form is unweighted: a handle with leg weights anneals with the dense kernel only");
  if (!(time_limit_ms > 0.0) || !std::isfinite(time_limit_ms)) return fail(QP_EINVAL, "time_limit_ms must be > 0");
  qp_schedule full = *sc;
  full.sweep_begin = 0;
  full.sweep_end = full.n_sweeps;
  QP_TRY(check_schedule(&full));
  if ((int64_t)R * 2 > INT32_MAX) return fail(QP_ERANGE, "too many replicas");
  DevSet ds(h->dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  const size_t n = (size_t)h->n;
  const int C = h->C;
  QP_TRY(h->t_states[0].ensure((size_t)R * n));
  QP_TRY(h->t_states[1].ensure((size_t)R * n));
  QP_TRY(h->t_E.ensure((size_t)R * 8));
  QP_TRY(h->t_paths.ensure((size_t)R * C * 4));
  QP_TRY(h->t_len.ensure((size_t)R * 8));
  QP_TRY(h->t_stat.ensure((size_t)R * 4));
  uint8_t *S0 = h->t_states[0].as<uint8_t>(), *S1 = h->t_states[1].as<uint8_t>();
  int64_t *E = h->t_E.as<int64_t>(), *Ld = h->t_len.as<int64_t>();
  int32_t *Pd = h->t_paths.as<int32_t>(), *Sd = h->t_stat.as<int32_t>();
  DeviceSchedule dsched;
  QP_TRY(device_schedule(full, &dsched, nullptr));  // build the tables before the rounds

  std::vector<int64_t> len(R), en(R);
  std::vector<int32_t> stat(R);
  struct Best {
    int64_t length = INT64_MAX, energy = 0;
    int32_t replica = -1, status = 0;
  } best;
  int64_t n_feasible = 0;
  // Repair the R final states in `S`, fold them into `best` (shortest path,
  // ties to the smaller replica index) and keep the winner's path and state.
  auto harvest = [&](const uint8_t *S, int32_t offset) -> qp_status {
    QP_CU(launch_repair(S, R, C, h->start, h->d32_dev.as<int32_t>(), max_passes, Pd, Ld, Sd, st));
    QP_CU(cudaMemcpyAsync(len.data(), Ld, (size_t)R * 8, cudaMemcpyDeviceToHost, st));
    QP_CU(cudaMemcpyAsync(stat.data(), Sd, (size_t)R * 4, cudaMemcpyDeviceToHost, st));
    QP_CU(cudaMemcpyAsync(en.data(), E, (size_t)R * 8, cudaMemcpyDeviceToHost, st));
    QP_CU(cudaStreamSynchronize(st));
    int arg = -1;
    for (int r = 0; r < R; ++r) {
      n_feasible += stat[r] != 2;
      if (len[r] < best.length) {
        best.length = len[r];
        arg = r;
      }
    }
    if (arg >= 0) {
      best.replica = offset + arg;
      best.status = stat[arg];
      best.energy = en[arg];
      QP_CU(cudaMemcpyAsync(path_out, Pd + (size_t)arg * C, (size_t)C * 4, cudaMemcpyDeviceToHost, st));
      if (state_out) QP_CU(cudaMemcpyAsync(state_out, S + (size_t)arg * n, n, cudaMemcpyDeviceToHost, st));
      QP_CU(cudaStreamSynchronize(st));
    }
    return QP_OK;
  };
  auto run = [&](const qp_schedule &s, int32_t b, int32_t e, const uint8_t *init, uint8_t *out,
                 int32_t offset) -> qp_status {
    qp_schedule part = s;
    part.sweep_begin = b;
    part.sweep_end = e;
    qp_anneal_opts o{};
    o.replica_offset = offset;
    o.flags = QP_ANNEAL_SKIP_SETTLED;  // same results, settled sweeps cost nothing
    return qp_anneal_ex(h, R, &part, seed, init, out, E, nullptr, &o, st);
  };

  // Probes: 9 sweeps at the constant temperature T0, then 9 at T1 starting
  // from the first probe's states; sweeps 1..8 of each are timed (sweep 0 of
  // the first also pays any first-launch cost).  Hot sweeps are the slowest
  // and cold ones the fastest; the schedule's time per sweep is taken as the
  // mean of the two.  The probes' chains are thrown away; their tables are 9
  // short rows each.
  auto probe_at = [&](double T, const uint8_t *init, uint8_t *out, double *ms_out) -> qp_status {
    qp_schedule pr = full;
    pr.n_sweeps = 9;
    pr.T0 = pr.T1 = T;
    pr.sweep_end = 9;
    QP_TRY(run(pr, 0, 1, init, S1, 0));
    QP_CU(cudaStreamSynchronize(st));
    const double ta = ms_since(t0);
    QP_TRY(run(pr, 1, 9, S1, out, 0));
    QP_CU(cudaStreamSynchronize(st));
    *ms_out = (ms_since(t0) - ta) / 8.0;
    return QP_OK;
  };
  double t_hot = 0.0, t_cold = 0.0;
  QP_TRY(probe_at(full.T0, nullptr, S0, &t_hot));
  QP_TRY(probe_at(full.T1, S0, S0, &t_cold));
  const double probe_ms = ms_since(t0);
  const double per_sweep = std::max(0.5 * (t_hot + t_cold), 1e-6);
  const double left = time_limit_ms - probe_ms;
  int32_t n_used = full.n_sweeps;
  if (per_sweep * full.n_sweeps > 0.9 * left)  // the schedule does not fit: a shorter one that does
    n_used = std::min(full.n_sweeps, quantize_sweeps((int64_t)std::max(1.0, 0.8 * left / per_sweep)));
  qp_schedule used = full;
  used.n_sweeps = n_used;
  used.sweep_end = n_used;
  // Rounds of fresh chains (replica indices k*R .. k*R+R-1 in round k); a
  // round starts while the previous one's duration still fits in what is left.
  int32_t rounds = 0;
  double round_ms = 0.0;
  while ((int64_t)(rounds + 1) * R <= INT32_MAX) {
    const double now = ms_since(t0);
    if (rounds > 0 && now + round_ms > time_limit_ms) break;
    QP_TRY(run(used, 0, n_used, nullptr, S0, rounds * R));
    QP_TRY(harvest(S0, rounds * R));
    round_ms = ms_since(t0) - now;
    ++rounds;
  }
  *length_out = best.length;
  if (info) {
    info->n_sweeps = n_used;
    info->rounds = rounds;
    info->replica = best.replica;
    info->status = best.status;
    info->n_feasible = n_feasible;
    info->energy = best.energy;
    info->probe_ms = probe_ms;
    info->elapsed_ms = ms_since(t0);
  }
  return QP_OK;
}

