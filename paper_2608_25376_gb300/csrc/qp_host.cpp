// Host side of libqpath: argument checks, the QUBO build of Section II and
// Eqs. 3-6, the schedule and acceptance-threshold tables, buffer staging and
// kernel dispatch, and path decoding (Algorithm 1, last step).  The public
// contract of every function is documented in include/qpath.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "qp_host.h"

using namespace qp;
using namespace qp::host;

// --------------------------------------------------------------------------- errors
namespace qp {
namespace host {

thread_local std::string g_err;

qp_status fail(qp_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

}  // namespace host

cudaError_t dev_malloc(void **p, size_t bytes) {
  static std::mutex mu;
  static std::string seen;
  static long left = -1;  // allocations before injected failures start; -1 = none
  {
    const char *env = std::getenv("QPATH_FAIL_ALLOC");
    const std::string v = env ? env : "";
    std::lock_guard<std::mutex> lk(mu);
    if (v != seen) {
      seen = v;
      left = v.empty() ? -1 : std::max(0L, std::strtol(v.c_str(), nullptr, 10));
    }
    if (left == 0) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
    if (left > 0) --left;
  }
  return cudaMalloc(p, bytes);
}

namespace host {

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace host
}  // namespace qp

namespace {

int round_up_i(int x, int m) { return (x + m - 1) / m * m; }

// Exact round(scale * sqrt(q)): r = floor(sqrt(N)) for N = scale^2 q by a
// floating-point estimate corrected in integers, then round half up, which
// is round(sqrt(N)) because N - r^2 > r  <=>  sqrt(N) > r + 1/2.
int64_t round_scaled_sqrt(int64_t q, int64_t scale) {
  const int64_t N = scale * scale * q;
  int64_t r = (int64_t)std::sqrt((double)N);
  while (r > 0 && r * r > N) --r;
  while ((r + 1) * (r + 1) <= N) ++r;
  return (N - r * r > r) ? r + 1 : r;
}

}  // namespace

// --------------------------------------------------------------------------- schedules
namespace qp {
namespace host {

double temperature(const qp_schedule &sc, int s) {
  if (sc.n_sweeps <= 1) return sc.T0;
  return sc.T0 * std::pow(sc.T1 / sc.T0, (double)s / (double)(sc.n_sweeps - 1));
}

// thr[dE] = floor(2^32 exp(-dE/T)) for dE >= 1 until it reaches 0; thr[0] unused.
void build_thresholds(double T, std::vector<uint32_t> &out) {
  out.clear();
  out.push_back(0xFFFFFFFFu);
  for (int64_t de = 1;; ++de) {
    const double v = std::floor(std::ldexp(std::exp(-(double)de / T), 32));
    if (v <= 0.0) break;
    out.push_back((uint32_t)v);
  }
}

qp_status check_schedule(const qp_schedule *sc) {
  if (!sc) return fail(QP_EINVAL, "schedule is NULL");
  if (sc->n_sweeps < 1) return fail(QP_EINVAL, "n_sweeps must be >= 1");
  if (!(sc->T0 > 0.0) || !(sc->T1 > 0.0) || !std::isfinite(sc->T0) || !std::isfinite(sc->T1))
    return fail(QP_EINVAL, "temperatures must be finite and > 0");
  if (sc->T0 > 1e8 || sc->T1 > 1e8) return fail(QP_ERANGE, "temperatures above 1e8 make tables too large");
  if (sc->sweep_begin < 0 || sc->sweep_end < sc->sweep_begin || sc->sweep_end > sc->n_sweeps)
    return fail(QP_EINVAL, "need 0 <= sweep_begin <= sweep_end <= n_sweeps");
  return QP_OK;
}

namespace {
struct SchedEntry {
  DevBuf thr, off, len, c;
  DeviceSchedule view;
  size_t bytes = 0;
  uint64_t last_use = 0;
};

// Schedules cached per device, least recently used dropped first once the
// tables exceed kSchedCacheBytes.  Entries are shared: a caller keeps the
// tables it launches with alive for as long as it holds its reference (a
// batch for its whole life), and the device memory is freed by the last
// holder; cudaFree waits for the device, so no kernel still reading the
// tables can see them go.
constexpr size_t kSchedCacheBytes = size_t(4) << 30;

// The cache's size limit: QPATH_SCHEDULE_CACHE_MB (MiB) when set, else 4 GiB.
size_t sched_cache_limit() {
  const char *v = std::getenv("QPATH_SCHEDULE_CACHE_MB");
  if (v && *v) {
    const long long mb = std::atoll(v);
    if (mb > 0) return (size_t)mb << 20;
  }
  return kSchedCacheBytes;
}
std::mutex g_sched_mu;
std::map<SchedKey, std::shared_ptr<SchedEntry>> g_sched;
size_t g_sched_bytes = 0;
uint64_t g_sched_clock = 0;

SchedKey key_of(int dev, const qp_schedule &sc) {
  SchedKey key{dev, sc.n_sweeps, 0, 0};
  std::memcpy(&key.t0, &sc.T0, 8);
  std::memcpy(&key.t1, &sc.T1, 8);
  return key;
}
}  // namespace

qp_status device_schedule(const qp_schedule &sc, DeviceSchedule *out, std::shared_ptr<const void> *keep) {
  int dev = 0;
  QP_CU(cudaGetDevice(&dev));
  const SchedKey key = key_of(dev, sc);
  std::lock_guard<std::mutex> lk(g_sched_mu);
  auto it = g_sched.find(key);
  if (it != g_sched.end()) {
    it->second->last_use = ++g_sched_clock;
    *out = it->second->view;
    if (keep) *keep = it->second;
    return QP_OK;
  }
  auto e = std::make_shared<SchedEntry>();
  std::vector<int64_t> off(sc.n_sweeps);
  std::vector<int32_t> len(sc.n_sweeps);
  std::vector<float> cf(sc.n_sweeps);
  const double log2e = 1.0 / std::log(2.0);
  // The tables of long hot schedules run to tens of MB; host threads build
  // contiguous sweep ranges (every entry is computed the same way whatever
  // the split), then the ranges are placed one after another.
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int parts = std::max(1, std::min({hw, 16, sc.n_sweeps / 32 + 1}));
  std::vector<std::vector<uint32_t>> chunk(parts);
  auto work = [&](int p) {
    const int s0 = (int)((int64_t)sc.n_sweeps * p / parts), s1 = (int)((int64_t)sc.n_sweeps * (p + 1) / parts);
    std::vector<uint32_t> tab;
    for (int s = s0; s < s1; ++s) {
      const double T = temperature(sc, s);
      build_thresholds(T, tab);
      cf[s] = (float)(log2e / T);
      off[s] = (int64_t)chunk[p].size();  // local; made global below
      len[s] = (int32_t)tab.size();
      chunk[p].insert(chunk[p].end(), tab.begin(), tab.end());
    }
  };
  {
    std::vector<std::thread> pool;
    for (int p = 1; p < parts; ++p) pool.emplace_back(work, p);
    work(0);
    for (auto &t : pool) t.join();
  }
  std::vector<uint32_t> all;
  size_t total = 0;
  for (auto &c : chunk) total += c.size();
  all.reserve(total);
  for (int p = 0; p < parts; ++p) {
    const int s0 = (int)((int64_t)sc.n_sweeps * p / parts), s1 = (int)((int64_t)sc.n_sweeps * (p + 1) / parts);
    for (int s = s0; s < s1; ++s) off[s] += (int64_t)all.size();
    all.insert(all.end(), chunk[p].begin(), chunk[p].end());
    std::vector<uint32_t>().swap(chunk[p]);
  }
  int32_t max_len = 0;
  for (int s = 0; s < sc.n_sweeps; ++s) max_len = std::max(max_len, len[s]);
  QP_TRY(e->thr.ensure(all.size() * 4));
  QP_TRY(e->off.ensure(off.size() * 8));
  QP_TRY(e->len.ensure(len.size() * 4));
  QP_TRY(e->c.ensure(cf.size() * 4));
  QP_CU(cudaMemcpy(e->c.p, cf.data(), cf.size() * 4, cudaMemcpyHostToDevice));
  QP_CU(cudaMemcpy(e->thr.p, all.data(), all.size() * 4, cudaMemcpyHostToDevice));
  QP_CU(cudaMemcpy(e->off.p, off.data(), off.size() * 8, cudaMemcpyHostToDevice));
  QP_CU(cudaMemcpy(e->len.p, len.data(), len.size() * 4, cudaMemcpyHostToDevice));
  e->view.thr = e->thr.as<uint32_t>();
  e->view.off = e->off.as<int64_t>();
  e->view.len = e->len.as<int32_t>();
  e->view.c = e->c.as<float>();
  e->view.n_sweeps = sc.n_sweeps;
  e->view.max_len = max_len;
  e->view.total = (int64_t)all.size();
  e->bytes = all.size() * 4 + off.size() * 8 + len.size() * 4 + cf.size() * 4;
  e->last_use = ++g_sched_clock;
  // make room: drop the least recently used schedules (their holders keep them alive)
  const size_t limit = sched_cache_limit();
  while (g_sched_bytes + e->bytes > limit && !g_sched.empty()) {
    auto lru = g_sched.begin();
    for (auto j = g_sched.begin(); j != g_sched.end(); ++j)
      if (j->second->last_use < lru->second->last_use) lru = j;
    g_sched_bytes -= lru->second->bytes;
    g_sched.erase(lru);
  }
  *out = e->view;
  if (keep) *keep = e;
  g_sched_bytes += e->bytes;
  g_sched.emplace(key, std::move(e));
  return QP_OK;
}

}  // namespace host
}  // namespace qp

namespace {

qp_status upload_bits(qp_handle *h, const std::vector<uint8_t> &fr, const std::vector<uint8_t> &fv) {
  const int64_t nw = (h->n + 31) / 32;
  std::vector<uint32_t> fb(nw, 0), vb(nw, 0);
  for (int64_t k = 0; k < h->n; ++k) {
    if (fr[k]) fb[k >> 5] |= 1u << (k & 31);
    if (fr[k] && fv[k]) vb[k >> 5] |= 1u << (k & 31);
  }
  QP_TRY(h->frozen_bits.ensure(nw * 4));
  QP_TRY(h->fval_bits.ensure(nw * 4));
  QP_CU(cudaMemcpy(h->frozen_bits.p, fb.data(), nw * 4, cudaMemcpyHostToDevice));
  QP_CU(cudaMemcpy(h->fval_bits.p, vb.data(), nw * 4, cudaMemcpyHostToDevice));
  return QP_OK;
}

}  // namespace

// --------------------------------------------------------------------------- build
// The path QUBO of a field; w (host, n_legs entries) replaces B on the
// distance term leg by leg when given (the dense form only).
static qp_status build_field_qubo(const qp_field *f, int32_t A, int32_t B, int32_t scale, int32_t flags,
                                  const int32_t *w, int32_t n_legs, qp_handle **out) {
  g_err.clear();
  if (!f || !out) return fail(QP_EINVAL, "field and out must not be NULL");
  *out = nullptr;
  if (f->rows < 1 || f->cols < 1 || (int64_t)f->rows * f->cols > (1 << 24))
    return fail(QP_EINVAL, "bad grid size %d x %d", f->rows, f->cols);
  if (B < 0 || scale < 1) return fail(QP_EINVAL, "need B >= 0 and scale >= 1");
  if (w && is_device_ptr(w)) return fail(QP_EINVAL, "leg weights must be host memory");
  if (f->start < 0 || f->start >= f->rows * f->cols) return fail(QP_EINVAL, "start out of the grid");
  if (f->free_mask && !f->free_mask[f->start]) return fail(QP_EINVAL, "start cell is an obstacle");
  if (flags == 0) flags = QP_STRUCTURED;
  if (flags & ~(QP_DENSE | QP_STRUCTURED | QP_DIST_I16)) return fail(QP_EINVAL, "unknown flags 0x%x", flags);

  auto h = std::make_unique<qp_handle>();
  QP_CU(cudaGetDevice(&h->dev));
  noalloc_preload();
  std::vector<int32_t> cr, cc;
  for (int r = 0; r < f->rows; ++r)
    for (int c = 0; c < f->cols; ++c) {
      const int g = r * f->cols + c;
      if (f->free_mask && !f->free_mask[g]) continue;
      if (g == f->start) h->start = (int32_t)cr.size();
      cr.push_back(r);
      cc.push_back(c);
    }
  const int C = (int)cr.size();
  if (C < 2) return fail(QP_EINVAL, "a field needs at least 2 free cells (has %d)", C);
  if (C > kMaxCells) return fail(QP_ERANGE, "%d cells exceed the limit %d", C, kMaxCells);
  int64_t maxw = B;  // the largest weight on any leg
  if (w) {
    if (n_legs != C - 1) return fail(QP_EINVAL, "need C - 1 = %d leg weights (got %d)", C - 1, n_legs);
    maxw = 0;
    for (int t = 0; t < C - 1; ++t) {
      if (w[t] < 0) return fail(QP_EINVAL, "leg weight %d is negative", t);
      maxw = std::max<int64_t>(maxw, w[t]);
    }
    flags |= QP_DENSE;
    h->weighted = true;
  }
  h->path = true;
  h->C = C;
  h->n = (int64_t)C * C;
  h->d.resize((size_t)C * C);
  int64_t maxd = 0;
  for (int i = 0; i < C; ++i)
    for (int j = 0; j < C; ++j) {
      const int64_t dr = cr[i] - cr[j], dc = cc[i] - cc[j];
      const int64_t v = round_scaled_sqrt(dr * dr + dc * dc, scale);
      if (v > INT32_MAX) return fail(QP_ERANGE, "distance beyond int32");
      h->d[(size_t)i * C + j] = (int32_t)v;
      maxd = std::max(maxd, v);
    }
  h->max_d = (int32_t)maxd;
  const int64_t Aeff = A > 0 ? A : 2 * maxd * (w ? std::max<int64_t>(1, maxw) : 1);
  if (Aeff > INT32_MAX / 4) return fail(QP_ERANGE, "penalty A beyond int32/4");
  h->A = (int32_t)Aeff;
  h->B = B;
  h->c0 = 2 * (int64_t)h->A * C;
  // |dE| <= B * max_d * 2C + 2A(2C + 1) must fit int32 (B: the largest leg weight)
  const double bound = (double)maxw * maxd * 2.0 * C + 2.0 * h->A * (2.0 * C + 1.0);
  if (bound >= 2147483647.0) return fail(QP_ERANGE, "|dE| bound %.3g exceeds int32", bound);

  h->Cp = round_up_i(C, 8);
  h->d_i16 = (flags & QP_DIST_I16) || maxd <= 32767;
  if (h->d_i16 && maxd > 32767) return fail(QP_ERANGE, "QP_DIST_I16 but max d = %lld", (long long)maxd);
  // device copies of d
  QP_TRY(h->d32_dev.ensure((size_t)C * C * 4));
  QP_CU(cudaMemcpy(h->d32_dev.p, h->d.data(), (size_t)C * C * 4, cudaMemcpyHostToDevice));
  {
    const size_t es = h->d_i16 ? 2 : 4;
    std::vector<uint8_t> pad((size_t)C * h->Cp * es, 0);
    for (int i = 0; i < C; ++i)
      for (int j = 0; j < C; ++j) {
        const int32_t v = h->d[(size_t)i * C + j];
        if (h->d_i16) reinterpret_cast<int16_t *>(pad.data())[(size_t)i * h->Cp + j] = (int16_t)v;
        else reinterpret_cast<int32_t *>(pad.data())[(size_t)i * h->Cp + j] = v;
      }
    QP_TRY(h->d_dev.ensure(pad.size()));
    QP_CU(cudaMemcpy(h->d_dev.p, pad.data(), pad.size(), cudaMemcpyHostToDevice));
  }
  if (flags & QP_DENSE) {
    if (h->n > 65536) return fail(QP_ERANGE, "dense form of %lld variables is too large", (long long)h->n);
    const int64_t maxS = std::max<int64_t>(2 * (int64_t)h->A, maxw * maxd);
    h->S_i16 = maxS <= 32767;
    h->np = round_up_i((int)h->n, 8);
    QP_TRY(h->S_dev.ensure((size_t)h->n * h->np * (h->S_i16 ? 2 : 4)));
    DevBuf w_dev;
    if (w) {
      QP_TRY(w_dev.ensure((size_t)(C - 1) * 4));
      QP_CU(cudaMemcpy(w_dev.p, w, (size_t)(C - 1) * 4, cudaMemcpyHostToDevice));
    }
    QP_CU(launch_build_dense(h->S_dev.p, h->S_i16, h->np, C, h->d32_dev.as<int32_t>(), h->A, B, 0,
                             w ? w_dev.as<int32_t>() : nullptr));
    QP_CU(cudaDeviceSynchronize());
    std::vector<uint8_t> fr(h->n, 0), fv(h->n, 0);
    for (int t = 0; t < C; ++t)
      for (int i = 0; i < C; ++i)
        if (t == 0 || i == h->start) {
          fr[(size_t)t * C + i] = 1;
          fv[(size_t)t * C + i] = (t == 0 && i == h->start);
        }
    QP_TRY(upload_bits(h.get(), fr, fv));
    h->has_dense = true;
  }
  *out = h.release();
  return QP_OK;
}

extern "C" qp_status qp_build_qubo(const qp_field *f, int32_t A, int32_t B, int32_t scale, int32_t flags,
                                   qp_handle **out) {
  return build_field_qubo(f, A, B, scale, flags, nullptr, 0, out);
}

extern "C" qp_status qp_build_qubo_weighted(const qp_field *f, int32_t A, const int32_t *leg_weights,
                                            int32_t n_legs, int32_t scale, qp_handle **out) {
  if (!leg_weights) {
    g_err.clear();
    return fail(QP_EINVAL, "leg_weights must not be NULL");
  }
  return build_field_qubo(f, A, 1, scale, QP_STRUCTURED | QP_DENSE, leg_weights, n_legs, out);
}

extern "C" qp_status qp_build_from_dense(const int32_t *S, int64_t n, const uint8_t *frozen,
                                         const uint8_t *frozen_val, int64_t c0, qp_handle **out) {
  g_err.clear();
  if (!S || !out) return fail(QP_EINVAL, "S and out must not be NULL");
  *out = nullptr;
  if (n < 1 || n > 65536) return fail(QP_EINVAL, "need 1 <= n <= 65536 (got %lld)", (long long)n);
  if (is_device_ptr(S)) return fail(QP_EINVAL, "S must be host memory");
  auto h = std::make_unique<qp_handle>();
  QP_CU(cudaGetDevice(&h->dev));
  h->n = n;
  h->c0 = c0;
  int64_t maxabs = 0;
  for (int64_t k = 0; k < n; ++k) {
    int64_t rowabs = 0;
    for (int64_t l = 0; l < n; ++l) {
      const int32_t v = S[k * n + l];
      if (v != S[l * n + k]) return fail(QP_EINVAL, "S is not symmetric at (%lld, %lld)", (long long)k, (long long)l);
      rowabs += std::llabs((long long)v);
      maxabs = std::max<int64_t>(maxabs, std::llabs((long long)v));
    }
    if (rowabs > INT32_MAX) return fail(QP_ERANGE, "row %lld of S has absolute sum beyond int32", (long long)k);
  }
  h->S_i16 = maxabs <= 32767;
  h->np = round_up_i((int)n, 8);
  const size_t es = h->S_i16 ? 2 : 4;
  std::vector<uint8_t> pad((size_t)n * h->np * es, 0);
  for (int64_t k = 0; k < n; ++k)
    for (int64_t l = 0; l < n; ++l) {
      if (h->S_i16) reinterpret_cast<int16_t *>(pad.data())[k * h->np + l] = (int16_t)S[k * n + l];
      else reinterpret_cast<int32_t *>(pad.data())[k * h->np + l] = S[k * n + l];
    }
  QP_TRY(h->S_dev.ensure(pad.size()));
  QP_CU(cudaMemcpy(h->S_dev.p, pad.data(), pad.size(), cudaMemcpyHostToDevice));
  h->frozen_host.assign(n, 0);
  h->fval_host.assign(n, 0);
  for (int64_t k = 0; k < n; ++k) {
    h->frozen_host[k] = frozen ? (frozen[k] != 0) : 0;
    h->fval_host[k] = (frozen && frozen[k] && frozen_val) ? (frozen_val[k] != 0) : 0;
  }
  QP_TRY(upload_bits(h.get(), h->frozen_host, h->fval_host));
  h->has_dense = true;
  *out = h.release();
  return QP_OK;
}

extern "C" qp_status qp_qubo_info(const qp_handle *h, int64_t *n_vars, int32_t *n_cells,
                                  int64_t *c0, int32_t *max_d, int32_t *A_used) {
  if (!h) return fail(QP_EINVAL, "handle is NULL");
  if (n_vars) *n_vars = h->n;
  if (n_cells) *n_cells = h->path ? h->C : 0;
  if (c0) *c0 = h->c0;
  if (max_d) *max_d = h->max_d;
  if (A_used) *A_used = h->A;
  return QP_OK;
}

extern "C" qp_status qp_export_dist(const qp_handle *h, int32_t *d_out) {
  if (!h || !d_out) return fail(QP_EINVAL, "handle and d_out must not be NULL");
  if (!h->path) return fail(QP_EINVAL, "a generic QUBO has no distance matrix");
  std::memcpy(d_out, h->d.data(), h->d.size() * 4);
  return QP_OK;
}

extern "C" qp_status qp_export_dense(const qp_handle *h, int32_t *S_out) {
  if (!h || !S_out) return fail(QP_EINVAL, "handle and S_out must not be NULL");
  if (!h->has_dense) return fail(QP_EINVAL, "handle was built without QP_DENSE");
  DevSet ds(h->dev);
  const size_t es = h->S_i16 ? 2 : 4;
  std::vector<uint8_t> tmp((size_t)h->n * h->np * es);
  QP_CU(cudaMemcpy(tmp.data(), h->S_dev.p, tmp.size(), cudaMemcpyDeviceToHost));
  for (int64_t k = 0; k < h->n; ++k)
    for (int64_t l = 0; l < h->n; ++l)
      S_out[k * h->n + l] = h->S_i16 ? reinterpret_cast<int16_t *>(tmp.data())[k * h->np + l]
                                     : reinterpret_cast<int32_t *>(tmp.data())[k * h->np + l];
  return QP_OK;
}

extern "C" qp_status qp_device_checks(int32_t *enabled, uint32_t *first_failure) {
  g_err.clear();
  if (!enabled || !first_failure) return fail(QP_EINVAL, "enabled and first_failure are required");
  *enabled = qp::chk::enabled();
  uint32_t w = 0;
  bool read_failed = false;
  for (uint32_t (*take)() : {qp::chk::rows, qp::chk::kernels, qp::chk::group, qp::chk::repair}) {
    const uint32_t v = take();
    if (v == 0xFFFFFFFFu) {  // the record could not be read from the device
      read_failed = true;
      continue;
    }
    if (!w) w = v;
  }
  *first_failure = w;
  if (read_failed) return fail(QP_ECUDA, "could not read the device check record");
  return QP_OK;
}

extern "C" qp_status qp_thresholds(const qp_schedule *sc, int32_t sweep, uint32_t *out, int32_t cap,
                                   int32_t *len_out) {
  g_err.clear();
  if (!sc) return fail(QP_EINVAL, "schedule is NULL");
  if (sc->n_sweeps < 1 || sweep < 0 || sweep >= sc->n_sweeps) return fail(QP_EINVAL, "sweep out of range");
  if (!(sc->T0 > 0.0) || !(sc->T1 > 0.0)) return fail(QP_EINVAL, "temperatures must be > 0");
  std::vector<uint32_t> tab;
  build_thresholds(temperature(*sc, sweep), tab);
  if (len_out) *len_out = (int32_t)tab.size();
  if (!out) return QP_OK;
  if (cap < (int32_t)tab.size()) return fail(QP_ERANGE, "cap %d < len %zu", cap, tab.size());
  std::memcpy(out, tab.data(), tab.size() * 4);
  return QP_OK;
}

// --------------------------------------------------------------------------- anneal
namespace qp {
namespace host {

// The structured sweep of a.R replicas: the row kernel when allowed and the
// field fits it, else the flat kernel (spins in global memory when a
// replica's bitset does not fit shared memory comfortably).
qp_status launch_structured_auto(qp_handle *h, StructArgs &a, int W, bool allow_rows, cudaStream_t st,
                                 LaunchInfo *info, bool rows_shared_spins) {
  if (allow_rows && !rows_shared_spins && rows_g_supported(h->C, h->d_i16, 1)) {
    int Wg = W > 0 ? W : rows_g_auto_warps(h->C, h->d_i16, a.R);
    while (Wg > 1 && !rows_g_supported(h->C, h->d_i16, Wg)) --Wg;
    QP_TRY(h->gstate.ensure((size_t)a.R * rows_g_words(h->C) * 4));
    a.gstate = h->gstate.as<uint32_t>();
    QP_TRY(h->rg_aux.ensure((size_t)(2 + a.R) * 4));
    QP_TRY(h->rg_carry.ensure((size_t)a.R * 16));
    QP_TRY(h->kernel_err.ensure(4));
    QP_CU(cudaMemsetAsync(h->rg_aux.p, 0, (size_t)(2 + a.R) * 4, st));
    int *aux = h->rg_aux.as<int>();
    QP_CU(launch_rows_g(a, h->d_i16, Wg, aux, aux + 2, h->rg_carry.as<long long>(), h->kernel_err.as<int>(), st,
                        info));
    return QP_OK;
  }
  if (allow_rows) {
    int Wr = W > 0 ? W : rows_auto_warps(h->C, h->d_i16, a.R);
    while (Wr > 1 && !rows_supported(h->C, h->d_i16, Wr)) --Wr;
    if (rows_supported(h->C, h->d_i16, Wr)) {
      QP_CU(launch_rows(a, h->d_i16, Wr, st, info));
      return QP_OK;
    }
  }
  if (W <= 0) W = 4;
  a.nw_pad = (int32_t)structured_gstate_words(h->C);
  const bool want_smem = structured_state_fits_smem(h->C, h->d_i16, W) &&
                         4 * structured_gstate_words(h->C) <= 8 * 1024;
  if (!want_smem) {
    QP_TRY(h->gstate.ensure((size_t)a.R * a.nw_pad * 4));
    a.gstate = h->gstate.as<uint32_t>();
  }
  QP_CU(launch_structured(a, h->d_i16, W, want_smem, st, info));
  return QP_OK;
}

}  // namespace host
}  // namespace qp

extern "C" qp_status qp_anneal_ex(qp_handle *h, int32_t R, const qp_schedule *sc, uint64_t seed,
                                  const uint8_t *init, uint8_t *states_out, int64_t *energies_out,
                                  int64_t *best_out, const qp_anneal_opts *opts, void *stream_) {
  g_err.clear();
  if (!h) return fail(QP_EINVAL, "handle is NULL");
  if (R < 1) return fail(QP_EINVAL, "replicas must be >= 1");
  if (!states_out || !energies_out) return fail(QP_EINVAL, "states_out and energies_out are required");
  QP_TRY(check_schedule(sc));
  qp_anneal_opts o{};
  if (opts) o = *opts;
  if (o.replica_offset < 0 || (int64_t)o.replica_offset + R > INT32_MAX)
    return fail(QP_EINVAL, "replica_offset out of range");
  int kernel = o.kernel;
  if (kernel == QP_KERNEL_AUTO) kernel = h->path && !h->weighted ? QP_KERNEL_STRUCTURED : QP_KERNEL_DENSE;
  const bool structured = kernel == QP_KERNEL_STRUCTURED || kernel == QP_KERNEL_STRUCTURED_FLAT ||
                          kernel == QP_KERNEL_STRUCTURED_ROWS || kernel == QP_KERNEL_STRUCTURED_GROUP ||
                          kernel == QP_KERNEL_STRUCTURED_ROWS_SHARED;
  if (structured && !h->path) return fail(QP_EINVAL, "no structured form in this handle");
  if (structured && h->weighted)
    return fail(QP_EINVAL, "a handle with leg weights anneals with the dense kernel (the structured form is unweighted)");
  if (kernel == QP_KERNEL_DENSE && !h->has_dense) return fail(QP_EINVAL, "handle was built without QP_DENSE");
  if (!structured && kernel != QP_KERNEL_DENSE) return fail(QP_EINVAL, "unknown kernel %d", kernel);
  if (o.replicas_per_cta < 0 || o.replicas_per_cta > kMaxWarpsPerCta)
    return fail(QP_EINVAL, "replicas_per_cta must be in [0, %d]", kMaxWarpsPerCta);

  DevSet ds(h->dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  DeviceSchedule sched;
  std::shared_ptr<const void> sched_keep;  // the tables stay alive until the launch is queued
  QP_TRY(device_schedule(*sc, &sched, &sched_keep));
  const size_t n = (size_t)h->n;

  QP_DEV_FITS(init, (size_t)R * n, "init_states");
  QP_DEV_FITS(states_out, (size_t)R * n, "states_out");
  QP_DEV_FITS(energies_out, (size_t)R * 8, "energies_out");
  QP_DEV_FITS(best_out, (size_t)R * 8, "best_out");
  QP_DEV_FITS(o.accepts_out, (size_t)R * 8, "accepts_out");
  // stage host buffers
  const uint8_t *init_d = init;
  if (init && !is_device_ptr(init)) {
    QP_TRY(h->in_stage.ensure((size_t)R * n));
    QP_CU(cudaMemcpyAsync(h->in_stage.p, init, (size_t)R * n, cudaMemcpyHostToDevice, st));
    init_d = h->in_stage.as<uint8_t>();
  }
  const bool st_host = !is_device_ptr(states_out);
  const bool e_host = !is_device_ptr(energies_out);
  const bool b_host = best_out && !is_device_ptr(best_out);
  const bool a_host = o.accepts_out && !is_device_ptr(o.accepts_out);
  uint8_t *st_d = states_out;
  int64_t *e_d = energies_out, *b_d = best_out, *a_d = o.accepts_out;
  if (st_host) { QP_TRY(h->st_stage.ensure((size_t)R * n)); st_d = h->st_stage.as<uint8_t>(); }
  if (e_host) { QP_TRY(h->e_stage.ensure((size_t)R * 8)); e_d = h->e_stage.as<int64_t>(); }
  if (b_host) { QP_TRY(h->b_stage.ensure((size_t)R * 8)); b_d = h->b_stage.as<int64_t>(); }
  if (a_host) { QP_TRY(h->a_stage.ensure((size_t)R * 8)); a_d = h->a_stage.as<int64_t>(); }
  const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);

  LaunchInfo info;
  bool err_armed = false;
  if (structured) {
    int W = o.replicas_per_cta ? o.replicas_per_cta : 4;
    StructArgs a{};
    a.C = h->C; a.Cp = h->Cp; a.start = h->start; a.A = h->A; a.B = h->B;
    a.d = h->d_dev.p;
    a.R = R; a.rep_offset = o.replica_offset;
    a.sweep_begin = sc->sweep_begin; a.sweep_end = sc->sweep_end;
    a.key0 = key0; a.key1 = key1;
    a.thr = sched.thr; a.thr_off = sched.off; a.thr_len = sched.len; a.thr_c = sched.c;
    a.init = init_d; a.states_out = st_d; a.E_out = e_d; a.best_out = b_d; a.acc_out = a_d;
    a.skip_settled = (o.flags & QP_ANNEAL_SKIP_SETTLED) ? 1 : 0;
    if (kernel == QP_KERNEL_STRUCTURED_GROUP) {
      if (group_size_for(h->C) < 2) return fail(QP_EINVAL, "the grouped kernel takes fields of up to 128 cells");
      int Wg = W;
      while (Wg > 1 && !group_supported(h->C, h->d_i16, Wg)) --Wg;
      if (!group_supported(h->C, h->d_i16, Wg)) return fail(QP_ERANGE, "grouped kernel: no launch fits");
      QP_CU(launch_group(a, h->d_i16, Wg, st, &info));
      goto launched;
    }
    // replicas per CTA as asked, else chosen for the most resident chains
    QP_TRY(h->kernel_err.ensure(4));
    QP_CU(cudaMemsetAsync(h->kernel_err.p, 0, 4, st));
    err_armed = true;
    QP_TRY(launch_structured_auto(h, a, o.replicas_per_cta, kernel != QP_KERNEL_STRUCTURED_FLAT, st, &info,
                                  kernel == QP_KERNEL_STRUCTURED_ROWS_SHARED));
  } else {
    int W = o.replicas_per_cta ? o.replicas_per_cta : 4;
    while (W > 1 && !dense_h_fits_smem(h->n, h->path ? h->C : 0, W)) --W;
    DenseArgs a{};
    a.n = h->n; a.np = h->np; a.S = h->S_dev.p; a.c0 = h->c0; a.C = h->path ? h->C : 0;
    a.frozen_bits = h->frozen_bits.as<uint32_t>(); a.fval_bits = h->fval_bits.as<uint32_t>();
    a.R = R; a.rep_offset = o.replica_offset;
    a.sweep_begin = sc->sweep_begin; a.sweep_end = sc->sweep_end;
    a.key0 = key0; a.key1 = key1;
    a.thr = sched.thr; a.thr_off = sched.off; a.thr_len = sched.len; a.thr_c = sched.c;
    a.init = init_d; a.states_out = st_d; a.E_out = e_d; a.best_out = b_d; a.acc_out = a_d;
    if (!dense_h_fits_smem(h->n, a.C, W)) {
      QP_TRY(h->hbuf.ensure((size_t)R * h->np * 4));
      a.hbuf = h->hbuf.as<int32_t>();
    }
    QP_TRY(h->kernel_err.ensure(4));
    QP_CU(cudaMemsetAsync(h->kernel_err.p, 0, 4, st));
    a.err = h->kernel_err.as<int32_t>();
    QP_CU(launch_dense(a, h->S_i16, W, st, &info));
    err_armed = true;
  }
launched:
  if (st_host) QP_CU(cudaMemcpyAsync(states_out, st_d, (size_t)R * n, cudaMemcpyDeviceToHost, st));
  if (e_host) QP_CU(cudaMemcpyAsync(energies_out, e_d, (size_t)R * 8, cudaMemcpyDeviceToHost, st));
  if (b_host) QP_CU(cudaMemcpyAsync(best_out, b_d, (size_t)R * 8, cudaMemcpyDeviceToHost, st));
  if (a_host) QP_CU(cudaMemcpyAsync(o.accepts_out, a_d, (size_t)R * 8, cudaMemcpyDeviceToHost, st));
  if (st_host || e_host || b_host || a_host || (init && init_d != init)) {
    QP_CU(cudaStreamSynchronize(st));
    if (err_armed) {
      int32_t err = 0;
      QP_CU(cudaMemcpy(&err, h->kernel_err.p, 4, cudaMemcpyDeviceToHost));
      if (err) return fail(QP_ETIMEOUT, "a bounded device wait gave up (a bulk row copy of the dense sweep, or "
                                        "a chain segment of the row kernel); the affected replicas report "
                                        "energy INT64_MIN");
    }
  }
  return QP_OK;
}

extern "C" qp_status qp_anneal(qp_handle *h, int32_t R, const qp_schedule *sc, uint64_t seed,
                               const uint8_t *init, uint8_t *states_out, int64_t *energies_out,
                               int64_t *best_out, void *stream) {
  return qp_anneal_ex(h, R, sc, seed, init, states_out, energies_out, best_out, nullptr, stream);
}

// --------------------------------------------------------------------------- decode
extern "C" qp_status qp_decode_path(const qp_handle *h, const uint8_t *state, int32_t *path_out,
                                    int64_t *length_out) {
  g_err.clear();
  if (!h || !state || !path_out || !length_out) return fail(QP_EINVAL, "NULL argument");
  if (!h->path) return fail(QP_EINVAL, "a generic QUBO has no path");
  const int C = h->C;
  std::vector<uint8_t> x;
  const uint8_t *xs = state;
  if (is_device_ptr(state)) {
    DevSet ds(h->dev);
    x.resize((size_t)C * C);
    QP_CU(cudaMemcpy(x.data(), state, x.size(), cudaMemcpyDeviceToHost));
    xs = x.data();
  }
  std::vector<int32_t> path(C, -1), colcnt(C, 0);
  for (int t = 0; t < C; ++t) {
    int cnt = 0;
    for (int i = 0; i < C; ++i)
      if (xs[(size_t)t * C + i]) {
        ++cnt;
        path[t] = i;
        ++colcnt[i];
      }
    if (cnt != 1) return fail(QP_EINFEASIBLE, "step %d has %d cells", t, cnt);
  }
  for (int i = 0; i < C; ++i)
    if (colcnt[i] != 1) return fail(QP_EINFEASIBLE, "cell %d is visited %d times", i, colcnt[i]);
  int64_t L = 0;
  for (int t = 0; t + 1 < C; ++t) L += h->d[(size_t)path[t] * C + path[t + 1]];
  std::memcpy(path_out, path.data(), C * 4);
  *length_out = L;
  return QP_OK;
}

extern "C" qp_status qp_decode_batch(const qp_handle *hc, int32_t R, const uint8_t *states,
                                     int32_t *paths_out, int64_t *lengths_out, void *stream_) {
  g_err.clear();
  qp_handle *h = const_cast<qp_handle *>(hc);
  if (!h || !states || !paths_out || !lengths_out || R < 1) return fail(QP_EINVAL, "bad argument");
  if (!h->path) return fail(QP_EINVAL, "a generic QUBO has no path");
  DevSet ds(h->dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  const size_t n = (size_t)h->n;
  QP_DEV_FITS(states, (size_t)R * n, "states");
  QP_DEV_FITS(paths_out, (size_t)R * h->C * 4, "paths_out");
  QP_DEV_FITS(lengths_out, (size_t)R * 8, "lengths_out");
  const uint8_t *sd = states;
  bool sync = false;
  if (!is_device_ptr(states)) {
    QP_TRY(h->in_stage.ensure((size_t)R * n));
    QP_CU(cudaMemcpyAsync(h->in_stage.p, states, (size_t)R * n, cudaMemcpyHostToDevice, st));
    sd = h->in_stage.as<uint8_t>();
    sync = true;
  }
  int32_t *pd = paths_out;
  int64_t *ld = lengths_out;
  const bool ph = !is_device_ptr(paths_out), lh = !is_device_ptr(lengths_out);
  if (ph) { QP_TRY(h->p_stage.ensure((size_t)R * h->C * 4)); pd = h->p_stage.as<int32_t>(); }
  if (lh) { QP_TRY(h->l_stage.ensure((size_t)R * 8)); ld = h->l_stage.as<int64_t>(); }
  QP_CU(launch_decode(sd, R, h->C, h->d32_dev.as<int32_t>(), pd, ld, st));
  if (ph) QP_CU(cudaMemcpyAsync(paths_out, pd, (size_t)R * h->C * 4, cudaMemcpyDeviceToHost, st));
  if (lh) QP_CU(cudaMemcpyAsync(lengths_out, ld, (size_t)R * 8, cudaMemcpyDeviceToHost, st));
  if (sync || ph || lh) QP_CU(cudaStreamSynchronize(st));
  return QP_OK;
}

extern "C" void qp_destroy(qp_handle *h) {
  if (!h) return;
  DevSet ds(h->dev);
  delete h;
}

extern "C" const char *qp_last_error(void) { return g_err.c_str(); }

// --------------------------------------------------------------------------- lookups that never allocate
namespace qp {

bool handle_struct_view(const qp_handle *h, StructView *out) {
  if (!h || !h->path) return false;
  out->dev = h->dev;
  out->C = h->C;
  out->Cp = h->Cp;
  out->start = h->start;
  out->A = h->A;
  out->B = h->B;
  out->d = h->d_dev.p;
  out->d_i16 = h->d_i16;
  out->max_d = h->max_d;
  out->d32 = h->d32_dev.as<int32_t>();
  out->weighted = h->weighted;
  return true;
}

bool schedule_lookup(const qp_schedule &sc, DeviceSchedule *out, std::shared_ptr<const void> *keep) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  const SchedKey key = key_of(dev, sc);
  std::lock_guard<std::mutex> lk(g_sched_mu);
  auto it = g_sched.find(key);
  if (it == g_sched.end()) return false;
  it->second->last_use = ++g_sched_clock;
  *out = it->second->view;
  if (keep) *keep = it->second;
  return true;
}

qp_status set_error(qp_status s, const char *msg) { return fail(s, "%s", msg); }

void clear_error() { g_err.clear(); }

bool device_pointer(const void *p) { return is_device_ptr(p); }

namespace {
using GetAddressRange = int (*)(unsigned long long *, size_t *, unsigned long long);
GetAddressRange address_range_fn() {
  static std::once_flag once;
  static GetAddressRange fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<GetAddressRange>(p);
    else
      cudaGetLastError();
  });
  return fn;
}
}  // namespace

bool device_range_fits(const void *p, size_t bytes) {
  if (!p || bytes == 0) return true;
  GetAddressRange fn = address_range_fn();
  if (!fn) return true;
  unsigned long long base = 0;
  size_t size = 0;
  const unsigned long long a = reinterpret_cast<uintptr_t>(p);
  if (fn(&base, &size, a) != 0) return true;  // not an allocation the driver knows: cannot tell
  return a >= base && a - base <= size && bytes <= size - (a - base);
}

}  // namespace qp

