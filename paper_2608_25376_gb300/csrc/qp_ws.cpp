// Host side of the learned warm start: per-cell features of a field, the MLP
// (16 -> 256 -> 256 -> 256 -> 256 step logits, bf16 weights with fp32 masters
// and Adam moments), its forward pass, one training step (forward, softmax
// cross-entropy, backward, Adam) built from the tcgen05 GEMM and the small
// kernels of qp_mlp.cu, and the greedy decode of step logits into a feasible
// one-hot state.  The public contract is in include/qpath.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "qp_internal.h"
#include "qp_mlp.h"

using namespace qp;

namespace {

constexpr int kIn = 16, kHid = 256, kOut = 256;
constexpr int kLayers = 4;
const int kDimIn[kLayers] = {kIn, kHid, kHid, kHid};
const int kDimOut[kLayers] = {kHid, kHid, kHid, kOut};

struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
  ~Buf() {
    if (p) cudaFree(p);
  }
  bool ensure(size_t want) {
    if (want <= bytes) return true;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    if (dev_malloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return false;
    }
    bytes = want;
    return true;
  }
  template <typename T>
  T *as() const { return static_cast<T *>(p); }
};

#define WS_CU(call)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return set_error(QP_ECUDA, cudaGetErrorString(e_));        \
  } while (0)
#define WS_ALLOC(buf, bytes)                                                          \
  do {                                                                                \
    if (!(buf).ensure(bytes)) return set_error(QP_ENOMEM, "warm start: cudaMalloc failed"); \
  } while (0)

uint16_t f32_to_bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);  // inf / nan
  u += 0x7FFFu + ((u >> 16) & 1u);                                     // round half to even
  return (uint16_t)(u >> 16);
}

uint64_t splitmix64(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct qp_ws {
  int dev = 0;
  int step = 0;
  Buf w[kLayers], b[kLayers];          // fp32 masters
  Buf mw[kLayers], vw[kLayers], mb[kLayers], vb[kLayers];
  Buf gw[kLayers], gb[kLayers];        // fp32 gradients
  Buf wb[kLayers], wt[kLayers];        // bf16 weight and its transpose
  int cap = 0;                         // rows the activation buffers hold
  int fwd_mode = QP_WS_FORWARD_FUSED;
  Buf x0, h[3], z, dz, dh[3], t1, t2, lab, stp, loss, err;
  Buf gws, cws, lrow;  // split-K partials, column-sum partials, per-row losses (fixed-order sums)
};

namespace {

size_t n_params() {
  size_t n = 0;
  for (int l = 0; l < kLayers; ++l) n += (size_t)kDimOut[l] * kDimIn[l] + kDimOut[l];
  return n;
}

qp_status ensure_rows(qp_ws *m, int Mp) {
  if (Mp <= m->cap) return QP_OK;
  m->cap = 0;  // a failed growth below leaves some buffers empty: check them all next time
  WS_ALLOC(m->x0, (size_t)Mp * kIn * 2);
  for (int i = 0; i < 3; ++i) {
    WS_ALLOC(m->h[i], (size_t)Mp * kHid * 2);
    WS_ALLOC(m->dh[i], (size_t)Mp * kHid * 2);
  }
  WS_ALLOC(m->z, (size_t)Mp * kOut * 4);
  WS_ALLOC(m->dz, (size_t)Mp * kOut * 2);
  WS_ALLOC(m->t1, (size_t)Mp * kHid * 2);
  WS_ALLOC(m->t2, (size_t)Mp * kHid * 2);
  WS_ALLOC(m->lab, (size_t)Mp * 4);
  WS_ALLOC(m->stp, (size_t)Mp * 4);
  WS_ALLOC(m->lrow, (size_t)Mp * 4);
  WS_ALLOC(m->cws, (size_t)mlp::kColsumSlabs * kOut * 4);
  m->cap = Mp;
  return QP_OK;
}

// bf16 copies of every weight (and transposes) from the fp32 masters
qp_status refresh_bf16(qp_ws *m, cudaStream_t st) {
  for (int l = 0; l < kLayers; ++l) {
    const int rows = kDimOut[l], cols = kDimIn[l];
    std::vector<float> wh((size_t)rows * cols);
    WS_CU(cudaMemcpyAsync(wh.data(), m->w[l].p, wh.size() * 4, cudaMemcpyDeviceToHost, st));
    WS_CU(cudaStreamSynchronize(st));
    std::vector<uint16_t> a(wh.size()), t(wh.size());
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) {
        const uint16_t v = f32_to_bf16_bits(wh[(size_t)r * cols + c]);
        a[(size_t)r * cols + c] = v;
        t[(size_t)c * rows + r] = v;
      }
    WS_CU(cudaMemcpyAsync(m->wb[l].p, a.data(), a.size() * 2, cudaMemcpyHostToDevice, st));
    WS_CU(cudaMemcpyAsync(m->wt[l].p, t.data(), t.size() * 2, cudaMemcpyHostToDevice, st));
  }
  WS_CU(cudaStreamSynchronize(st));
  return QP_OK;
}

qp_status upload_inputs(qp_ws *m, const float *feats, int M, int Mp, const int32_t *labels, const int32_t *steps,
                        cudaStream_t st) {
  if (qp_status s = ensure_rows(m, Mp); s != QP_OK) return s;
  std::vector<uint16_t> xb((size_t)Mp * kIn, 0);
  for (size_t e = 0; e < (size_t)M * kIn; ++e) xb[e] = f32_to_bf16_bits(feats[e]);
  WS_CU(cudaMemcpyAsync(m->x0.p, xb.data(), xb.size() * 2, cudaMemcpyHostToDevice, st));
  if (labels && steps) {
    std::vector<int32_t> lb(Mp, -1), sp(Mp, 1);
    std::memcpy(lb.data(), labels, (size_t)M * 4);
    std::memcpy(sp.data(), steps, (size_t)M * 4);
    WS_CU(cudaMemcpyAsync(m->lab.p, lb.data(), (size_t)Mp * 4, cudaMemcpyHostToDevice, st));
    WS_CU(cudaMemcpyAsync(m->stp.p, sp.data(), (size_t)Mp * 4, cudaMemcpyHostToDevice, st));
    WS_CU(cudaStreamSynchronize(st));
  } else {
    WS_CU(cudaStreamSynchronize(st));
  }
  return QP_OK;
}

mlp::GemmArgs gargs(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N, int K,
                    int mode, int *err) {
  mlp::GemmArgs g{};
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.M = M; g.N = N; g.K = K; g.mode = mode; g.err = err;
  return g;
}

// Logits into m->z; the hidden activations into m->h[] when keep_hidden (the
// backward pass reads them) or when the layers run as separate launches.
qp_status forward(qp_ws *m, int Mp, bool keep_hidden, cudaStream_t st) {
  if (m->fwd_mode == QP_WS_FORWARD_FUSED) {
    mlp::FwdArgs g{};
    g.x0 = m->x0.as<__nv_bfloat16>();
    const __nv_bfloat16 *w[kLayers];
    for (int l = 0; l < kLayers; ++l) {
      g.bias[l] = m->b[l].as<float>();
      w[l] = m->wb[l].as<__nv_bfloat16>();
    }
    for (int l = 0; l < 3; ++l) g.h[l] = keep_hidden ? m->h[l].as<__nv_bfloat16>() : nullptr;
    g.z = m->z.as<float>();
    g.Mp = Mp;
    g.err = m->err.as<int>();
    WS_CU(mlp::forward(g, w, st));
    return QP_OK;
  }
  const __nv_bfloat16 *in = m->x0.as<__nv_bfloat16>();
  int ldin = kIn;
  for (int l = 0; l < kLayers; ++l) {
    mlp::GemmArgs g = gargs(in, ldin, m->wb[l].as<__nv_bfloat16>(), kDimIn[l], Mp, kDimOut[l], kDimIn[l],
                            l < 3 ? mlp::kEpiBiasRelu : mlp::kEpiBiasF32, m->err.as<int>());
    g.bias = m->b[l].as<float>();
    if (l < 3) {
      g.out_bf16 = m->h[l].as<__nv_bfloat16>();
      g.ldo = kHid;
    } else {
      g.out_f32 = m->z.as<float>();
      g.ldo = kOut;
    }
    WS_CU(mlp::gemm(g, 1, st));
    in = m->h[l < 3 ? l : 2].as<__nv_bfloat16>();
    ldin = kHid;
  }
  return QP_OK;
}

// Gradients of the mean cross-entropy into gw/gb (fp32); loss sum into m->loss.
// Every sum over rows is taken in a fixed order (split-K partials and slabs
// added in index order, no atomics), so a training run repeats bit for bit.
qp_status backward(qp_ws *m, int M, int Mp, cudaStream_t st) {
  WS_CU(mlp::softmax_ce(m->z.as<float>(), kOut, m->lab.as<int32_t>(), m->stp.as<int32_t>(), Mp, 1.0f / (float)M,
                        m->dz.as<__nv_bfloat16>(), kOut, m->lrow.as<float>(), m->loss.as<float>(), st));
  const __nv_bfloat16 *dy = m->dz.as<__nv_bfloat16>();
  const int splits = std::max(1, Mp / 512);
  WS_ALLOC(m->gws, (size_t)mlp::gemm_splits(Mp, splits) * kHid * kHid * 4);
  for (int l = kLayers - 1; l >= 0; --l) {
    const int nout = kDimOut[l], nin = kDimIn[l];
    const __nv_bfloat16 *x = l == 0 ? m->x0.as<__nv_bfloat16>() : m->h[l - 1].as<__nv_bfloat16>();
    // dW[out][in] = sum_m dY[m][out] X[m][in]  (operands transposed so m is contiguous)
    __nv_bfloat16 *dyt = m->t1.as<__nv_bfloat16>(), *xt = m->t2.as<__nv_bfloat16>();
    WS_CU(mlp::transpose(dy, Mp, nout, nout, dyt, Mp, st));
    WS_CU(mlp::transpose(x, Mp, nin, nin, xt, Mp, st));
    mlp::GemmArgs g = gargs(dyt, Mp, xt, Mp, nout, nin, Mp, mlp::kEpiPartialF32, m->err.as<int>());
    g.out_f32 = m->gws.as<float>();
    g.ldo = nin;
    WS_CU(mlp::gemm(g, splits, st));
    WS_CU(mlp::sum_splits(m->gws.as<float>(), mlp::gemm_splits(Mp, splits), nout * nin, m->gw[l].as<float>(), st));
    WS_CU(mlp::colsum(dy, nout, Mp, nout, m->cws.as<float>(), m->gb[l].as<float>(), st));
    if (l == 0) break;
    // dX[m][in] = relu'(X) * sum_out dY[m][out] W[out][in]  (B = W^T, out contiguous)
    mlp::GemmArgs gx = gargs(dy, nout, m->wt[l].as<__nv_bfloat16>(), nout, Mp, nin, nout, mlp::kEpiReluMask,
                             m->err.as<int>());
    gx.out_bf16 = m->dh[l - 1].as<__nv_bfloat16>();
    gx.ldo = nin;
    gx.relu_ref = x;
    gx.ldr = nin;
    WS_CU(mlp::gemm(gx, 1, st));
    dy = m->dh[l - 1].as<__nv_bfloat16>();
  }
  return QP_OK;
}

qp_status check_err(qp_ws *m, cudaStream_t st) {
  int e = 0;
  WS_CU(cudaMemcpyAsync(&e, m->err.p, 4, cudaMemcpyDeviceToHost, st));
  WS_CU(cudaStreamSynchronize(st));
  if (e) {
    WS_CU(cudaMemsetAsync(m->err.p, 0, 4, st));
    return set_error(QP_ETIMEOUT, "warm start: a tensor-core wait gave up");
  }
  return QP_OK;
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    int cur = 0;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev) {
      prev = cur;
      cudaSetDevice(dev);
    }
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" qp_status qp_ws_create(uint64_t seed, qp_ws **out) {
  if (!out) return set_error(QP_EINVAL, "out is NULL");
  *out = nullptr;
  qp_ws *m = new qp_ws();
  if (cudaGetDevice(&m->dev) != cudaSuccess) {
    delete m;
    return set_error(QP_ECUDA, "cudaGetDevice failed");
  }
  uint64_t s = seed;
  for (int l = 0; l < kLayers; ++l) {
    const int rows = kDimOut[l], cols = kDimIn[l];
    const size_t nw = (size_t)rows * cols;
    bool ok = m->w[l].ensure(nw * 4) && m->b[l].ensure(rows * 4) && m->mw[l].ensure(nw * 4) &&
              m->vw[l].ensure(nw * 4) && m->mb[l].ensure(rows * 4) && m->vb[l].ensure(rows * 4) &&
              m->gw[l].ensure(nw * 4) && m->gb[l].ensure(rows * 4) && m->wb[l].ensure(nw * 2) &&
              m->wt[l].ensure(nw * 2);
    if (!ok) {
      delete m;
      return set_error(QP_ENOMEM, "warm start: cudaMalloc failed");
    }
    // He-uniform initialisation from a splitmix64 stream
    const double lim = std::sqrt(6.0 / cols);
    std::vector<float> wh(nw);
    for (size_t e = 0; e < nw; ++e) {
      const double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
      wh[e] = (float)((2.0 * u - 1.0) * lim);
    }
    cudaMemcpy(m->w[l].p, wh.data(), nw * 4, cudaMemcpyHostToDevice);
    cudaMemset(m->b[l].p, 0, rows * 4);
    cudaMemset(m->mw[l].p, 0, nw * 4);
    cudaMemset(m->vw[l].p, 0, nw * 4);
    cudaMemset(m->mb[l].p, 0, rows * 4);
    cudaMemset(m->vb[l].p, 0, rows * 4);
  }
  if (!m->loss.ensure(4) || !m->err.ensure(4)) {
    delete m;
    return set_error(QP_ENOMEM, "warm start: cudaMalloc failed");
  }
  cudaMemset(m->err.p, 0, 4);
  const qp_status st = refresh_bf16(m, nullptr);
  if (st != QP_OK) {
    delete m;
    return st;
  }
  *out = m;
  return QP_OK;
}

extern "C" void qp_ws_destroy(qp_ws *m) {
  if (!m) return;
  DevGuard g(m->dev);
  delete m;
}

extern "C" int64_t qp_ws_param_count(void) { return (int64_t)n_params(); }

extern "C" qp_status qp_ws_get_params(qp_ws *m, float *out) {
  if (!m || !out) return set_error(QP_EINVAL, "NULL argument");
  DevGuard g(m->dev);
  size_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    const size_t nw = (size_t)kDimOut[l] * kDimIn[l];
    WS_CU(cudaMemcpy(out + o, m->w[l].p, nw * 4, cudaMemcpyDeviceToHost));
    o += nw;
    WS_CU(cudaMemcpy(out + o, m->b[l].p, (size_t)kDimOut[l] * 4, cudaMemcpyDeviceToHost));
    o += kDimOut[l];
  }
  return QP_OK;
}

extern "C" qp_status qp_ws_set_params(qp_ws *m, const float *in) {
  if (!m || !in) return set_error(QP_EINVAL, "NULL argument");
  DevGuard g(m->dev);
  size_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    const size_t nw = (size_t)kDimOut[l] * kDimIn[l];
    WS_CU(cudaMemcpy(m->w[l].p, in + o, nw * 4, cudaMemcpyHostToDevice));
    o += nw;
    WS_CU(cudaMemcpy(m->b[l].p, in + o, (size_t)kDimOut[l] * 4, cudaMemcpyHostToDevice));
    o += kDimOut[l];
  }
  return refresh_bf16(m, nullptr);
}

extern "C" qp_status qp_ws_forward(qp_ws *m, const float *feats, int32_t M, float *logits_out, void *stream) {
  if (!m || !feats || !logits_out || M < 1) return set_error(QP_EINVAL, "bad argument");
  if (device_pointer(logits_out) && !device_range_fits(logits_out, (size_t)M * kOut * 4))
    return set_error(QP_EINVAL, "qp_ws_forward: the device buffer for the logits is too small");
  DevGuard g(m->dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int Mp = (M + 127) / 128 * 128;
  if (qp_status s = upload_inputs(m, feats, M, Mp, nullptr, nullptr, st); s != QP_OK) return s;
  if (qp_status s = forward(m, Mp, false, st); s != QP_OK) return s;
  WS_CU(cudaMemcpyAsync(logits_out, m->z.p, (size_t)M * kOut * 4, cudaMemcpyDefault, st));
  return check_err(m, st);
}

extern "C" qp_status qp_ws_set_forward_mode(qp_ws *m, int32_t mode) {
  if (!m || (mode != QP_WS_FORWARD_FUSED && mode != QP_WS_FORWARD_LAYERED))
    return set_error(QP_EINVAL, "bad argument");
  m->fwd_mode = mode;
  return QP_OK;
}

extern "C" qp_status qp_ws_grads(qp_ws *m, const float *feats, const int32_t *labels, const int32_t *steps,
                                 int32_t M, float *grads_out, float *loss_out, void *stream) {
  if (!m || !feats || !labels || !steps || M < 1) return set_error(QP_EINVAL, "bad argument");
  DevGuard g(m->dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int Mp = (M + 127) / 128 * 128;
  if (qp_status s = upload_inputs(m, feats, M, Mp, labels, steps, st); s != QP_OK) return s;
  if (qp_status s = forward(m, Mp, true, st); s != QP_OK) return s;
  if (qp_status s = backward(m, M, Mp, st); s != QP_OK) return s;
  if (qp_status s = check_err(m, st); s != QP_OK) return s;
  if (grads_out) {
    size_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
      const size_t nw = (size_t)kDimOut[l] * kDimIn[l];
      WS_CU(cudaMemcpy(grads_out + o, m->gw[l].p, nw * 4, cudaMemcpyDeviceToHost));
      o += nw;
      WS_CU(cudaMemcpy(grads_out + o, m->gb[l].p, (size_t)kDimOut[l] * 4, cudaMemcpyDeviceToHost));
      o += kDimOut[l];
    }
  }
  if (loss_out) {
    float ls = 0.0f;
    WS_CU(cudaMemcpy(&ls, m->loss.p, 4, cudaMemcpyDeviceToHost));
    *loss_out = ls / (float)M;
  }
  return QP_OK;
}

extern "C" qp_status qp_ws_train_step(qp_ws *m, const float *feats, const int32_t *labels, const int32_t *steps,
                                      int32_t M, float lr, float *loss_out, void *stream) {
  const qp_status s0 = qp_ws_grads(m, feats, labels, steps, M, nullptr, loss_out, stream);
  if (s0 != QP_OK) return s0;
  DevGuard g(m->dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  m->step += 1;
  for (int l = 0; l < kLayers; ++l) {
    const int rows = kDimOut[l], cols = kDimIn[l];
    WS_CU(mlp::adam(m->w[l].as<float>(), m->mw[l].as<float>(), m->vw[l].as<float>(), m->gw[l].as<float>(), rows,
                    cols, lr, 0.9f, 0.999f, 1e-8f, m->step, m->wb[l].as<__nv_bfloat16>(),
                    m->wt[l].as<__nv_bfloat16>(), st));
    WS_CU(mlp::adam(m->b[l].as<float>(), m->mb[l].as<float>(), m->vb[l].as<float>(), m->gb[l].as<float>(), 1,
                    rows, lr, 0.9f, 0.999f, 1e-8f, m->step, nullptr, nullptr, st));
  }
  return QP_OK;
}

// ----------------------------------------------------------------------------- read-back
extern "C" qp_status qp_ws_get_state(qp_ws *m, int32_t which, float *out) {
  if (!m || !out || which < QP_WS_STATE_PARAMS || which > QP_WS_STATE_GRADS)
    return set_error(QP_EINVAL, "bad argument");
  DevGuard g(m->dev);
  WS_CU(cudaDeviceSynchronize());
  size_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    const Buf &W = which == QP_WS_STATE_PARAMS ? m->w[l]
                   : which == QP_WS_STATE_ADAM_M ? m->mw[l]
                   : which == QP_WS_STATE_ADAM_V ? m->vw[l] : m->gw[l];
    const Buf &B = which == QP_WS_STATE_PARAMS ? m->b[l]
                   : which == QP_WS_STATE_ADAM_M ? m->mb[l]
                   : which == QP_WS_STATE_ADAM_V ? m->vb[l] : m->gb[l];
    const size_t nw = (size_t)kDimOut[l] * kDimIn[l];
    WS_CU(cudaMemcpy(out + o, W.p, nw * 4, cudaMemcpyDeviceToHost));
    o += nw;
    WS_CU(cudaMemcpy(out + o, B.p, (size_t)kDimOut[l] * 4, cudaMemcpyDeviceToHost));
    o += kDimOut[l];
  }
  return QP_OK;
}

extern "C" qp_status qp_ws_get_buffer(qp_ws *m, int32_t which, int32_t rows, void *out) {
  if (!m || !out) return set_error(QP_EINVAL, "bad argument");
  DevGuard g(m->dev);
  if (which >= QP_WS_BUF_W_BF16 && which < QP_WS_BUF_W_BF16 + kLayers) {
    const int l = which - QP_WS_BUF_W_BF16;
    WS_CU(cudaDeviceSynchronize());
    WS_CU(cudaMemcpy(out, m->wb[l].p, (size_t)kDimOut[l] * kDimIn[l] * 2, cudaMemcpyDeviceToHost));
    return QP_OK;
  }
  if (which >= QP_WS_BUF_WT_BF16 && which < QP_WS_BUF_WT_BF16 + kLayers) {
    const int l = which - QP_WS_BUF_WT_BF16;
    WS_CU(cudaDeviceSynchronize());
    WS_CU(cudaMemcpy(out, m->wt[l].p, (size_t)kDimOut[l] * kDimIn[l] * 2, cudaMemcpyDeviceToHost));
    return QP_OK;
  }
  if (rows < 1 || rows > m->cap) return set_error(QP_EINVAL, "rows beyond the last pass's buffers");
  const Buf *b = nullptr;
  size_t row_bytes = (size_t)kHid * 2;
  switch (which) {
    case QP_WS_BUF_X0: b = &m->x0; row_bytes = (size_t)kIn * 2; break;
    case QP_WS_BUF_H1: case QP_WS_BUF_H2: case QP_WS_BUF_H3: b = &m->h[which - QP_WS_BUF_H1]; break;
    case QP_WS_BUF_Z: b = &m->z; row_bytes = (size_t)kOut * 4; break;
    case QP_WS_BUF_DZ: b = &m->dz; row_bytes = (size_t)kOut * 2; break;
    case QP_WS_BUF_DH1: case QP_WS_BUF_DH2: case QP_WS_BUF_DH3: b = &m->dh[which - QP_WS_BUF_DH1]; break;
    default: return set_error(QP_EINVAL, "unknown buffer");
  }
  WS_CU(cudaDeviceSynchronize());
  WS_CU(cudaMemcpy(out, b->p, (size_t)rows * row_bytes, cudaMemcpyDeviceToHost));
  return QP_OK;
}

// ----------------------------------------------------------------------------- features
extern "C" qp_status qp_ws_features(const qp_field *f, float *feats_out, int32_t *n_cells) {
  if (!f || f->rows < 1 || f->cols < 1) return set_error(QP_EINVAL, "bad field");
  const int H = f->rows, W = f->cols;
  auto isfree = [&](int r, int c) {
    if (r < 0 || r >= H || c < 0 || c >= W) return false;
    return !f->free_mask || f->free_mask[r * W + c] != 0;
  };
  if (f->start < 0 || f->start >= H * W || !isfree(f->start / W, f->start % W))
    return set_error(QP_EINVAL, "start cell is not a free cell of the grid");
  const int rs = f->start / W, cs = f->start % W;
  int C = 0;
  for (int r = 0; r < H; ++r)
    for (int c = 0; c < W; ++c) C += isfree(r, c);
  if (n_cells) *n_cells = C;
  if (!feats_out) return QP_OK;
  int k = 0;
  for (int r = 0; r < H; ++r)
    for (int c = 0; c < W; ++c) {
      if (!isfree(r, c)) continue;
      int blocked8 = 0, free25 = 0;
      for (int dr = -2; dr <= 2; ++dr)
        for (int dc = -2; dc <= 2; ++dc) {
          const bool fr = isfree(r + dr, c + dc);
          free25 += fr;
          if (std::abs(dr) <= 1 && std::abs(dc) <= 1 && (dr || dc)) blocked8 += !fr;
        }
      float *x = feats_out + (size_t)k * kIn;
      x[0] = c / 15.0f;                        // x
      x[1] = r / 15.0f;                        // y
      x[2] = blocked8 / 8.0f;                  // obstacle context: blocked or outside among the 8 neighbours
      x[3] = cs / 15.0f;
      x[4] = rs / 15.0f;
      x[5] = W / 16.0f;
      x[6] = H / 16.0f;
      x[7] = C / 256.0f;
      x[8] = (c - cs) / 15.0f;
      x[9] = (r - rs) / 15.0f;
      x[10] = W > 1 ? c / (float)(W - 1) : 0.0f;
      x[11] = H > 1 ? r / (float)(H - 1) : 0.0f;
      x[12] = free25 / 25.0f;
      x[13] = (float)(r & 1);
      x[14] = 1.0f;
      x[15] = 0.0f;
      ++k;
    }
  return QP_OK;
}

// ----------------------------------------------------------------------------- decode
extern "C" qp_status qp_ws_decode(const float *logits, int32_t ld, int32_t C, int32_t start_cell, uint8_t *state_out,
                                  int32_t *path_out) {
  if (!logits || C < 1 || C > kOut || start_cell < 0 || start_cell >= C || ld < C)
    return set_error(QP_EINVAL, "bad argument");
  // Greedy matching: the start cell takes step 0; then repeatedly the largest
  // logit among unassigned cells and free steps 1..C-1 fixes one (cell, step)
  // pair (ties: smaller cell, then smaller step).  Each unassigned cell keeps
  // its best free step; only cells whose best step was just taken rescan.
  std::vector<int32_t> path(C, -1), best(C, -1);
  std::vector<char> cell_done(C, 0), step_done(C, 0);
  path[0] = start_cell;
  cell_done[start_cell] = 1;
  step_done[0] = 1;
  auto rescan = [&](int i) {
    int bt = -1;
    float bv = 0.0f;
    for (int t = 1; t < C; ++t) {
      if (step_done[t]) continue;
      const float v = logits[(size_t)i * ld + t];
      if (bt < 0 || v > bv) {
        bt = t;
        bv = v;
      }
    }
    best[i] = bt;
  };
  for (int i = 0; i < C; ++i)
    if (!cell_done[i]) rescan(i);
  for (int round = 1; round < C; ++round) {
    int bi = -1;
    float bv = 0.0f;
    for (int i = 0; i < C; ++i) {
      if (cell_done[i]) continue;
      const float v = logits[(size_t)i * ld + best[i]];
      if (bi < 0 || v > bv || (v == bv && i < bi)) {
        bi = i;
        bv = v;
      }
    }
    const int t = best[bi];
    path[t] = bi;
    cell_done[bi] = 1;
    step_done[t] = 1;
    for (int i = 0; i < C; ++i)
      if (!cell_done[i] && best[i] == t) rescan(i);
  }
  if (state_out) {
    std::memset(state_out, 0, (size_t)C * C);
    for (int t = 0; t < C; ++t) state_out[(size_t)t * C + path[t]] = 1;
  }
  if (path_out) std::memcpy(path_out, path.data(), (size_t)C * 4);
  return QP_OK;
}

// A walk guided by the predicted steps: from the start cell, move each step to
// the unvisited cell nearest to the current one (distance matrix d), choosing
// among equally near cells the one with the smallest expected step
// E_j = sum_t softmax(logits_j)_t * t over t < C (then the smaller cell id).
extern "C" qp_status qp_ws_decode_walk(const float *logits, int32_t ld, int32_t C, int32_t start_cell,
                                       const int32_t *d, uint8_t *state_out, int32_t *path_out) {
  if (!logits || !d || C < 1 || C > kOut || start_cell < 0 || start_cell >= C || ld < C)
    return set_error(QP_EINVAL, "bad argument");
  std::vector<double> e(C);
  for (int i = 0; i < C; ++i) {
    const float *z = logits + (size_t)i * ld;
    double mx = z[0];
    for (int t = 1; t < C; ++t) mx = std::max(mx, (double)z[t]);
    double s = 0.0, st = 0.0;
    for (int t = 0; t < C; ++t) {
      const double p = std::exp((double)z[t] - mx);
      s += p;
      st += p * t;
    }
    e[i] = st / s;
  }
  std::vector<int32_t> path(C);
  std::vector<char> seen(C, 0);
  int cur = start_cell;
  path[0] = cur;
  seen[cur] = 1;
  for (int t = 1; t < C; ++t) {
    int nb = -1;
    for (int j = 0; j < C; ++j) {
      if (seen[j]) continue;
      if (nb < 0) {
        nb = j;
        continue;
      }
      const int32_t dj = d[(size_t)cur * C + j], db = d[(size_t)cur * C + nb];
      if (dj < db || (dj == db && e[j] < e[nb])) nb = j;
    }
    path[t] = nb;
    seen[nb] = 1;
    cur = nb;
  }
  if (state_out) {
    std::memset(state_out, 0, (size_t)C * C);
    for (int t = 0; t < C; ++t) state_out[(size_t)t * C + path[t]] = 1;
  }
  if (path_out) std::memcpy(path_out, path.data(), (size_t)C * 4);
  return QP_OK;
}

// ----------------------------------------------------------------------------- one-call inference
extern "C" qp_status qp_ws_infer(qp_ws *m, const qp_field *field, const int32_t *d, uint8_t *state_out,
                                 int32_t *path_out, void *stream) {
  if (!m || !field || (!state_out && !path_out)) return set_error(QP_EINVAL, "bad argument");
  int32_t C = 0;
  qp_status s = qp_ws_features(field, nullptr, &C);
  if (s != QP_OK) return s;
  if (C < 1 || C > kOut) return set_error(QP_ERANGE, "the field has more cells than the network has steps");
  std::vector<float> feats((size_t)C * kIn), logits((size_t)C * kOut);
  s = qp_ws_features(field, feats.data(), nullptr);
  if (s != QP_OK) return s;
  s = qp_ws_forward(m, feats.data(), C, logits.data(), stream);
  if (s != QP_OK) return s;
  // the start cell's id: free cells before it in row-major order
  int start = 0;
  for (int g = 0; g < field->start; ++g) start += !field->free_mask || field->free_mask[g] != 0;
  return d ? qp_ws_decode_walk(logits.data(), kOut, C, start, d, state_out, path_out)
           : qp_ws_decode(logits.data(), kOut, C, start, state_out, path_out);
}
