// Device decode of the learned warm start: the expected step of every cell
// under its step logits, the walk that turns a field (with or without a
// per-cell score) into a feasible one-hot seed, and the greedy matching of
// cells to steps.  The public contract is in include/qpath.h
// (qp_ws_expected_steps, qp_ws_walk, qp_ws_greedy).
//
// Walk: from the start cell, step t goes to a cell not yet on the path.  The
// candidates are the unvisited cells within `slack` of the nearest unvisited
// distance from the current cell; among them the smallest (score, distance,
// cell id) wins, or the smallest (distance, cell id) without a score.  One
// warp runs a field: per step it reads the current cell's row of d twice
// (the nearest distance, then the winning key, both by warp reductions) and
// keeps the visited cells as a bitset in shared memory.
#include <climits>

#include "qp_device.cuh"
#include "qp_internal.h"

namespace qp {
namespace {

using namespace dev;

constexpr int kWalkMaxCells = kMaxCells;
constexpr int kWalkMaxD = (1 << 20) - 1;  // distances pack into 20 bits of the key

// E_m = sum_{t < T_m} t softmax(z_m)_t with T_m = steps[m] (clamped to
// [1, min(256, ld)]): one warp per cell, 8 logits per lane.
__global__ void k_expected_step(const float *Z, int ldz, const int32_t *steps, int M, float *E) {
  const int lane = threadIdx.x & 31;
  const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (m >= M) return;
  const int T = max(1, min(steps[m], min(256, ldz)));
  float v[8];
  float mx = -INFINITY;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int t = lane * 8 + i;
    v[i] = t < T ? Z[(size_t)m * ldz + t] : -INFINITY;
    mx = fmaxf(mx, v[i]);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
  float s = 0.0f, st = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int t = lane * 8 + i;
    const float p = t < T ? expf(v[i] - mx) : 0.0f;
    s += p;
    st += p * (float)t;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    s += __shfl_xor_sync(kFull, s, o);
    st += __shfl_xor_sync(kFull, st, o);
  }
  if (lane == 0) E[m] = st / s;
}

// Order-preserving 32-bit code of a finite float (-0 taken as +0).
__device__ __forceinline__ uint32_t float_key(float f) {
  uint32_t u = __float_as_uint(f);
  if (u == 0x80000000u) u = 0u;
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(kFull, v, o);
    v = w < v ? w : v;
  }
  return v;
}

__global__ void __launch_bounds__(32) k_ws_walk(const int32_t *d, int C, int start, const float *score, int slack,
                                                uint8_t *state, int32_t *path, int64_t *length) {
  __shared__ uint32_t vis[kWalkMaxCells / 32];
  __shared__ int32_t pth[kWalkMaxCells];
  const int lane = threadIdx.x;
  const int Cw = (C + 31) >> 5;
  for (int w = lane; w < Cw; w += 32) vis[w] = 0u;
  __syncwarp();
  if (lane == 0) {
    vis[start >> 5] = 1u << (start & 31);
    pth[0] = start;
  }
  __syncwarp();
  int cur = start;
  long long L = 0;
  for (int t = 1; t < C; ++t) {
    const int32_t *row = d + (size_t)cur * C;
    int dmin = INT_MAX;
    for (int j = lane; j < C; j += 32)
      if (!((vis[j >> 5] >> (j & 31)) & 1u)) dmin = min(dmin, __ldg(row + j));
    dmin = __reduce_min_sync(kFull, dmin);
    const int lim = dmin + slack;  // dmin <= kWalkMaxD and slack <= 2^30
    unsigned long long best = ~0ull;
    for (int j = lane; j < C; j += 32) {
      if ((vis[j >> 5] >> (j & 31)) & 1u) continue;
      const int dj = __ldg(row + j);
      if (dj > lim) continue;
      const uint32_t hi = score ? float_key(__ldg(score + j)) : 0u;
      const unsigned long long key = ((unsigned long long)hi << 32) | ((unsigned long long)dj << 12) | (unsigned)j;
      best = key < best ? key : best;
    }
    best = warp_min_u64(best);
    const int nxt = (int)(best & 0xFFFu);
    L += __ldg(row + nxt);
    if (lane == 0) {
      vis[nxt >> 5] |= 1u << (nxt & 31);
      pth[t] = nxt;
    }
    __syncwarp();
    cur = nxt;
  }
  for (int t = lane; t < C; t += 32) {
    const int i = pth[t];
    if (path) path[t] = i;
    if (state) state[(size_t)t * C + i] = 1;
  }
  if (lane == 0 && length) *length = L;
}

// Greedy matching of cells to steps (the device form of qp_ws_decode): step 0
// is the start cell; each round fixes the (cell, step) pair with the largest
// logit over the unassigned cells and the free steps 1..C-1, ties to the
// smaller cell, then the smaller step.  One CTA, one thread per cell: a
// thread keeps its cell's best free step (the smaller step on equal logits);
// a round is a block-wide maximum of (logit, -cell), after which the cells
// whose best step was just taken scan their row again.
constexpr int kGreedyThreads = 256;

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(kFull, v, o);
    v = w > v ? w : v;
  }
  return v;
}

__global__ void __launch_bounds__(kGreedyThreads) k_ws_greedy(const float *Z, int ld, int C, int start,
                                                              uint8_t *state, int32_t *path) {
  __shared__ unsigned char step_done[kGreedyThreads];
  __shared__ int32_t pth[kGreedyThreads];
  __shared__ unsigned long long wmax[kGreedyThreads / 32];
  __shared__ int32_t taken;
  const int i = threadIdx.x, lane = i & 31, warp = i >> 5;
  step_done[i] = (i == 0 || i >= C) ? 1 : 0;
  if (i == 0) pth[0] = start;
  bool open = i < C && i != start;
  __syncthreads();
  const float *zi = Z + (size_t)min(i, C - 1) * ld;
  int bt = -1;
  float bv = 0.0f;
  auto rescan = [&]() {
    bt = -1;
    for (int t = 1; t < C; ++t) {
      if (step_done[t]) continue;
      const float v = __ldg(zi + t);
      if (bt < 0 || v > bv) {
        bt = t;
        bv = v;
      }
    }
  };
  if (open) rescan();
  for (int round = 1; round < C; ++round) {
    // keys are > 0 for finite logits; the low bits prefer the smaller cell
    const unsigned long long key =
        open ? ((unsigned long long)float_key(bv) << 32) | (unsigned)(0xFFFFu - (unsigned)i) : 0ull;
    const unsigned long long wm = warp_max_u64(key);
    if (lane == 0) wmax[warp] = wm;
    __syncthreads();
    unsigned long long m = wmax[0];
#pragma unroll
    for (int w = 1; w < kGreedyThreads / 32; ++w) m = wmax[w] > m ? wmax[w] : m;
    const int bi = (int)(0xFFFFu - (unsigned)(m & 0xFFFFu));
    if (i == bi) {
      taken = bt;
      pth[bt] = i;
      step_done[bt] = 1;
      open = false;
    }
    __syncthreads();
    if (open && bt == taken) rescan();
  }
  __syncthreads();
  if (i < C) {
    const int c = pth[i];
    if (path) path[i] = c;
    if (state) state[(size_t)i * C + c] = 1;
  }
}

}  // namespace
}  // namespace qp

extern "C" qp_status qp_ws_expected_steps(const float *logits, int32_t ld, int32_t M, const int32_t *steps,
                                          float *E_out, void *stream) {
  using namespace qp;
  clear_error();
  if (!logits || !steps || !E_out || M < 1 || ld < 1)
    return set_error(QP_EINVAL, "qp_ws_expected_steps: bad argument");
  if (!device_pointer(logits) || !device_pointer(steps) || !device_pointer(E_out))
    return set_error(QP_EINVAL, "qp_ws_expected_steps: every buffer must be device memory");
  if (!device_range_fits(logits, (size_t)M * ld * 4) || !device_range_fits(steps, (size_t)M * 4) ||
      !device_range_fits(E_out, (size_t)M * 4))
    return set_error(QP_EINVAL, "qp_ws_expected_steps: a device buffer is smaller than the call needs");
  k_expected_step<<<(M + 7) / 8, 256, 0, static_cast<cudaStream_t>(stream)>>>(logits, ld, steps, M, E_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(QP_ECUDA, cudaGetErrorString(e));
  return QP_OK;
}

extern "C" qp_status qp_ws_walk(qp_handle *h, const float *score, int32_t slack, uint8_t *state_out,
                                int32_t *path_out, int64_t *length_out, void *stream) {
  using namespace qp;
  clear_error();
  StructView v;
  if (!h || !handle_struct_view(h, &v)) return set_error(QP_EINVAL, "qp_ws_walk needs a handle built by qp_build_qubo");
  if (slack < 0 || slack > (1 << 30) || (!state_out && !path_out))
    return set_error(QP_EINVAL, "qp_ws_walk: need 0 <= slack <= 2^30 and a state or path output");
  if (v.C > kWalkMaxCells) return set_error(QP_ERANGE, "qp_ws_walk: more than 4096 cells");
  if (v.max_d > kWalkMaxD) return set_error(QP_ERANGE, "qp_ws_walk: distances above 2^20 - 1");
  if ((score && !device_pointer(score)) || (state_out && !device_pointer(state_out)) ||
      (path_out && !device_pointer(path_out)) || (length_out && !device_pointer(length_out)))
    return set_error(QP_EINVAL, "qp_ws_walk: every buffer must be device memory");
  if ((score && !device_range_fits(score, (size_t)v.C * 4)) ||
      (state_out && !device_range_fits(state_out, (size_t)v.C * v.C)) ||
      (path_out && !device_range_fits(path_out, (size_t)v.C * 4)) || (length_out && !device_range_fits(length_out, 8)))
    return set_error(QP_EINVAL, "qp_ws_walk: a device buffer is smaller than the call needs");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return set_error(QP_ECUDA, "qp_ws_walk: cudaGetDevice failed");
  if (prev != v.dev && cudaSetDevice(v.dev) != cudaSuccess) return set_error(QP_ECUDA, "qp_ws_walk: cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (state_out) e = cudaMemsetAsync(state_out, 0, (size_t)v.C * v.C, st);
  if (e == cudaSuccess) {
    k_ws_walk<<<1, 32, 0, st>>>(v.d32, v.C, v.start, score, slack, state_out, path_out, length_out);
    e = cudaGetLastError();
  }
  if (prev != v.dev) cudaSetDevice(prev);
  if (e != cudaSuccess) return set_error(QP_ECUDA, cudaGetErrorString(e));
  return QP_OK;
}

extern "C" qp_status qp_ws_greedy(const float *logits, int32_t ld, int32_t C, int32_t start_cell, uint8_t *state_out,
                                  int32_t *path_out, void *stream) {
  using namespace qp;
  clear_error();
  if (!logits || C < 1 || C > kGreedyThreads || start_cell < 0 || start_cell >= C || ld < C ||
      (!state_out && !path_out))
    return set_error(QP_EINVAL, "qp_ws_greedy: bad argument");
  if (!device_pointer(logits) || (state_out && !device_pointer(state_out)) || (path_out && !device_pointer(path_out)))
    return set_error(QP_EINVAL, "qp_ws_greedy: every buffer must be device memory");
  if (!device_range_fits(logits, ((size_t)(C - 1) * ld + C) * 4) ||
      (state_out && !device_range_fits(state_out, (size_t)C * C)) ||
      (path_out && !device_range_fits(path_out, (size_t)C * 4)))
    return set_error(QP_EINVAL, "qp_ws_greedy: a device buffer is smaller than the call needs");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (state_out) e = cudaMemsetAsync(state_out, 0, (size_t)C * C, st);
  if (e == cudaSuccess) {
    k_ws_greedy<<<1, kGreedyThreads, 0, st>>>(logits, ld, C, start_cell, state_out, path_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return set_error(QP_ECUDA, cudaGetErrorString(e));
  return QP_OK;
}
