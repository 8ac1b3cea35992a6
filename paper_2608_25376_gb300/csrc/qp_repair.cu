// Repair of annealed states into flight paths, on the device (one warp per
// replica).  The reconstruction step of Algorithm 1 reads the path off the
// best state and must hand back a feasible flight path; a state whose row or
// column sums are not all 1 has none, so it is repaired:
//
//   Greedy fix.  path[0] = s.  For t = 1 .. C-1, with prev = path[t-1]: the
//   candidates are the cells not yet on the path that are hot in row t
//   (x_{t,i} = 1); if there are none, every cell not yet on the path.  path[t]
//   is the candidate nearest to prev (smallest d), ties to the smaller id.  A
//   feasible state (every row and column sum 1, x_{0,s} = 1) comes out as its
//   own decoded path.
//
//   2-opt (open path, path[0] fixed).  Move (i, j), 1 <= i < j <= C-1,
//   reverses path[i..j]: edges (i-1, i) and (j, j+1) become (i-1, j) and
//   (i, j+1) (no edge after j = C-1); inner edges keep their lengths because
//   d is symmetric.  One pass: for i = 1 .. C-2, for j = i+1 .. C-1 in order,
//   apply the move when it makes the path strictly shorter, then go on with
//   j+1 on the changed path.  Passes repeat while the last one moved and fewer
//   than max_passes have run (max_passes < 0: until no move helps, which ends
//   because every move shortens an integer length).
//
// The warp evaluates 32 consecutive j at once on the current path and applies
// the first improving one, then restarts at the j after it: the same moves, in
// the same order, as the scan one j at a time.
#include "qp_device.cuh"
#include "qp_internal.h"

namespace qp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t w = __shfl_xor_sync(kFull, v, o);
    v = w < v ? w : v;
  }
  return v;
}

// Reverse path[i..j] and the inner edges edge[i..j-1] (edge[t] = d(path[t], path[t+1])).
__device__ __forceinline__ void reverse_segment(int32_t *path, int32_t *edge, int i, int j, int lane) {
  const int L = j - i + 1;
  for (int k = lane; k < L / 2; k += 32) {
    const int32_t a = path[i + k], b = path[j - k];
    path[i + k] = b;
    path[j - k] = a;
  }
  for (int k = lane; k < (L - 1) / 2; k += 32) {
    const int32_t a = edge[i + k], b = edge[j - 1 - k];
    edge[i + k] = b;
    edge[j - 1 - k] = a;
  }
  __syncwarp();
}

// smem per warp: path[C], edge[C], used bits[ceil(C/32)]  (int32 words)
__global__ void k_repair(const uint8_t *__restrict__ states, int R, int C, int start,
                         const int32_t *__restrict__ d, int max_passes, int32_t *__restrict__ paths,
                         int64_t *__restrict__ lengths, int32_t *__restrict__ status) {
  extern __shared__ int32_t sm_all[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int r = blockIdx.x * W + warp;
  if (r >= R) return;
  const int nwu = (C + 31) >> 5;
  int32_t *path = sm_all + (size_t)warp * (2 * C + nwu);
  int32_t *edge = path + C;
  uint32_t *used = reinterpret_cast<uint32_t *>(edge + C);
  const uint8_t *x = states + (size_t)r * C * C;

  for (int w = lane; w < nwu; w += 32) used[w] = 0;
  __syncwarp();
  // row 0 must be exactly {s} for the state to be feasible
  int hot0 = 0;
  for (int i = lane; i < C; i += 32) hot0 += x[i] != 0;
  hot0 = __reduce_add_sync(kFull, hot0);
  bool feasible = hot0 == 1 && x[start] != 0;
  if (lane == 0) {
    path[0] = start;
    used[start >> 5] |= 1u << (start & 31);
  }
  __syncwarp();

  // greedy fix
  for (int t = 1; t < C; ++t) {
    const int prev = path[t - 1];
    const int32_t *drow = d + (size_t)QP_IX(prev, C, 5) * C;
    const uint8_t *xr = x + (size_t)t * C;
    uint64_t best_hot = ~0ull, best_any = ~0ull;
    int hot = 0;
    for (int i = lane; i < C; i += 32) {
      const bool h = xr[i] != 0;
      hot += h;
      if (!((used[i >> 5] >> (i & 31)) & 1u)) {
        const uint64_t key = ((uint64_t)(uint32_t)drow[i] << 32) | (uint32_t)i;
        best_any = key < best_any ? key : best_any;
        if (h) best_hot = key < best_hot ? key : best_hot;
      }
    }
    hot = __reduce_add_sync(kFull, hot);
    best_hot = warp_min_u64(best_hot);
    best_any = warp_min_u64(best_any);
    // feasible so far iff this row has one hot cell and it is not on the path yet
    feasible = feasible && hot == 1 && best_hot != ~0ull;
    const int pick = (int)(uint32_t)(best_hot != ~0ull ? best_hot : best_any);
    __syncwarp();
    if (lane == 0) {
      path[t] = pick;
      used[pick >> 5] |= 1u << (pick & 31);
    }
    __syncwarp();
  }

  // 2-opt
  for (int t = lane; t + 1 < C; t += 32) edge[t] = d[QP_IX((size_t)path[t] * C + path[t + 1], (size_t)C * C, 5)];
  __syncwarp();
  bool changed = false;
  bool moved = true;
  for (int pass = 0; moved && (max_passes < 0 || pass < max_passes); ++pass) {
    moved = false;
    for (int i = 1; i + 1 < C; ++i) {
      int j0 = i + 1;
      while (j0 < C) {
        const int a = path[i - 1], b = path[i];
        const int j = j0 + lane;
        int32_t n1 = 0, n2 = 0;
        bool imp = false;
        if (j < C) {
          const int pj = path[j];
          int64_t old = edge[i - 1];
          n1 = d[QP_IX((size_t)a * C + pj, (size_t)C * C, 5)];
          if (j + 1 < C) {
            old += edge[j];
            n2 = d[QP_IX((size_t)b * C + path[j + 1], (size_t)C * C, 5)];
          }
          imp = (int64_t)n1 + n2 < old;
        }
        const unsigned m = __ballot_sync(kFull, imp);
        if (m) {
          const int f = __ffs(m) - 1, js = j0 + f;
          const int32_t n1s = __shfl_sync(kFull, n1, f), n2s = __shfl_sync(kFull, n2, f);
          __syncwarp();
          reverse_segment(path, edge, i, js, lane);
          if (lane == 0) {
            edge[i - 1] = n1s;
            if (js + 1 < C) edge[js] = n2s;
          }
          __syncwarp();
          moved = true;
          changed = true;
          j0 = js + 1;
        } else {
          j0 += 32;
        }
      }
    }
  }

  int32_t *out = paths + (size_t)r * C;
  long long L = 0;
  for (int t = lane; t < C; t += 32) {
    out[t] = path[t];
    if (t + 1 < C) L += d[QP_IX((size_t)path[t] * C + path[t + 1], (size_t)C * C, 5)];
  }
  L = dev::warp_sum64(L);
  if (lane == 0) {
    lengths[r] = L;
    status[r] = feasible ? (changed ? 1 : 0) : 2;
  }
}

}  // namespace

size_t repair_smem_per_warp(int32_t C) { return (size_t)(2 * C + (C + 31) / 32) * 4; }

cudaError_t launch_repair(const uint8_t *states, int32_t R, int32_t C, int32_t start, const int32_t *d32,
                          int32_t max_passes, int32_t *paths, int64_t *lengths, int32_t *status,
                          cudaStream_t st) {
  const size_t per = repair_smem_per_warp(C);
  int W = 8;
  while (W > 1 && W * per > 96 * 1024) W >>= 1;
  const size_t smem = W * per;
  if (smem > 96 * 1024) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lk(launch_mutex());
  cudaError_t e = cudaFuncSetAttribute(k_repair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_repair<<<(R + W - 1) / W, W * 32, smem, st>>>(states, R, C, start, d32, max_passes, paths, lengths, status);
  return cudaGetLastError();
}

}  // namespace qp

namespace qp {
namespace chk {
QP_CHECK_ACCESSOR(repair)
}  // namespace chk
}  // namespace qp
