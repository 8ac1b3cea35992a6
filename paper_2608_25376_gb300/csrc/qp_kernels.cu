// Device code of libqpath for sm_103a: the structured and dense Metropolis
// sweeps over the one-hot path QUBO (Eqs. 3-6), the dense-form builder and the
// batch path decoder (Algorithm 1, last step).
//
// Mapping.  One warp owns one replica (an independent Markov chain).  A sweep
// proposes the free variables k = t*C + i in increasing order.  The warp
// evaluates 128 consecutive proposals at once (lane L owns the Philox block
// m = k>>2, i.e. the four variables 4m..4m+3, so one Philox4x32-10 call
// serves all of a lane's draws), all against the current state.  A ballot
// finds the first accepted proposal; everything before it is final and
// exactly what the sequential sweep would have done; the flip is applied and
// evaluation resumes at the next variable.  The result is bit-identical to the
// sequential chain.  Random numbers are drawn lazily: a proposal needs its
// draw only when 1 <= dE < len_s, and the counter-based generator makes the
// draw independent of when (or whether) it is computed.
#include <climits>

#include "qp_device.cuh"
#include "qp_internal.h"

namespace qp {
namespace {

using dev::kFull;
using dev::philox4x32_10;
using dev::warp_sum64;
using dev::word_of;

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Bits of state word w that fall in [kb, ke); requires (w<<5) < ke and
// (w<<5) + 32 > kb.
__device__ __forceinline__ uint32_t range_mask(int w, int kb, int ke) {
  const int lo = w << 5;
  uint32_t m = 0xffffffffu;
  if (lo < kb) m &= 0xffffffffu << (kb - lo);
  if (lo + 32 > ke) m &= (1u << (ke - lo)) - 1u;
  return m;
}

// Appends to hot[] (warp-uniform) the cells i with bit kb + i set, i < C.
__device__ __forceinline__ int collect_hot(const uint32_t *st, int kb, int C, int16_t *hot, int nh,
                                           int lane) {
  const int ke = kb + C;
  const int w0 = kb >> 5, w1 = (ke - 1) >> 5;
  for (int wb = w0; wb <= w1; wb += 32) {
    const int w = wb + lane;
    uint32_t word = 0;
    if (w <= w1) word = st[w] & range_mask(w, kb, ke);
    uint32_t bal = __ballot_sync(kFull, word != 0);
    while (bal) {
      const int L = __ffs(bal) - 1;
      bal &= bal - 1;
      uint32_t wd = __shfl_sync(kFull, word, L);
      const int base = ((wb + L) << 5) - kb;
      while (wd) {
        const int b = __ffs(wd) - 1;
        wd &= wd - 1;
        if (lane == 0) hot[nh] = (int16_t)(base + b);
        ++nh;
      }
    }
  }
  __syncwarp();
  return nh;
}

template <typename T>
__device__ __forceinline__ int ld_elem(const T *p, bool smem) {
  return smem ? (int)*p : (int)__ldg(p);
}

// ---------------------------------------------------------------------------
// Structured sweep.  Per replica: the spins as a flat bitset over k (in shared
// memory, or in global memory for large C), the row and column one-hot sums
// (int16, shared) and, per row t, the list of hot cells of rows t-1 and t+1.
// dE of x_{t,i} = (1-2x)[B f_i + A(2r'-1) + A(2c'-1)] with
// f_i = sum over hot cells h of rows t-1, t+1 of d_{h,i} (the derivation from
// Eq. 6 is in the oracle; the kernel never forms S).
template <typename DT, bool STATE_SMEM, bool D_SMEM>
__global__ void __launch_bounds__(kMaxWarpsPerCta * 32)
    k_sweep_structured(const StructArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int C = a.C, Cp = a.Cp, s0 = a.start, A = a.A, B = a.B;
  const int n = C * C;
  const int nw = (n + 31) >> 5;
  unsigned char *p = smem;
  const DT *d = static_cast<const DT *>(a.d);
  if (D_SMEM) {
    DT *ds = reinterpret_cast<DT *>(p);
    const int nv = (int)((size_t)C * Cp * sizeof(DT) / 16);
    const int4 *src = static_cast<const int4 *>(a.d);
    int4 *dst = reinterpret_cast<int4 *>(ds);
    for (int v = threadIdx.x; v < nv; v += blockDim.x) dst[v] = __ldg(src + v);
    d = ds;
    p += align16((size_t)C * Cp * sizeof(DT));
  }
  const size_t per_warp = 8 * (size_t)Cp + (STATE_SMEM ? 4 * (size_t)a.nw_pad : 0);
  unsigned char *wp = p + warp * per_warp;
  int16_t *rowsum = reinterpret_cast<int16_t *>(wp);
  int16_t *colsum = rowsum + Cp;
  int16_t *hot = colsum + Cp;  // 2*Cp entries: rows t-1 and t+1 hold at most 2C hot cells
  uint32_t *st = STATE_SMEM ? reinterpret_cast<uint32_t *>(hot + 2 * Cp) : nullptr;
  __syncthreads();
  const int r = blockIdx.x * W + warp;
  if (r >= a.R) return;  // no CTA-wide barrier after this point
  if (!STATE_SMEM) st = a.gstate + (size_t)r * a.nw_pad;
  const uint32_t rg = (uint32_t)(a.rep_offset + r);

  // ---- initial state: given or all zero, then the start clamp
  const uint8_t *init = a.init ? a.init + (size_t)r * n : nullptr;
  for (int w = lane; w < nw; w += 32) {
    uint32_t word = 0;
    if (init) {
      for (int b = 0; b < 32; ++b) {
        const int k = (w << 5) + b;
        if (k < n && init[k]) word |= 1u << b;
      }
    }
    st[w] = word;
  }
  __syncwarp();
  if (init) {
    for (int w = lane; w <= (C - 1) >> 5; w += 32) atomicAnd(&st[w], ~range_mask(w, 0, C));
    for (int t = lane; t < C; t += 32) {
      const int k = t * C + s0;
      atomicAnd(&st[k >> 5], ~(1u << (k & 31)));
    }
    __syncwarp();
  }
  if (lane == 0) st[s0 >> 5] |= 1u << (s0 & 31);
  __syncwarp();

  // ---- sums, violation count and the energy by its definition (Eqs. 3-6)
  long long hd = 0, pen = 0;
  int viol = 0;
  for (int t = lane; t < C; t += 32) {
    const int kb = t * C;
    int cnt = 0;
    for (int w = kb >> 5; w <= (kb + C - 1) >> 5; ++w) cnt += __popc(st[w] & range_mask(w, kb, kb + C));
    rowsum[t] = (int16_t)cnt;
    pen += (long long)(1 - cnt) * (1 - cnt);
    viol += cnt != 1;
    if (t + 1 < C) {
      const int kb2 = kb + C;
      for (int w = kb >> 5; w <= (kb + C - 1) >> 5; ++w) {
        uint32_t word = st[w] & range_mask(w, kb, kb + C);
        while (word) {
          const int i = (w << 5) + __ffs(word) - 1 - kb;
          word &= word - 1;
          for (int w2 = kb2 >> 5; w2 <= (kb2 + C - 1) >> 5; ++w2) {
            uint32_t word2 = st[w2] & range_mask(w2, kb2, kb2 + C);
            while (word2) {
              const int j = (w2 << 5) + __ffs(word2) - 1 - kb2;
              word2 &= word2 - 1;
              hd += ld_elem(d + (size_t)i * Cp + j, D_SMEM);
            }
          }
        }
      }
    }
  }
  for (int i = lane; i < C; i += 32) {
    int cnt = 0;
    for (int t = 0; t < C; ++t) {
      const int k = t * C + i;
      cnt += (st[k >> 5] >> (k & 31)) & 1;
    }
    colsum[i] = (int16_t)cnt;
    pen += (long long)(1 - cnt) * (1 - cnt);
    viol += cnt != 1;
  }
  __syncwarp();
  long long E = (long long)B * warp_sum64(hd) + (long long)A * warp_sum64(pen);
  viol = __reduce_add_sync(kFull, viol);
  long long best = LLONG_MAX, acc = 0;
  const int lev = a.level ? __ldg(a.level + r) : -1;

  // ---- sweeps
  for (int s = a.sweep_begin; s < a.sweep_end; ++s) {
    const int ts = lev >= 0 ? lev : s;  // table row: the sweep, or the replica's ladder level
    const uint32_t *thr = a.thr + a.thr_off[ts];
    const int len = a.thr_len[ts];
    const float cT = a.thr_c[ts];
    for (int t = 1; t < C; ++t) {
      int nh = collect_hot(st, (t - 1) * C, C, hot, 0, lane);
      if (t + 1 < C) nh = collect_hot(st, (t + 1) * C, C, hot, nh, lane);
      int rt = rowsum[t];
      const int rt0 = rt;
      const int kb = t * C, ke = kb + C;
      const int mb = kb >> 2, me = (ke - 1) >> 2;
      int pos = kb;
      for (int m0 = mb; m0 <= me; m0 += 32) {
        const int m = m0 + lane;
        const int k0 = m << 2;
        uint32_t xn = 0;
        int valid = 0;
        int g[4] = {0, 0, 0, 0};
        if (m <= me) {
          xn = (st[k0 >> 5] >> (k0 & 31)) & 0xFu;
          int f[4] = {0, 0, 0, 0};
          for (int h = 0; h < nh; ++h) {
            const DT *drow = d + (size_t)QP_IX((int)hot[h], C, 6) * Cp;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int i = k0 + j - kb;
              if (i >= 0 && i < C) f[j] += ld_elem(drow + i, D_SMEM);
            }
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int i = k0 + j - kb;
            if (i >= 0 && i < C && i != s0) {
              valid |= 1 << j;
              const int x = (xn >> j) & 1;
              g[j] = B * f[j] + A * (2 * (colsum[i] - x) - 1);
            }
          }
        }
        bool have_u = false;
        uint4 u = make_uint4(0, 0, 0, 0);
        while (true) {
          int accm = 0, need = 0;
          int dE[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int x = (xn >> j) & 1;
            dE[j] = (1 - 2 * x) * (g[j] + A * (2 * (rt - x) - 1));
            if (((valid >> j) & 1) && k0 + j >= pos) {
              if (dE[j] <= 0) accm |= 1 << j;
              else if (dE[j] < len) need |= 1 << j;
            }
          }
          if (__any_sync(kFull, need != 0 && !have_u)) {
            if (need != 0 && !have_u) {
              u = philox4x32_10(make_uint4((uint32_t)m, (uint32_t)s, rg, kRngTag), a.key0, a.key1);
              have_u = true;
            }
          }
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (((need >> j) & 1) && dev::accept_draw(word_of(u, j), dE[j], cT, thr, len)) accm |= 1 << j;
          const uint32_t bal = __ballot_sync(kFull, accm != 0);
          if (bal == 0) break;
          const int L = __ffs(bal) - 1;
          const int jl = accm ? __ffs(accm) - 1 : 0;
          const int dsel = jl == 0 ? dE[0] : (jl == 1 ? dE[1] : (jl == 2 ? dE[2] : dE[3]));
          const int jj = __shfl_sync(kFull, jl, L);
          const int de = __shfl_sync(kFull, dsel, L);
          const uint32_t xnL = __shfl_sync(kFull, xn, L);
          const int k = ((m0 + L) << 2) + jj;
          const int i = k - kb;
          const int dlt = 1 - 2 * (int)((xnL >> jj) & 1);
          E += de;
          ++acc;
          rt += dlt;
          const int cold = colsum[i];
          viol += ((cold + dlt) != 1) - (cold != 1);
          __syncwarp();
          if (lane == L) {
            xn ^= 1u << jj;
            colsum[i] = (int16_t)(cold + dlt);
            st[k >> 5] ^= 1u << (k & 31);
          }
          __syncwarp();
          pos = k + 1;
        }
      }
      viol += (rt != 1) - (rt0 != 1);
      if (lane == 0) rowsum[t] = (int16_t)rt;
      __syncwarp();
    }
    if (viol == 0 && E < best) best = E;
  }

  // ---- outputs
  uint8_t *out = a.states_out + (size_t)r * n;
  for (int k = lane; k < n; k += 32) out[k] = (uint8_t)((st[k >> 5] >> (k & 31)) & 1);
  if (lane == 0) {
    a.E_out[r] = E;
    if (a.best_out) a.best_out[r] = best;
    if (a.acc_out) a.acc_out[r] = acc;
  }
}

// ---------------------------------------------------------------------------
// Dense sweep for a generic QUBO.  Per replica: the local fields
// h_k = S_kk + sum_{l != k} S_kl x_l (int32, shared memory or global), the
// spins (bitset, shared) and, for path QUBOs, the row/column sums that decide
// feasibility.  dE_k = (1 - 2x_k) h_k; an accepted flip of k streams row k of S
// (= column k, S is symmetric) with 16-byte loads into h.
// h += dlt * row, the row already staged in shared memory.
template <typename ST>
__device__ __forceinline__ void add_row_staged(int32_t *h, const ST *stage, int np, int dlt, int lane) {
#pragma unroll 2
  for (int c = lane * 8; c < np; c += 256) {
    int v[8];
    if (sizeof(ST) == 2) {
      const int4 q = *reinterpret_cast<const int4 *>(stage + c);
      v[0] = (int)(short)(q.x & 0xFFFF); v[1] = q.x >> 16;
      v[2] = (int)(short)(q.y & 0xFFFF); v[3] = q.y >> 16;
      v[4] = (int)(short)(q.z & 0xFFFF); v[5] = q.z >> 16;
      v[6] = (int)(short)(q.w & 0xFFFF); v[7] = q.w >> 16;
    } else {
      const int4 q0 = *reinterpret_cast<const int4 *>(stage + c);
      const int4 q1 = *(reinterpret_cast<const int4 *>(stage + c) + 1);
      v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
      v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
    }
    int4 *hp = reinterpret_cast<int4 *>(h + c);
    int4 a0 = hp[0], a1 = hp[1];
    a0.x += dlt * v[0]; a0.y += dlt * v[1]; a0.z += dlt * v[2]; a0.w += dlt * v[3];
    a1.x += dlt * v[4]; a1.y += dlt * v[5]; a1.z += dlt * v[6]; a1.w += dlt * v[7];
    hp[0] = a0;
    hp[1] = a1;
  }
}

template <typename ST>
__device__ __forceinline__ void add_row(int32_t *h, const ST *row, int np, int dlt, int lane) {
  if constexpr (sizeof(ST) == 2) {
    // 8 loads of 16 bytes in flight per lane (4 KB per warp) before any use
    constexpr int MLP = 8;
    for (int c0 = lane * 8; c0 < np; c0 += 256 * MLP) {
      int4 q[MLP];
#pragma unroll
      for (int b = 0; b < MLP; ++b) {
        const int c = c0 + b * 256;
        q[b] = c < np ? __ldg(reinterpret_cast<const int4 *>(row + c)) : make_int4(0, 0, 0, 0);
      }
#pragma unroll
      for (int b = 0; b < MLP; ++b) {
        const int c = c0 + b * 256;
        if (c < np) {
          int4 *hp = reinterpret_cast<int4 *>(h + c);
          int4 a0 = hp[0], a1 = hp[1];
          a0.x += dlt * (int)(short)(q[b].x & 0xFFFF); a0.y += dlt * (q[b].x >> 16);
          a0.z += dlt * (int)(short)(q[b].y & 0xFFFF); a0.w += dlt * (q[b].y >> 16);
          a1.x += dlt * (int)(short)(q[b].z & 0xFFFF); a1.y += dlt * (q[b].z >> 16);
          a1.z += dlt * (int)(short)(q[b].w & 0xFFFF); a1.w += dlt * (q[b].w >> 16);
          hp[0] = a0;
          hp[1] = a1;
        }
      }
    }
  } else {
    for (int c0 = lane * 8; c0 < np; c0 += 1024) {
      int v[4][8];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = c0 + b * 256;
        if (c < np) {
          const int4 q0 = __ldg(reinterpret_cast<const int4 *>(row + c));
          const int4 q1 = __ldg(reinterpret_cast<const int4 *>(row + c) + 1);
          v[b][0] = q0.x; v[b][1] = q0.y; v[b][2] = q0.z; v[b][3] = q0.w;
          v[b][4] = q1.x; v[b][5] = q1.y; v[b][6] = q1.z; v[b][7] = q1.w;
        }
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = c0 + b * 256;
        if (c < np) {
          int4 *hp = reinterpret_cast<int4 *>(h + c);
          int4 a0 = hp[0], a1 = hp[1];
          a0.x += dlt * v[b][0]; a0.y += dlt * v[b][1]; a0.z += dlt * v[b][2]; a0.w += dlt * v[b][3];
          a1.x += dlt * v[b][4]; a1.y += dlt * v[b][5]; a1.z += dlt * v[b][6]; a1.w += dlt * v[b][7];
          hp[0] = a0;
          hp[1] = a1;
        }
      }
    }
  }
}

// BULK: an accepted flip's row of S comes into a per-warp shared buffer by one
// bulk copy (cp.async.bulk, completion on an mbarrier) and is added from
// there; otherwise the warp streams it with 16-byte loads.
template <typename ST, bool H_SMEM, bool BULK>
__global__ void __launch_bounds__(kMaxWarpsPerCta * 32) k_sweep_dense(const DenseArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int n = (int)a.n, np = a.np, C = a.C;
  const int Cp = round_up(C > 0 ? C : 1, 8);
  const int nw = (n + 31) >> 5;
  const int nw_pad = round_up(nw, 4);
  const ST *S = static_cast<const ST *>(a.S);
  uint32_t *fz = reinterpret_cast<uint32_t *>(smem);
  for (int w = threadIdx.x; w < nw_pad; w += blockDim.x) fz[w] = w < nw ? a.frozen_bits[w] : 0u;
  unsigned char *p = smem + 4 * (size_t)nw_pad;
  const size_t stage_bytes = BULK ? sizeof(ST) * (size_t)np + 16 : 0;  // row buffer + mbarrier
  const size_t per_warp =
      (H_SMEM ? 4 * (size_t)np : 0) + stage_bytes + 4 * (size_t)nw_pad + (C > 0 ? 4 * (size_t)Cp : 0);
  unsigned char *wp = p + warp * per_warp;
  int32_t *h = H_SMEM ? reinterpret_cast<int32_t *>(wp) : nullptr;
  ST *stage = BULK ? reinterpret_cast<ST *>(wp + (H_SMEM ? 4 * (size_t)np : 0)) : nullptr;
  const uint32_t mbar = BULK ? dev::smem_addr(wp + (H_SMEM ? 4 * (size_t)np : 0) + sizeof(ST) * (size_t)np) : 0u;
  uint32_t parity = 0;
  uint32_t *st = reinterpret_cast<uint32_t *>(wp + (H_SMEM ? 4 * (size_t)np : 0) + stage_bytes);
  int16_t *rowsum = reinterpret_cast<int16_t *>(st + nw_pad);
  int16_t *colsum = rowsum + Cp;
  __syncthreads();
  const int r = blockIdx.x * W + warp;
  if (r >= a.R) return;  // no CTA-wide barrier after this point
  if (!H_SMEM) h = a.hbuf + (size_t)r * np;
  const uint32_t rg = (uint32_t)(a.rep_offset + r);
  if (BULK) {
    if (lane == 0) {
      dev::mbar_init1(mbar);
      dev::mbar_init_fence();
    }
    __syncwarp();
  }

  // ---- initial state and local fields
  const uint8_t *init = a.init ? a.init + (size_t)r * n : nullptr;
  for (int w = lane; w < nw_pad; w += 32) {
    uint32_t word = 0;
    if (init && w < nw) {
      for (int b = 0; b < 32; ++b) {
        const int k = (w << 5) + b;
        if (k < n && init[k]) word |= 1u << b;
      }
    }
    if (w < nw) word = (word & ~fz[w]) | (a.fval_bits[w] & fz[w]);
    st[w] = word;
  }
  for (int k = lane; k < np; k += 32) h[k] = k < n ? ld_elem(S + (size_t)k * np + k, false) : 0;
  __syncwarp();
  for (int w0 = 0; w0 < nw; w0 += 32) {
    const int w = w0 + lane;
    const uint32_t word = w < nw ? st[w] : 0u;
    uint32_t bal = __ballot_sync(kFull, word != 0);
    while (bal) {
      const int L = __ffs(bal) - 1;
      bal &= bal - 1;
      uint32_t wd = __shfl_sync(kFull, word, L);
      while (wd) {
        const int l = ((w0 + L) << 5) + __ffs(wd) - 1;
        wd &= wd - 1;
        add_row(h, S + (size_t)QP_IX(l, n, 4) * np, np, 1, lane);
        __syncwarp();
        if (lane == 0) h[l] -= ld_elem(S + (size_t)l * np + l, false);
        __syncwarp();
      }
    }
  }
  long long esum = 0;
  for (int k = lane; k < n; k += 32)
    if ((st[k >> 5] >> (k & 31)) & 1) esum += (long long)ld_elem(S + (size_t)k * np + k, false) + h[k];
  long long E = a.c0 + warp_sum64(esum) / 2;
  int viol = 0;
  if (C > 0) {
    for (int t = lane; t < C; t += 32) {
      int cnt = 0;
      for (int i = 0; i < C; ++i) {
        const int k = t * C + i;
        cnt += (st[k >> 5] >> (k & 31)) & 1;
      }
      rowsum[t] = (int16_t)cnt;
      viol += cnt != 1;
    }
    for (int i = lane; i < C; i += 32) {
      int cnt = 0;
      for (int t = 0; t < C; ++t) {
        const int k = t * C + i;
        cnt += (st[k >> 5] >> (k & 31)) & 1;
      }
      colsum[i] = (int16_t)cnt;
      viol += cnt != 1;
    }
    viol = __reduce_add_sync(kFull, viol);
  }
  __syncwarp();
  long long best = LLONG_MAX, acc = 0;
  const int nblk = (n + 3) >> 2;

  // ---- sweeps
  for (int s = a.sweep_begin; s < a.sweep_end; ++s) {
    const uint32_t *thr = a.thr + a.thr_off[s];
    const int len = a.thr_len[s];
    const float cT = a.thr_c[s];
    int pos = 0;
    const int lenq = len > 1 ? len : 1;  // a proposal matters if dE < len, or dE <= 0
    for (int m0 = 0; m0 < nblk; m0 += 32) {
      // Four groups of 128 proposals at once, when they start a block of four:
      // independent loads of their local fields and one vote; if no proposal
      // there has dE < len (none can be accepted, none needs a draw) the four
      // groups change nothing and are passed over.  Earlier flips are all
      // before them (pos <= their first proposal).
      if ((m0 & 127) == 0) {
        bool matters = false;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int mg = m0 + 32 * g + lane;
          if (mg < nblk) {
            const int kg = mg << 2;
            const uint32_t xg = (st[kg >> 5] >> (kg & 31)) & 0xFu;
            const uint32_t fg = (fz[kg >> 5] >> (kg & 31)) & 0xFu;
            const int ing = n - kg >= 4 ? 0xF : ((1 << (n - kg)) - 1);
            const int vg = (int)(~fg & 0xFu) & ing;
            const int4 hg = *reinterpret_cast<const int4 *>(h + kg);
            const int hh[4] = {hg.x, hg.y, hg.z, hg.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int dEj = ((xg >> j) & 1) ? -hh[j] : hh[j];
              matters |= ((vg >> j) & 1) && dEj < lenq;
            }
          }
        }
        if (!__any_sync(kFull, matters)) {
          m0 += 96;
          continue;
        }
      }
      const int m = m0 + lane;
      const int k0 = m << 2;
      uint32_t xn = 0;
      int valid = 0;
      int4 hv = make_int4(0, 0, 0, 0);
      if (m < nblk) {
        xn = (st[k0 >> 5] >> (k0 & 31)) & 0xFu;
        const uint32_t fzn = (fz[k0 >> 5] >> (k0 & 31)) & 0xFu;
        const int in = n - k0 >= 4 ? 0xF : ((1 << (n - k0)) - 1);
        valid = (int)(~fzn & 0xFu) & in;
        hv = *reinterpret_cast<const int4 *>(h + k0);
      }
      bool have_u = false;
      uint4 u = make_uint4(0, 0, 0, 0);
      while (true) {
        const int hj[4] = {hv.x, hv.y, hv.z, hv.w};
        int accm = 0, need = 0;
        int dE[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          dE[j] = ((xn >> j) & 1) ? -hj[j] : hj[j];
          if (((valid >> j) & 1) && k0 + j >= pos) {
            if (dE[j] <= 0) accm |= 1 << j;
            else if (dE[j] < len) need |= 1 << j;
          }
        }
        if (__any_sync(kFull, need != 0 && !have_u)) {
          if (need != 0 && !have_u) {
            u = philox4x32_10(make_uint4((uint32_t)m, (uint32_t)s, rg, kRngTag), a.key0, a.key1);
            have_u = true;
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (((need >> j) & 1) && dev::accept_draw(word_of(u, j), dE[j], cT, thr, len)) accm |= 1 << j;
        const uint32_t bal = __ballot_sync(kFull, accm != 0);
        if (bal == 0) break;
        const int L = __ffs(bal) - 1;
        const int jl = accm ? __ffs(accm) - 1 : 0;
        const int dsel = jl == 0 ? dE[0] : (jl == 1 ? dE[1] : (jl == 2 ? dE[2] : dE[3]));
        const int jj = __shfl_sync(kFull, jl, L);
        const int de = __shfl_sync(kFull, dsel, L);
        const uint32_t xnL = __shfl_sync(kFull, xn, L);
        const int k = ((m0 + L) << 2) + jj;
        const int dlt = 1 - 2 * (int)((xnL >> jj) & 1);
        E += de;
        ++acc;
        int32_t skk;
        if (BULK) {
          __syncwarp();
          if (lane == 0)
            dev::bulk_copy(dev::smem_addr(stage), S + (size_t)QP_IX(k, n, 4) * np, (uint32_t)(sizeof(ST) * np), mbar);
          const bool done = __all_sync(kFull, dev::mbar_wait_bounded(mbar, parity));
          parity ^= 1u;
          if (!done) {
            // the copy did not complete: flag it, let it land (bounded), drop this chain
            if (lane == 0) {
              if (a.err) atomicExch(a.err, 1);
              dev::mbar_wait_bounded(mbar, parity ^ 1u);
              a.E_out[r] = LLONG_MIN;
            }
            return;
          }
          add_row_staged(h, stage, np, dlt, lane);
          skk = (int32_t)stage[k];
        } else {
          add_row(h, S + (size_t)QP_IX(k, n, 4) * np, np, dlt, lane);
          skk = 0;
        }
        __syncwarp();
        int t = 0, i = 0, ro = 0, co = 0;
        if (C > 0) {
          t = k / C;
          i = k - t * C;
          ro = rowsum[t];
          co = colsum[i];
          viol += ((ro + dlt) != 1) - (ro != 1) + ((co + dlt) != 1) - (co != 1);
        }
        __syncwarp();
        if (lane == 0) {
          h[k] -= dlt * (BULK ? skk : ld_elem(S + (size_t)k * np + k, false));
          st[k >> 5] ^= 1u << (k & 31);
          if (C > 0) {
            rowsum[t] = (int16_t)(ro + dlt);
            colsum[i] = (int16_t)(co + dlt);
          }
        }
        __syncwarp();
        if (lane == L) xn ^= 1u << jj;
        if (m < nblk) hv = *reinterpret_cast<const int4 *>(h + k0);
        pos = k + 1;
      }
    }
    if ((C == 0 || viol == 0) && E < best) best = E;
  }

  uint8_t *out = a.states_out + (size_t)r * n;
  for (int k = lane; k < n; k += 32) out[k] = (uint8_t)((st[k >> 5] >> (k & 31)) & 1);
  if (lane == 0) {
    a.E_out[r] = E;
    if (a.best_out) a.best_out[r] = best;
    if (a.acc_out) a.acc_out[r] = acc;
  }
}

// ---------------------------------------------------------------------------
// Dense form of Eq. 6 from the distance matrix (n x np, zero padding).  w:
// one weight per leg (the leg from step t to t+1 gets w[t] in place of B; the
// extended objective), or null.
template <typename ST>
__global__ void k_build_dense(ST *S, int np, int C, const int32_t *d, int A, int B, const int32_t *w) {
  const long long n = (long long)C * C;
  const long long total = n * np;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / np), l = (int)(e - (long long)k * np);
    int v = 0;
    if (l < n) {
      const int t = k / C, i = k - t * C, u = l / C, j = l - u * C;
      if (l == k) {
        v = -2 * A;
      } else {
        if (u == t) v += 2 * A;
        if (j == i) v += 2 * A;
        if (u == t + 1 || u + 1 == t) v += (w ? w[min(t, u)] : B) * d[i * C + j];
      }
    }
    S[e] = (ST)v;
  }
}

// Algorithm 1 last step for a batch of states: one warp per state.
__global__ void k_decode(const uint8_t *states, int R, int C, const int32_t *d, int32_t *paths,
                         int64_t *lengths) {
  extern __shared__ int32_t colcnt_all[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int r = blockIdx.x * W + warp;
  if (r >= R) return;
  int32_t *colcnt = colcnt_all + warp * C;
  const size_t n = (size_t)C * C;
  const uint8_t *x = states + (size_t)r * n;
  int32_t *path = paths + (size_t)r * C;
  for (int i = lane; i < C; i += 32) colcnt[i] = 0;
  __syncwarp();
  bool ok = true;
  for (int t = 0; t < C; ++t) {
    int cnt = 0, at = -1;
    for (int i = lane; i < C; i += 32) {
      if (x[(size_t)t * C + i]) {
        ++cnt;
        at = i;
        colcnt[i] += 1;
      }
    }
    cnt = __reduce_add_sync(kFull, cnt);
    at = __reduce_max_sync(kFull, at);
    ok = ok && cnt == 1;
    if (lane == 0) path[t] = at;
  }
  __syncwarp();
  int bad = 0;
  for (int i = lane; i < C; i += 32) bad |= colcnt[i] != 1;
  ok = ok && !__any_sync(kFull, bad);
  long long L = 0;
  if (ok)
    for (int t = lane; t + 1 < C; t += 32) L += d[(size_t)path[t] * C + path[t + 1]];
  L = warp_sum64(L);
  if (lane == 0) lengths[r] = ok ? L : -1;
}

template <typename DT, bool SS, bool DS>
cudaError_t launch_s(const StructArgs &a, int W, size_t smem, cudaStream_t st) {
  auto k = k_sweep_structured<DT, SS, DS>;
  std::lock_guard<std::mutex> lk(launch_mutex());
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (a.R + W - 1) / W;
  k<<<blocks, W * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename ST, bool HS, bool BULK>
cudaError_t launch_d(const DenseArgs &a, int W, size_t smem, cudaStream_t st) {
  auto k = k_sweep_dense<ST, HS, BULK>;
  std::lock_guard<std::mutex> lk(launch_mutex());
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (a.R + W - 1) / W;
  k<<<blocks, W * 32, smem, st>>>(a);
  return cudaGetLastError();
}

constexpr size_t kSmemLimit = 227 * 1024;

size_t structured_smem(int C, bool d_i16, int W, bool state_smem, bool d_smem) {
  const int Cp = round_up(C, 8);
  const size_t dbytes = d_smem ? align16((size_t)C * Cp * (d_i16 ? 2 : 4)) : 0;
  const size_t per = 8 * (size_t)Cp + (state_smem ? 4 * structured_gstate_words(C) : 0);
  return dbytes + W * per;
}

size_t dense_smem(int64_t n, int C, int W, bool h_smem, size_t elem_bytes = 0) {
  const int np = round_up((int)n, 8);
  const int nw_pad = round_up((int)((n + 31) >> 5), 4);
  const int Cp = round_up(C > 0 ? C : 1, 8);
  const size_t stage = elem_bytes ? elem_bytes * (size_t)np + 16 : 0;  // bulk row buffer + mbarrier
  const size_t per = (h_smem ? 4 * (size_t)np : 0) + stage + 4 * (size_t)nw_pad + (C > 0 ? 4 * (size_t)Cp : 0);
  return 4 * (size_t)nw_pad + W * per;
}

}  // namespace

size_t structured_gstate_words(int C) {
  const int n = C * C;
  return (size_t)round_up(((n + 31) >> 5) + 1, 4);
}

bool structured_state_fits_smem(int C, bool d_i16, int W) {
  const int Cp = round_up(C, 8);
  const bool d_smem = (size_t)C * Cp * (d_i16 ? 2 : 4) <= 96 * 1024;
  return structured_smem(C, d_i16, W, true, d_smem) <= kSmemLimit;
}

cudaError_t launch_structured(const StructArgs &a, bool d_i16, int W, bool want_state_smem,
                              cudaStream_t st, LaunchInfo *info) {
  const int Cp = a.Cp;
  bool d_smem = (size_t)a.C * Cp * (d_i16 ? 2 : 4) <= 96 * 1024;
  bool state_smem = want_state_smem && structured_smem(a.C, d_i16, W, true, d_smem) <= kSmemLimit;
  if (!state_smem && a.gstate == nullptr) return cudaErrorInvalidValue;
  size_t smem = structured_smem(a.C, d_i16, W, state_smem, d_smem);
  if (smem > kSmemLimit) {
    d_smem = false;
    smem = structured_smem(a.C, d_i16, W, state_smem, d_smem);
  }
  if (smem > kSmemLimit) return cudaErrorInvalidValue;
  if (info) {
    info->warps_per_cta = W;
    info->blocks = (a.R + W - 1) / W;
    info->smem = smem;
    info->variant = state_smem ? (d_smem ? "state:smem,d:smem" : "state:smem,d:global")
                               : (d_smem ? "state:global,d:smem" : "state:global,d:global");
  }
  if (d_i16) {
    if (state_smem) return d_smem ? launch_s<int16_t, true, true>(a, W, smem, st) : launch_s<int16_t, true, false>(a, W, smem, st);
    return d_smem ? launch_s<int16_t, false, true>(a, W, smem, st) : launch_s<int16_t, false, false>(a, W, smem, st);
  }
  if (state_smem) return d_smem ? launch_s<int32_t, true, true>(a, W, smem, st) : launch_s<int32_t, true, false>(a, W, smem, st);
  return d_smem ? launch_s<int32_t, false, true>(a, W, smem, st) : launch_s<int32_t, false, false>(a, W, smem, st);
}

bool dense_h_fits_smem(int64_t n, int C, int W) { return dense_smem(n, C, W, true) <= kSmemLimit; }

cudaError_t launch_dense(const DenseArgs &a, bool s_i16, int W, cudaStream_t st, LaunchInfo *info) {
  const bool h_smem = dense_smem(a.n, a.C, W, true) <= kSmemLimit;
  if (!h_smem && a.hbuf == nullptr) return cudaErrorInvalidValue;
  const size_t eb = s_i16 ? 2 : 4;
  const bool bulk = h_smem && dense_smem(a.n, a.C, W, true, eb) <= kSmemLimit;
  const size_t smem = dense_smem(a.n, a.C, W, h_smem, bulk ? eb : 0);
  if (smem > kSmemLimit) return cudaErrorInvalidValue;
  if (info) {
    info->warps_per_cta = W;
    info->blocks = (a.R + W - 1) / W;
    info->smem = smem;
    info->variant = bulk ? "h:smem, rows by bulk copy" : (h_smem ? "h:smem" : "h:global");
  }
  if (s_i16) {
    if (bulk) return launch_d<int16_t, true, true>(a, W, smem, st);
    return h_smem ? launch_d<int16_t, true, false>(a, W, smem, st) : launch_d<int16_t, false, false>(a, W, smem, st);
  }
  if (bulk) return launch_d<int32_t, true, true>(a, W, smem, st);
  return h_smem ? launch_d<int32_t, true, false>(a, W, smem, st) : launch_d<int32_t, false, false>(a, W, smem, st);
}

cudaError_t launch_build_dense(void *S, bool s_i16, int32_t np, int32_t C, const int32_t *d32,
                               int32_t A, int32_t B, cudaStream_t st, const int32_t *w) {
  const int threads = 256, blocks = 152 * 8;
  if (s_i16) k_build_dense<int16_t><<<blocks, threads, 0, st>>>(static_cast<int16_t *>(S), np, C, d32, A, B, w);
  else k_build_dense<int32_t><<<blocks, threads, 0, st>>>(static_cast<int32_t *>(S), np, C, d32, A, B, w);
  return cudaGetLastError();
}

cudaError_t launch_decode(const uint8_t *states, int32_t R, int32_t C, const int32_t *d32,
                          int32_t *paths, int64_t *lengths, cudaStream_t st) {
  int W = 8;
  while (W > 1 && (size_t)W * C * 4 > 48 * 1024) W >>= 1;
  const size_t smem = (size_t)W * C * 4;
  if (smem > 48 * 1024) return cudaErrorInvalidValue;
  k_decode<<<(R + W - 1) / W, W * 32, smem, st>>>(states, R, C, d32, paths, lengths);
  return cudaGetLastError();
}

}  // namespace qp

namespace qp {
std::mutex &launch_mutex() {
  static std::mutex mu;
  return mu;
}

namespace chk {
QP_CHECK_ACCESSOR(kernels)
int32_t enabled() { return QP_DEVICE_CHECKS; }
}  // namespace chk
}  // namespace qp
