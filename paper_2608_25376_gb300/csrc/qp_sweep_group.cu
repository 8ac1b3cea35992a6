// Grouped structured sweep: G replicas per warp for small fields (sm_103a).
//
// The same chain as the row kernel (qp_sweep_rows.cu), with the warp split
// into G groups of 32/G lanes, each group annealing its own replica.  Lane gl
// of a group owns the 8 columns i = 8 gl + j (j = 0..7), so a group covers
// 256/G columns: G = 2 for C <= 128, G = 4 for C <= 64.  Per row, every
// per-row overhead (votes, reductions, loop control, the loads of the next
// row) serves G replicas at once, and each lane has 8 independent proposals
// to evaluate.  Group-local quantities use the whole warp's votes and
// reductions: a ballot is split by lane range, and a per-group sum is packed
// into one register (the group's count shifted into its own 32/G-bit field).
//
// Per group and row t: x (8 bits per lane), 2A x column sum (registers), the
// distance fields of rows t-1, t, t+1 (registers, rotated), the row sum r.
// dE = base - 2A + 2A r (x = 0) or 6A - base - 2A r (x = 1),
// base = B (F_{t-1} + F_{t+1})(i) + 2A c_i.
// A row is skipped unless some proposal has dE <= 0 or 1 <= dE < len_s; then
// the group evaluates against the current state, takes its first accepted
// proposal, applies it and resumes after it (groups without one wait), which
// is the sequential order.  Draws: word k&3 of Philox4x32-10(k>>2, sweep,
// replica, tag); a lane's 8 proposals span counter blocks b0, b0+1 and (when
// t*C is not a multiple of 4) b0+2, which is the next lane's b0.
#include <climits>

#include "qp_device.cuh"
#include "qp_internal.h"

namespace qp {
namespace {

using namespace dev;

constexpr int V = 8;  // columns per lane

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

// 8 consecutive entries of row h of d, from column i (a multiple of 8).
// DMODE 0: global (DT), 1: shared (DT), 2: shared widened to int32.
template <typename DT, int DMODE>
__device__ __forceinline__ void drow8(const void *d, int Cp, int C, int h, int i, bool ok, int (&v)[V]) {
#pragma unroll
  for (int j = 0; j < V; ++j) v[j] = 0;
  if (!ok) return;
  h = QP_IX(h, C, 2);  // the eight entries i..i+7 < Cp of row h
  i = QP_IX(i, Cp - 7, 2);
  if (DMODE == 2) {
    const int4 *p = reinterpret_cast<const int4 *>(static_cast<const int *>(d) + (size_t)h * Cp + i);
    const int4 q0 = p[0], q1 = p[1];
    v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
    v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
  } else if (sizeof(DT) == 2) {
    const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const DT *>(d) + (size_t)h * Cp + i);
    const uint4 q = DMODE == 1 ? *p : __ldg(p);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      v[2 * e] = (int)(short)(w[e] & 0xFFFFu);
      v[2 * e + 1] = (int)w[e] >> 16;
    }
  } else {
    const int4 *p = reinterpret_cast<const int4 *>(static_cast<const DT *>(d) + (size_t)h * Cp + i);
    const int4 q0 = DMODE == 1 ? p[0] : __ldg(p), q1 = DMODE == 1 ? p[1] : __ldg(p + 1);
    v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
    v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
  }
}

template <typename DT, int DMODE>
__device__ __forceinline__ void add_drow8(const void *d, int Cp, int C, int h, int ib, int dlt, int (&F)[V]) {
  int v[V];
  drow8<DT, DMODE>(d, Cp, C, h, ib, ib < C, v);
#pragma unroll
  for (int j = 0; j < V; ++j) F[j] += dlt * v[j];
}

__device__ __forceinline__ int sel8(const int (&v)[V], int j) {
  int r = v[0];
#pragma unroll
  for (int k = 1; k < V; ++k) r = (j == k) ? v[k] : r;
  return r;
}

template <int G>
struct Grp {
  static constexpr int L = 32 / G;                    // lanes per group
  static constexpr unsigned kMask = (G == 1) ? 0xffffffffu : ((1u << L) - 1u);
  static constexpr int kBits = 32 / G;                // packed-sum field width
  __device__ static int sum(int v, int g) {           // v < 2^kBits per group
    const unsigned tot = __reduce_add_sync(kFull, (unsigned)v << (kBits * g));
    return (int)((tot >> (kBits * g)) & ((kBits == 32) ? 0xffffffffu : ((1u << kBits) - 1u)));
  }
  __device__ static long long sum64(long long v) {
#pragma unroll
    for (int o = L / 2; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
  }
  __device__ static unsigned mine(unsigned bal, int g) { return (bal >> (L * g)) & kMask; }
};

// F += the d rows of the set bits of this group's row (bits beyond C are 0).
template <typename DT, int DMODE, int G>
__device__ __forceinline__ void scan_field(const uint32_t *row, int Cw, const void *d, int Cp, int C, int g, int gl,
                                           int ib, int (&F)[V]) {
  constexpr int LL = Grp<G>::L;
  const uint32_t word = gl < Cw ? row[gl] : 0u;
  uint32_t bal = __ballot_sync(kFull, word != 0u);
  while (bal) {
    const int src = __ffs(bal) - 1;
    bal &= bal - 1;
    uint32_t wd = __shfl_sync(kFull, word, src);
    const bool mine = src / LL == g;
    const int wbase = (src % LL) << 5;
    while (wd) {
      const int h = wbase + __ffs(wd) - 1;
      wd &= wd - 1;
      if (mine) add_drow8<DT, DMODE>(d, Cp, C, h, ib, 1, F);
    }
  }
}

// The single set cell of this group's row, or -1.
template <int G>
__device__ __forceinline__ int single_cell(const uint32_t *row, int Cw, int g, int gl) {
  constexpr int LL = Grp<G>::L;
  const uint32_t word = gl < Cw ? row[gl] : 0u;
  const int cnt = Grp<G>::sum(__popc(word), g);
  const unsigned bal = Grp<G>::mine(__ballot_sync(kFull, word != 0u), g);
  const int src = bal ? __ffs(bal) - 1 + LL * g : LL * g;
  const uint32_t wd = __shfl_sync(kFull, word, src);
  return (cnt == 1) ? (((src % LL) << 5) + __ffs(wd) - 1) : -1;
}

template <typename DT, int DMODE, int G>
__global__ void __launch_bounds__(kMaxWarpsPerCta * 32) k_sweep_group(const StructArgs a) {
  constexpr int LL = Grp<G>::L;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int g = lane / LL, gl = lane % LL;
  const int C = a.C, Cp = a.Cp, s0 = a.start, A = a.A, B = a.B;
  const int twoA = 2 * A;
  const int Cw = (C + 31) >> 5;
  const int n = C * C;
  unsigned char *p = smem;
  const void *d = a.d;
  if (DMODE == 1) {
    const int nv = (int)((size_t)C * Cp * sizeof(DT) / 16);
    const int4 *src = static_cast<const int4 *>(a.d);
    int4 *dst = reinterpret_cast<int4 *>(p);
    for (int v = threadIdx.x; v < nv; v += blockDim.x) dst[v] = __ldg(src + v);
    d = p;
    p += al16((size_t)C * Cp * sizeof(DT));
  } else if (DMODE == 2) {
    const DT *src = static_cast<const DT *>(a.d);
    int *dst = reinterpret_cast<int *>(p);
    for (int e = threadIdx.x; e < C * Cp; e += blockDim.x) dst[e] = (int)__ldg(src + e);
    d = p;
    p += al16((size_t)C * Cp * 4);
  }
  const size_t per_rep = 4 * (size_t)a.nw_pad + al16(2 * (size_t)C);
  unsigned char *gp = p + ((size_t)warp * G + g) * per_rep;
  uint32_t *st = reinterpret_cast<uint32_t *>(gp);
  int16_t *hot1 = reinterpret_cast<int16_t *>(gp + 4 * (size_t)a.nw_pad);
  __syncthreads();
  const int r = (blockIdx.x * W + warp) * G + g;
  if (__all_sync(kFull, r >= a.R)) return;  // no CTA-wide barrier after this point
  const bool active = r < a.R;                // idle groups follow along without output
  const uint32_t rg = (uint32_t)(a.rep_offset + r);
  const int ib = V * gl;
  const int wsh = ib & 31, wix = ib >> 5;    // the lane's 8 bits in a row: word wix, from bit wsh

  // ---- initial state
  const uint8_t *init = (active && a.init) ? a.init + (size_t)r * n : nullptr;
  for (int e = gl; e < C * Cw; e += LL) {
    const int t = e / Cw, w = e - t * Cw;
    uint32_t word = 0;
    if (t == 0) {
      if ((s0 >> 5) == w) word = 1u << (s0 & 31);
    } else if (init) {
      for (int b = 0; b < 32; ++b) {
        const int i = (w << 5) + b;
        if (i < C && i != s0 && init[(size_t)t * C + i]) word |= 1u << b;
      }
    }
    st[e] = word;
  }
  __syncwarp();
  int validm = 0;
#pragma unroll
  for (int j = 0; j < V; ++j)
    if (ib + j < C && ib + j != s0) validm |= 1 << j;
  if (!active) validm = 0;

  // ---- column sums, single-cell cache, energy (Eqs. 3-6) of this group's replica
  int cs[V];
#pragma unroll
  for (int j = 0; j < V; ++j) cs[j] = 0;
  long long hd = 0, pen_rows = 0;
  int viol = 0;
  for (int t = 0; t < C; ++t) {
    const uint32_t *row = st + t * Cw;
    const int xb = ib < C ? (int)((row[wix] >> wsh) & 0xFFu) : 0;
#pragma unroll
    for (int j = 0; j < V; ++j) cs[j] += (xb >> j) & 1;
    const int rsum = Grp<G>::sum(__popc(xb), g);
    pen_rows += (long long)(1 - rsum) * (1 - rsum);
    viol += rsum != 1;
    const int h1 = single_cell<G>(row, Cw, g, gl);
    if (gl == 0) hot1[t] = (int16_t)h1;
    if (t + 1 < C) {
      int Fn[V];
#pragma unroll
      for (int j = 0; j < V; ++j) Fn[j] = 0;
      scan_field<DT, DMODE, G>(row + Cw, Cw, d, Cp, C, g, gl, ib, Fn);
#pragma unroll
      for (int j = 0; j < V; ++j)
        if ((xb >> j) & 1) hd += Fn[j];
    }
  }
  __syncwarp();
  long long pen_cols = 0;
  int viol_cols = 0;
#pragma unroll
  for (int j = 0; j < V; ++j)
    if (ib + j < C) {
      pen_cols += (long long)(1 - cs[j]) * (1 - cs[j]);
      viol_cols += cs[j] != 1;
    }
  long long E = (long long)B * Grp<G>::sum64(hd) + (long long)A * (pen_rows + Grp<G>::sum64(pen_cols));
  viol += Grp<G>::sum(viol_cols, g);
  int tAc[V];
#pragma unroll
  for (int j = 0; j < V; ++j) tAc[j] = twoA * cs[j];
  long long best = LLONG_MAX, acc = 0;

  // ---- sweeps
  for (int s = a.sweep_begin; s < a.sweep_end; ++s) {
    const uint32_t *thr = a.thr + a.thr_off[s];
    const int len = a.thr_len[s];
    const unsigned lenm1 = (unsigned)(len - 1);
    const unsigned hit_lo = 0x80000000u - lenm1;
    const float cT = a.thr_c[s];
    int P[V], Cu[V], N[V], Nn[V];
#pragma unroll
    for (int j = 0; j < V; ++j) P[j] = Cu[j] = Nn[j] = 0;
    add_drow8<DT, DMODE>(d, Cp, C, s0, ib, 1, P);
    {
      const int h = hot1[1];
      if (__all_sync(kFull, h >= 0)) add_drow8<DT, DMODE>(d, Cp, C, h, ib, 1, Cu);
      else if (h >= 0) add_drow8<DT, DMODE>(d, Cp, C, h, ib, 1, Cu);
      if (__any_sync(kFull, h < 0)) {
        int tmp[V];
#pragma unroll
        for (int j = 0; j < V; ++j) tmp[j] = 0;
        scan_field<DT, DMODE, G>(st + Cw, Cw, d, Cp, C, g, gl, ib, tmp);
        if (h < 0)
#pragma unroll
          for (int j = 0; j < V; ++j) Cu[j] += tmp[j];
      }
    }
    if (C > 2) {
      const int h = hot1[2];
      if (h >= 0) add_drow8<DT, DMODE>(d, Cp, C, h, ib, 1, Nn);
      if (__any_sync(kFull, h < 0)) {
        int tmp[V];
#pragma unroll
        for (int j = 0; j < V; ++j) tmp[j] = 0;
        scan_field<DT, DMODE, G>(st + 2 * Cw, Cw, d, Cp, C, g, gl, ib, tmp);
        if (h < 0)
#pragma unroll
          for (int j = 0; j < V; ++j) Nn[j] += tmp[j];
      }
    }
    int h2 = C > 3 ? hot1[3] : -1;
    int xnn = (C > 1 && ib < C) ? (int)((st[Cw + wix] >> wsh) & 0xFFu) : 0;
    for (int t = 1; t < C; ++t) {
      uint32_t *row = st + t * Cw;
      const int xn0 = xnn;
#pragma unroll
      for (int j = 0; j < V; ++j) {
        N[j] = Nn[j];
        Nn[j] = 0;
      }
      if (t + 2 < C) {
        if (h2 >= 0) add_drow8<DT, DMODE>(d, Cp, C, h2, ib, 1, Nn);
        if (__any_sync(kFull, h2 < 0)) {
          int tmp[V];
#pragma unroll
          for (int j = 0; j < V; ++j) tmp[j] = 0;
          scan_field<DT, DMODE, G>(row + 2 * Cw, Cw, d, Cp, C, g, gl, ib, tmp);
          if (h2 < 0)
#pragma unroll
            for (int j = 0; j < V; ++j) Nn[j] += tmp[j];
        }
      }
      h2 = t + 3 < C ? hot1[t + 3] : -1;
      xnn = (t + 1 < C && ib < C) ? (int)((row[Cw + wix] >> wsh) & 0xFFu) : 0;
      int xn = xn0;
      int rt = Grp<G>::sum(__popc(xn), g);
      const int rt0 = rt;
      const int tC = t * C;
      int base[V];
      unsigned hit = 0;
      {
        const int k0 = twoA * (rt - 1), k1 = twoA * (3 - rt);
#pragma unroll
        for (int j = 0; j < V; ++j) {
          base[j] = B * (P[j] + N[j]) + tAc[j];
          const int de = ((xn >> j) & 1) ? k1 - base[j] : base[j] + k0;
          hit |= (unsigned)((unsigned)(de - 1) - lenm1 >= hit_lo) << j;
        }
      }
      bool flipped = false;
      if (__any_sync(kFull, hit & validm)) {
        int cand = validm;
        bool have = false;
        uint4 u0 = make_uint4(0, 0, 0, 0), u1 = u0, u2 = u0;
        const int delta = tC & 3;
        while (true) {
          const int k0 = twoA * (rt - 1), k1 = twoA * (3 - rt);
          int accm = 0, need = 0, dE[V];
#pragma unroll
          for (int j = 0; j < V; ++j) {
            dE[j] = ((xn >> j) & 1) ? k1 - base[j] : base[j] + k0;
            const unsigned dm1 = (unsigned)(dE[j] - 1);
            accm |= (int)(dm1 >> 31) << j;
            need |= (int)(dm1 < lenm1) << j;
          }
          accm &= cand;
          need &= cand;
          if (__any_sync(kFull, need != 0)) {
            if (!have) {
              const uint32_t b0 = (uint32_t)((tC + ib) >> 2);
              u0 = philox4x32_10(make_uint4(b0, (uint32_t)s, rg, kRngTag), a.key0, a.key1);
              u1 = philox4x32_10(make_uint4(b0 + 1, (uint32_t)s, rg, kRngTag), a.key0, a.key1);
              u2.x = __shfl_down_sync(kFull, u0.x, 1);
              u2.y = __shfl_down_sync(kFull, u0.y, 1);
              u2.z = __shfl_down_sync(kFull, u0.z, 1);
              u2.w = __shfl_down_sync(kFull, u0.w, 1);
              // the group's last lane: its third block belongs to no neighbour
              if (delta != 0 && gl == LL - 1 && C > ib + 8 - delta)
                u2 = philox4x32_10(make_uint4(b0 + 2, (uint32_t)s, rg, kRngTag), a.key0, a.key1);
              have = true;
            }
#pragma unroll
            for (int j = 0; j < V; ++j) {
              if ((need >> j) & 1) {
                const int kb = (delta + j) >> 2, w = (delta + j) & 3;
                const uint32_t u = kb == 0 ? word_of(u0, w) : (kb == 1 ? word_of(u1, w) : word_of(u2, w));
                if (accept_draw(u, dE[j], cT, thr, len)) accm |= 1 << j;
              }
            }
          }
          const unsigned bal = __ballot_sync(kFull, accm != 0);
          if (bal == 0) break;
          const unsigned mb = Grp<G>::mine(bal, g);
          const int Lg = mb ? __ffs(mb) - 1 + LL * g : LL * g;  // first accepting lane of my group
          const int jl = accm ? __ffs(accm) - 1 : 0;
          const int xl = (xn >> jl) & 1;
          const int tc = sel8(tAc, jl);
          const int pk0 = jl | (xl << 3) | ((tc == twoA) << 4) | ((tc + (1 - 2 * xl) * twoA == twoA) << 5);
          const int de = __shfl_sync(kFull, sel8(dE, jl), Lg);
          const int pk = __shfl_sync(kFull, pk0, Lg);
          const int jj = pk & 7, dlt = 1 - 2 * ((pk >> 3) & 1);
          const int istar = V * (Lg % LL) + jj;
          if (mb) {
            E += de;
            ++acc;
            rt += dlt;
            viol += ((pk >> 5) & 1 ? 0 : 1) - ((pk >> 4) & 1 ? 0 : 1);
            flipped = true;
            if (lane == Lg) {
#pragma unroll
              for (int j = 0; j < V; ++j)
                if (j == jj) tAc[j] += dlt * twoA;
              xn ^= 1 << jj;
              row[istar >> 5] ^= 1u << (istar & 31);
            }
            add_drow8<DT, DMODE>(d, Cp, C, istar, ib, dlt, Cu);
            cand &= gl < (Lg % LL) ? 0 : (gl > (Lg % LL) ? 0xFF : (0xFF << (jj + 1)) & 0xFF);
          }
          __syncwarp();
        }
      }
      viol += (rt != 1) - (rt0 != 1);
      if (__any_sync(kFull, flipped)) {
        const int h1v = single_cell<G>(row, Cw, g, gl);
        if (flipped && gl == 0) hot1[t] = (int16_t)h1v;
        __syncwarp();
      }
#pragma unroll
      for (int j = 0; j < V; ++j) {
        P[j] = Cu[j];
        Cu[j] = N[j];
      }
    }
    if (viol == 0 && E < best) best = E;
  }

  // ---- outputs
  if (active) {
    uint8_t *out = a.states_out + (size_t)r * n;
    for (int e = gl; e < n; e += LL) {
      const int t = e / C, i = e - t * C;
      out[e] = (uint8_t)((st[t * Cw + (i >> 5)] >> (i & 31)) & 1u);
    }
    if (gl == 0) {
      a.E_out[r] = E;
      if (a.best_out) a.best_out[r] = best;
      if (a.acc_out) a.acc_out[r] = acc;
    }
  }
}

constexpr size_t kSmemLimitGroup = 227 * 1024;

size_t group_state_words(int C) {
  const int Cw = (C + 31) / 32;
  return (size_t)(C * Cw + 3) / 4 * 4;
}

size_t group_smem(int C, bool d_i16, int W, int G, int dmode) {
  const int Cp = (C + 7) / 8 * 8;
  size_t dbytes = 0;
  if (dmode == 1) dbytes = al16((size_t)C * Cp * (d_i16 ? 2 : 4));
  if (dmode == 2) dbytes = al16((size_t)C * Cp * 4);
  return dbytes + (size_t)W * G * (4 * group_state_words(C) + al16(2 * (size_t)C));
}

template <typename DT, int DMODE, int G>
cudaError_t launch_g(const StructArgs &a, int W, size_t smem, cudaStream_t st) {
  auto k = k_sweep_group<DT, DMODE, G>;
  std::lock_guard<std::mutex> lk(launch_mutex());
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int reps_per_cta = W * G;
  k<<<(a.R + reps_per_cta - 1) / reps_per_cta, W * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename DT, int G>
cudaError_t launch_g2(const StructArgs &a, int dmode, int W, size_t smem, cudaStream_t st) {
  if (dmode == 2) return launch_g<DT, 2, G>(a, W, smem, st);
  if (dmode == 1) return launch_g<DT, 1, G>(a, W, smem, st);
  return launch_g<DT, 0, G>(a, W, smem, st);
}

}  // namespace

int group_size_for(int C) { return C <= 64 ? 4 : (C <= 128 ? 2 : 1); }

bool group_supported(int C, bool d_i16, int W) {
  const int G = group_size_for(C);
  return G > 1 && W >= 1 && W <= kMaxWarpsPerCta && group_smem(C, d_i16, W, G, 0) <= kSmemLimitGroup;
}

cudaError_t launch_group(const StructArgs &a_in, bool d_i16, int W, cudaStream_t st, LaunchInfo *info) {
  StructArgs a = a_in;
  if (!group_supported(a.C, d_i16, W)) return cudaErrorInvalidValue;
  const int G = group_size_for(a.C);
  a.nw_pad = (int32_t)group_state_words(a.C);
  int dmode = 0;
  if (group_smem(a.C, d_i16, W, G, 2) <= kSmemLimitGroup) dmode = 2;
  else if (group_smem(a.C, d_i16, W, G, 1) <= kSmemLimitGroup) dmode = 1;
  const size_t smem = group_smem(a.C, d_i16, W, G, dmode);
  if (info) {
    info->warps_per_cta = W;
    info->blocks = (a.R + W * G - 1) / (W * G);
    info->smem = smem;
    info->variant = G == 4 ? "group4" : "group2";
  }
  if (d_i16) return G == 4 ? launch_g2<int16_t, 4>(a, dmode, W, smem, st) : launch_g2<int16_t, 2>(a, dmode, W, smem, st);
  return G == 4 ? launch_g2<int32_t, 4>(a, dmode, W, smem, st) : launch_g2<int32_t, 2>(a, dmode, W, smem, st);
}

}  // namespace qp

namespace qp {
namespace chk {
QP_CHECK_ACCESSOR(group)
}  // namespace chk
}  // namespace qp
