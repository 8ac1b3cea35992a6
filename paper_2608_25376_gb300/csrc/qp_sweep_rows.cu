// Row-parallel structured sweep for fields of up to 512 cells (sm_103a).
//
// One warp anneals one replica.  The sweep proposes x_{t,i} for t = 1..C-1 and
// every cell i != s in increasing i, exactly as the sequential chain does.
// Lane L owns the columns i = 128c + 4L + j (j = 0..3, chunk c < NCH) for the
// whole run, so everything indexed by column lives in its registers:
//   tAc[c][j]  2A times the column sums sum_t x_{t,i} (Eq. 4),
//   P, Cu, N   the distance fields F_u(i) = sum_{h : x_{u,h} = 1} d_{h,i} of
//              rows t-1, t and t+1 (Eq. 3), rotated from row to row; an accepted
//              flip in row t adds one row of d to Cu, and row t+1's field is the
//              d row of its single hot cell (cached per row) or, when the row
//              does not hold exactly one cell, a scan of its bits.
// With r the row-t sum and c_i the column sum (both including x), Eq. 6 gives
//   dE = base - 2A + 2A r          (x = 0)
//   dE = 6A - base - 2A r          (x = 1),     base = B (F_{t-1} + F_{t+1})(i) + 2A c_i.
// A row chunk (128 proposals) is first tested as a whole: a proposal matters
// only if dE < len_s (accepted outright when dE <= 0, decided by a draw when
// 1 <= dE < len_s), one compare each, and at low temperature most rows have
// none, so they cost a few instructions per proposal.  Otherwise the warp
// evaluates the chunk against the current state, a ballot finds the first
// accepted proposal, the flip is applied and evaluation resumes after it:
// exactly the sequential order.  The spins are a bitset per row
// (Cw = ceil(C/32) words) in shared memory; the distance matrix is staged in
// shared memory (widened to int32 when that fits) or read from L2.
//
// The draw of x_{t,i} is word k&3 of Philox4x32-10(counter = (k>>2, sweep,
// replica, tag)), k = t*C + i; a lane's four proposals span one or two counter
// blocks, each computed only when one of its proposals has 1 <= dE < len_s.
// Most draws are rejected by two integer compares (u >= thr[dq] with
// dq ~ 8 T ln 2 and dE >= dq) before the float estimate of exp(-dE/T).
#include <climits>
#include <map>
#include <mutex>
#include <tuple>

#include "qp_device.cuh"
#include "qp_internal.h"

namespace qp {
namespace {

using namespace dev;

#include "qp_rows.cuh"

// One replica of a field through the sweeps [sweep_begin, sweep_end): the
// whole chain of the row kernel, shared by the single-field launch and the
// batched persistent launch.  st: the replica's C x Cw row bitsets; hot1: its
// per-row single-cell cache (C entries); d: the distance matrix (global or
// shared memory, per DMODE).
template <typename DT, int NCH, int DMODE, int LA>
__device__ __forceinline__ void rows_replica(const StructArgs &a, int r, uint32_t *st, int16_t *hot1,
                                             const void *d, int lane) {
  static_assert(LA == 1 || LA == 2, "field look-ahead of 1 or 2 rows");
  const int C = a.C, Cp = a.Cp, s0 = a.start, A = a.A, B = a.B;
  const int twoA = 2 * A;
  const int Cw = (C + 31) >> 5;
  const int n = C * C;
  const uint32_t rg = (uint32_t)(a.rep_offset + r);

  int tAc[NCH][4];  // 2A * column sum, kept through the sweeps
  int validc[NCH];
  long long E;
  int viol;
  rows_init<DT, NCH, DMODE>(a, r, st, hot1, d, lane, tAc, validc, E, viol);
  long long best = LLONG_MAX, acc = 0;

  // ---- sweeps
  const int lev = a.level ? __ldg(a.level + r) : -1;
  // A sweep that met no proposal with dE < len leaves the state as it was, so
  // every later sweep with a table no longer than len does too (each of its
  // proposals sees the same state and the same dE): those sweeps are skipped
  // when asked to (results unchanged).
  bool settled = false;
  int settled_len = 0;
  for (int s = a.sweep_begin; s < a.sweep_end; ++s) {
    const int ts = lev >= 0 ? lev : s;  // table row: the sweep, or the replica's ladder level
    const uint32_t *thr = a.thr + a.thr_off[ts];
    const int len = a.thr_len[ts];
    if (settled && len <= settled_len) continue;
    bool any_hit = false;
    const unsigned lenm1 = (unsigned)(len - 1);
    const float cT = a.thr_c[ts];
    // quick rejection: a draw u >= thr[dq] rejects every dE >= dq (thr is
    // non-increasing); dq ~ 8 T ln 2 puts thr[dq] near 2^24, so almost every
    // draw of a proposal with dE >= dq is rejected by two compares
    const int dq = len > 1 ? min(len - 1, max(1, (int)fminf(8.0f / cT, 1.0e9f))) : 1;
    const uint32_t Q = len > 1 ? __ldg(a.thr + a.thr_off[ts] + dq) : 0u;
    // P, Cu, N: the fields of rows t-1, t, t+1; N1 (and N2 when LA = 2): rows
    // t+2 (and t+3).  Row t+1+LA's field is loaded LA rows ahead of its use, so
    // an L2 read of d (LA = 2 when d is in global memory) has that many rows of
    // work to hide behind.
    int P[NCH][4], Cu[NCH][4], N[NCH][4], N1[NCH][4], N2[NCH][4];
    int(&NL)[NCH][4] = LA == 2 ? N2 : N1;  // the field being loaded
    zero<NCH>(P);
    zero<NCH>(Cu);
    zero<NCH>(N1);
    zero<NCH>(N2);
    add_drow<DT, NCH, DMODE>(d, Cp, C, s0, lane, 1, P);  // row 0 holds only the start cell
    row_field<DT, NCH, DMODE>(st, Cw, hot1, 1, d, Cp, C, lane, Cu);
    if (C > 2) row_field<DT, NCH, DMODE>(st, Cw, hot1, 2, d, Cp, C, lane, N1);
    if (LA == 2 && C > 3) row_field<DT, NCH, DMODE>(st, Cw, hot1, 3, d, Cp, C, lane, N2);
    int hl = C > 2 + LA ? hot1[2 + LA] : -1;  // the single cell of row t+1+LA
    int hc = hot1[1];                          // the single cell of row t
    for (int t = 1; t < C; ++t) {
      uint32_t *row = st + t * Cw;
      int xn[NCH];
      int rt;
#pragma unroll
      for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          N[c][j] = N1[c][j];
          if (LA == 2) N1[c][j] = N2[c][j];
        }
      // F_{t+1+LA}: the d row of that row's single hot cell, else a scan of its bits
      if (t + 1 + LA < C && hl >= 0) {
        set_drow<DT, NCH, DMODE>(d, Cp, C, hl, lane, NL);
      } else {
        zero<NCH>(NL);
        if (t + 1 + LA < C) {
          int one;
          scan_row_field<DT, NCH, DMODE>(row + (1 + LA) * Cw, Cw, d, Cp, C, lane, NL, &one);
        }
      }
      hl = t + 2 + LA < C ? hot1[t + 2 + LA] : -1;
      const int hcn = t + 1 < C ? hot1[t + 1] : -1;
      // row t's sum: 1 from the cache when the row holds exactly one cell (its
      // bit groups are then derived only if the row needs the exact evaluation),
      // else from its bits
      if (hc >= 0) {
        rt = 1;
      } else {
        rt = 0;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          xn[c] = 128 * c + 4 * lane < C ? (int)((row[4 * c + (lane >> 3)] >> (4 * (lane & 7))) & 0xFu) : 0;
          rt += __popc(xn[c]);
        }
        rt = __reduce_add_sync(kFull, rt);
      }
      const int rt0 = rt;
      bool flipped = false;
      const int tC = t * C;
      // The whole row first, as one test: with base = B f + 2A c_i, a proposal
      // can matter (dE < len) only if base < len - 2A(r-1) (x = 0) or
      // base > 2A(3-r) - len (x = 1).  Both bounds for every column give a
      // superset of the proposals that matter (columns outside the field carry
      // base = 2A, inside both bounds when r = 1 and len < 2A); when none
      // passes, no proposal of the row can flip or needs a draw.
      // the whole row first, as one test (row_pretest's bounds as two compares)
      bool maybe = false;
      {
        const int lo = len - twoA * (rt - 1), hi = twoA * (3 - rt) - len;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          if (128 * c >= C) break;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int b = B * (P[c][j] + N[c][j]) + tAc[c][j];
            maybe |= (b < lo) | (b > hi);
          }
        }
      }
      if (__any_sync(kFull, maybe)) {
        if (hc >= 0) {
#pragma unroll
          for (int c = 0; c < NCH; ++c) xn[c] = (hc >> 2) == 32 * c + lane ? 1 << (hc & 3) : 0;
        }
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          if (128 * c >= C) break;
          // base = B f + 2A c_i;  dE = base + 2A(r-1) (x = 0),  2A(3-r) - base (x = 1)
          int base[4], de[4];
          unsigned hit = 0;
          {
            const int k0 = twoA * (rt - 1), k1 = twoA * (3 - rt);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              base[j] = B * (P[c][j] + N[c][j]) + tAc[c][j];
              de[j] = ((xn[c] >> j) & 1) ? k1 - base[j] : base[j] + k0;
              // the proposal matters iff dE <= 0 (accepted) or 1 <= dE < len (a draw decides): dE < len
              hit |= (unsigned)(de[j] < len) << j;
            }
          }
          if (__any_sync(kFull, hit & validc[c])) {
            any_hit = true;
            flipped |= row_chunk<DT, NCH, DMODE>(c, t, s, tC, base, de, xn[c], validc[c], tAc[c], rt, Cu, row, E,
                                                 acc, viol, d, Cp, C, lane, twoA, len, lenm1, cT, dq, Q, thr, rg,
                                                 PhiloxKey{a.key0, a.key1});
          }
        }
      }
      viol += (rt != 1) - (rt0 != 1);
      if (flipped) {
        const int h1v = row_single(row, Cw, lane);
        if (lane == 0) hot1[t] = (int16_t)h1v;
        __syncwarp();
      }
#pragma unroll
      for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          P[c][j] = Cu[c][j];
          Cu[c][j] = N[c][j];
        }
      hc = hcn;
    }
    if (viol == 0 && E < best) best = E;
    settled = a.skip_settled && !any_hit;
    settled_len = len;
  }

  // ---- outputs
  uint8_t *out = a.states_out + (size_t)r * n;
  for (int e = lane; e < n; e += 32) {
    const int t = e / C, i = e - t * C;
    out[e] = (uint8_t)((st[t * Cw + (i >> 5)] >> (i & 31)) & 1u);
  }
  if (lane == 0) {
    a.E_out[r] = E;
    if (a.best_out) a.best_out[r] = best;
    if (a.acc_out) a.acc_out[r] = acc;
  }
}


// ---------------------------------------------------------------------------
// Wide fields whose distance matrix lives in L2 (more than 256 cells, d not in
// shared memory): the same chain with the spins in global memory.  A replica's
// C x Cw row bitsets take 31 KB at 491 cells, and in shared memory they held
// the SM to 7 replicas; here shared memory keeps only, per replica, the
// single-cell cache hot[t] (the cell when row t holds exactly one, -1 when it
// holds none, -2 when it holds several) and a ring of K distance rows that
// cp.async fills K-1 rows ahead of use, so the L2 latency of d stays off the
// row's dependent chain.  A row that holds one cell or none needs no bits at
// all: its four-bit groups and sum follow from hot[t]; only rows with several
// cells read their bits (from L2).  Flips reach the bits by atomic XOR (no
// wait); the cache of a flipped row is rebuilt from the lanes' registers.

// cp.async (global -> shared, BYTES = 4, 8 or 16), group commit and wait
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The field of row u for the global-spins kernel: the d row of its single
// cell, zero for an empty row, a scan of its bits (from L2) otherwise.
template <typename DT, int NCH>
__device__ __forceinline__ void field_g(const uint32_t *st, int Cw, int code, int u, const void *d, int Cp, int C,
                                        int lane, int (&F)[NCH][4]) {
  if (code >= 0) set_drow<DT, NCH, 0>(d, Cp, C, code, lane, F);
  else {
    zero<NCH>(F);
    if (code == -2) { int one; scan_row_field<DT, NCH, 0, true>(st + (size_t)u * Cw, Cw, d, Cp, C, lane, F, &one); }
  }
}

template <typename DT, int NCH, int K>
__device__ __forceinline__ void ring_issue(const int16_t *hot, DT *ring, const void *d, int Cp, int C, int u,
                                           int lane) {
  if (u >= C) return;
  const int h = hot[u];
  if (h < 0) return;
  // the whole padded row (Cp entries, Cp a multiple of 8) in 16-byte pieces
  // spread over the lanes: a lane's columns come from other lanes' copies,
  // so a reader waits for its own copies and then syncs the warp
  char *slot = reinterpret_cast<char *>(ring + (size_t)((unsigned)u % K) * Cp);
  const char *src = reinterpret_cast<const char *>(static_cast<const DT *>(d) + (size_t)QP_IX(h, C, 2) * Cp);
  const int pieces = Cp * (int)sizeof(DT) / 16;
  constexpr int kIter = (128 * NCH * (int)sizeof(DT) / 16 + 31) / 32;
#pragma unroll
  for (int k = 0; k < kIter; ++k) {
    const int pc = lane + 32 * k;
    if (pc < pieces) cp_async<16>(slot + 16 * pc, src + 16 * pc);
  }
}

// The parameters of the whole-row test that stay fixed through a sweep.
struct RowTest {
  int B, twoA, len, C;
  unsigned W1;  // 4A - 2 len: the range width of the test when r = 1
};

// X0 <- X1 <- X2 <- X3 <- X0
template <int NCH>
__device__ __forceinline__ void rotate_fields(int (&X0)[NCH][4], int (&X1)[NCH][4], int (&X2)[NCH][4],
                                              int (&X3)[NCH][4]) {
#pragma unroll
  for (int c = 0; c < NCH; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int v = X0[c][j];
      X0[c][j] = X1[c][j];
      X1[c][j] = X2[c][j];
      X2[c][j] = X3[c][j];
      X3[c][j] = v;
    }
}

template <int NCH>
__device__ __forceinline__ void swap_fields(int (&X)[NCH][4], int (&Y)[NCH][4]) {
#pragma unroll
  for (int c = 0; c < NCH; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int v = X[c][j];
      X[c][j] = Y[c][j];
      Y[c][j] = v;
    }
}

// The front half of row t, the whole work of a row that cannot flip: F_{t+2}
// into Fl (from its ring slot, or from the row's bits when it does not hold
// exactly one cell), the ring copy of row t+K+1, row t's sum rt (and, for a
// row of several cells, its four-bit groups xn), and the whole-row test
// against P = F_{t-1}, N = F_{t+1}.  hn: the single-cell cache of row t.
template <typename DT, int NCH, int K>
__device__ __forceinline__ bool rows_g_front(const uint32_t *st, const int16_t *hot, DT *ring, const void *d, int Cp,
                                             int C, int Cw, int lane, int t, int hn, const int (&P)[NCH][4],
                                             const int (&N)[NCH][4], int (&Fl)[NCH][4], const int (&tAc)[NCH][4],
                                             const RowTest &rtst, int &rt, int (&xn)[NCH]) {
  if (t + 2 < C) {
    cp_async_wait<K - 2>();  // this lane's copies of row t+2 (issued K-1 rows ago) have landed
    __syncwarp();            // ... and every other lane's
    const int h2 = hot[t + 2];
    if (h2 >= 0) set_drow<DT, NCH, 1>(ring + (size_t)((unsigned)(t + 2) % K) * Cp, Cp, C, 0, lane, Fl);
    else field_g<DT, NCH>(st, Cw, h2, t + 2, d, Cp, C, lane, Fl);
  } else {
    zero<NCH>(Fl);  // past the last row
  }
  // row t+K+1 into the slot row t+1 has left (its data is in N now)
  ring_issue<DT, NCH, K>(hot, ring, d, Cp, C, t + K + 1, lane);
  cp_async_commit();
  // row t's sum (and, for a row of several cells, its bits): from the cache
  // when the row holds one cell or none
  if (hn >= 0) {
    rt = 1;
  } else if (hn == -1) {
    rt = 0;
  } else {
    const uint32_t *row = st + (size_t)t * Cw;
    rt = 0;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      xn[c] = 128 * c + 4 * lane < C ? (int)((__ldcg(row + 4 * c + (lane >> 3)) >> (4 * (lane & 7))) & 0xFu) : 0;
      rt += __popc(xn[c]);
    }
    rt = __reduce_add_sync(kFull, rt);
  }
  return __any_sync(kFull, row_pretest_shifted<NCH>(P, N, tAc, rtst.B, rtst.twoA, rt, rtst.len, rtst.W1));
}

// The back half of a row that may flip (P = F_{t-1}, Cu = F_t, N = F_{t+1}):
// every chunk with a proposal that can be accepted or needs a draw, the
// violation count, and the row's cache entry when a flip changed it.
// Returns whether any proposal had dE < len.
template <typename DT, int NCH>
__device__ __forceinline__ bool rows_g_flip(const StructArgs &a, uint32_t *st, int16_t *hot, const void *d, int Cp,
                                            int C, int Cw, int lane, int t, int s, int hn, int rt, int (&xn)[NCH],
                                            const int (&P)[NCH][4], int (&Cu)[NCH][4], const int (&N)[NCH][4],
                                            int (&tAc)[NCH][4], const int (&validc)[NCH], long long &E,
                                            long long &acc, int &viol, int twoA, int len, unsigned lenm1, float cT,
                                            int dq, uint32_t Q, const uint32_t *thr, uint32_t rg,
                                            const RoundKeys &rk) {
  uint32_t *row = st + (size_t)t * Cw;
  const int rt0 = rt;
  const int B = a.B;
  bool flipped = false, any_hit = false;
  const int tC = t * C;
  if (hn >= 0) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) xn[c] = (hn >> 2) == 32 * c + lane ? 1 << (hn & 3) : 0;
  } else if (hn == -1) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) xn[c] = 0;
  }
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    if (128 * c >= C) break;
    int base[4], de[4];
    unsigned hit = 0;
    {
      const int k0 = twoA * (rt - 1), k1 = twoA * (3 - rt);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        base[j] = B * (P[c][j] + N[c][j]) + tAc[c][j] + len;
        de[j] = ((xn[c] >> j) & 1) ? k1 - base[j] : base[j] + k0;
        hit |= (unsigned)(de[j] < len) << j;
      }
    }
    if (__any_sync(kFull, hit & validc[c])) {
      any_hit = true;
      flipped |= row_chunk<DT, NCH, 0, true>(c, t, s, tC, base, de, xn[c], validc[c], tAc[c], rt, Cu, row, E, acc,
                                             viol, d, Cp, C, lane, twoA, len, lenm1, cT, dq, Q, thr, rg, rk, len);
    }
  }
  viol += (rt != 1) - (rt0 != 1);
  if (flipped) {
    int code = rt == 0 ? -1 : -2;
    if (rt == 1) {
      int mine = -1;
#pragma unroll
      for (int c = 0; c < NCH; ++c)
        if (xn[c]) mine = 128 * c + 4 * lane + __ffs(xn[c]) - 1;
      const unsigned bal = __ballot_sync(kFull, mine >= 0);
      code = __shfl_sync(kFull, mine, __ffs(bal) - 1);
    }
    if (lane == 0) hot[t] = (int16_t)code;
    __syncwarp();
  }
  return any_hit;
}

// Sweeps [sb, se) of replica r.  fresh: the state comes from a.init (or zero);
// else it is already in the bitsets (a later segment of the chain) and only
// the cache, the column sums, E and the violation count are rebuilt from it
// (exactly: E is a function of the state).  best and acc carry the running
// best energy and accept count in and out; `last` writes the outputs.
template <typename DT, int NCH, int K>
__device__ __forceinline__ void rows_replica_g(const StructArgs &a, int r, uint32_t *st, int16_t *hot, DT *ring,
                                               int lane, int sb, int se, bool fresh, bool last, long long &best,
                                               long long &acc, const RoundKeys &rk) {
  static_assert(K >= 3, "the ring holds rows t+2 .. t+K+1");
  const int C = a.C, Cp = a.Cp, s0 = a.start, A = a.A, B = a.B;
  const int twoA = 2 * A;
  const int Cw = (C + 31) >> 5;
  const int n = C * C;
  const uint32_t rg = (uint32_t)(a.rep_offset + r);
  const void *d = a.d;

  int tAc[NCH][4];
  int validc[NCH];
  long long E;
  int viol;
  rows_init<DT, NCH, 0, true>(a, r, st, hot, d, lane, tAc, validc, E, viol, !fresh);
  int tl = 0;  // tAc holds 2A c_i - tl (shifted by the sweep's table length)

  const int lev = a.level ? __ldg(a.level + r) : -1;
  bool settled = false;
  int settled_len = 0;
  for (int s = sb; s < se; ++s) {
    const int ts = lev >= 0 ? lev : s;
    const uint32_t *thr = a.thr + a.thr_off[ts];
    const int len = a.thr_len[ts];
    if (settled && len <= settled_len) continue;
    bool any_hit = false;
    const unsigned lenm1 = (unsigned)(len - 1);
    const float cT = a.thr_c[ts];
    const int dq = len > 1 ? min(len - 1, max(1, (int)fminf(8.0f / cT, 1.0e9f))) : 1;
    const uint32_t Q = len > 1 ? __ldg(a.thr + a.thr_off[ts] + dq) : 0u;
    if (len != tl) {  // tAc holds 2A c_i - len for this sweep's len
#pragma unroll
      for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) tAc[c][j] += tl - len;
      tl = len;
    }
    // X0..X3 hold the fields of rows t-1, t, t+1 and t+2 (the last read from
    // the ring) in roles that rotate by one per row
    int X0[NCH][4], X1[NCH][4], X2[NCH][4], X3[NCH][4];
    zero<NCH>(X0);
    add_drow<DT, NCH, 0>(d, Cp, C, s0, lane, 1, X0);  // row 0 holds only the start cell
    field_g<DT, NCH>(st, Cw, hot[1], 1, d, Cp, C, lane, X1);
    if (C > 2) field_g<DT, NCH>(st, Cw, hot[2], 2, d, Cp, C, lane, X2);
    else zero<NCH>(X2);
    // the ring holds rows t+2 .. t+K+1 while row t runs; rows 3 .. K+1 first
    for (int u = 3; u <= K + 1; ++u) {
      ring_issue<DT, NCH, K>(hot, ring, d, Cp, C, u, lane);
      cp_async_commit();
    }
    int t = 1;
    int hn = hot[1];
    const RowTest rtst{B, twoA, len, C, (unsigned)(2 * twoA - 2 * len)};
    int rt, xn[NCH];
    if (len <= twoA) {
      // A cold sweep: in a row whose cells form a permutation with the rest of
      // the state, adding a cell costs dE >= 2A >= len and removing its own
      // costs dE = 2A - P - N >= A, inside the band only when len comes within
      // P + N of 2A, so almost every row is cleared by the whole-row test and
      // changes nothing.  Four of them run with
      // the fields' roles rotated, (P, N, F_{t+2}) = (X0, X2, X3), (X1, X3,
      // X0), (X2, X0, X1), (X3, X1, X2), so no register moves; this loop
      // holds no flip path (which keeps its registers free), and the first
      // row that may flip rotates its fields into P = X0, Cu = X1, N = X2,
      // F_{t+2} = X3 and finishes the sweep in the loop below.
      while (true) {
        if (rows_g_front<DT, NCH, K>(st, hot, ring, d, Cp, C, Cw, lane, t, hn, X0, X2, X3, tAc, rtst, rt, xn))
          goto flip;
        if (++t >= C) goto sweep_done;
        hn = hot[t];
        if (rows_g_front<DT, NCH, K>(st, hot, ring, d, Cp, C, Cw, lane, t, hn, X1, X3, X0, tAc, rtst, rt, xn)) {
          rotate_fields<NCH>(X0, X1, X2, X3);
          goto flip;
        }
        if (++t >= C) goto sweep_done;
        hn = hot[t];
        if (rows_g_front<DT, NCH, K>(st, hot, ring, d, Cp, C, Cw, lane, t, hn, X2, X0, X1, tAc, rtst, rt, xn)) {
          swap_fields<NCH>(X0, X2);
          swap_fields<NCH>(X1, X3);
          goto flip;
        }
        if (++t >= C) goto sweep_done;
        hn = hot[t];
        if (rows_g_front<DT, NCH, K>(st, hot, ring, d, Cp, C, Cw, lane, t, hn, X3, X1, X2, tAc, rtst, rt, xn)) {
          rotate_fields<NCH>(X3, X2, X1, X0);
          goto flip;
        }
        if (++t >= C) goto sweep_done;
        hn = hot[t];
      }
    }
    // a hot sweep (most rows may flip): P = X0, Cu = X1, N = X2, F_{t+2} = X3
    while (true) {
      if (rows_g_front<DT, NCH, K>(st, hot, ring, d, Cp, C, Cw, lane, t, hn, X0, X2, X3, tAc, rtst, rt, xn)) {
      flip:
        any_hit |= rows_g_flip<DT, NCH>(a, st, hot, d, Cp, C, Cw, lane, t, s, hn, rt, xn, X0, X1, X2, tAc, validc,
                                        E, acc, viol, twoA, len, lenm1, cT, dq, Q, thr, rg, rk);
      }
#pragma unroll
      for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          X0[c][j] = X1[c][j];
          X1[c][j] = X2[c][j];
          X2[c][j] = X3[c][j];
        }
      if (++t >= C) break;
      hn = hot[t];
    }
  sweep_done:
    cp_async_wait<0>();  // the next sweep refills every slot
    __syncwarp();
    if (viol == 0 && E < best) best = E;
    settled = a.skip_settled && !any_hit;
    settled_len = len;
  }

  if (!last) return;
  uint8_t *out = a.states_out + (size_t)r * n;
  for (int e = lane; e < n; e += 32) {
    const int t = e / C, i = e - t * C;
    out[e] = (uint8_t)((__ldcg(st + (size_t)t * Cw + (i >> 5)) >> (i & 31)) & 1u);
  }
  if (lane == 0) {
    a.E_out[r] = E;
    if (a.best_out) a.best_out[r] = best;
    if (a.acc_out) a.acc_out[r] = acc;
  }
}

constexpr int kRowsGMaxWarps = 12;  // 384 threads: at most 170 registers per thread
constexpr int kRowsGRing = 8;

// Persistent over (replica, segment) units: the sweeps are cut into G
// segments and a warp takes units from one counter, segment-major, so the
// chains' last segments, not whole chains, make up the tail of the launch.
// The state between segments is the replica's bitsets (global memory) plus
// its running best energy and accept count (carry[2r], carry[2r+1]).  A
// segment g > 0 of replica r starts once progress[r] == g: a bounded wait on
// a flag another running warp sets (units are handed out in order, so the
// unit it waits for was taken earlier and is running or done); a wait that
// gives up marks the replica's energy INT64_MIN and sets *err.
constexpr long long kSegmentWaitCycles = 20000000000LL;  // ~10 s at 2 GHz (a unit takes under 1 s)

template <typename DT, int NCH>
__global__ void __launch_bounds__(kRowsGMaxWarps * 32)
    k_sweep_rows_g(const StructArgs a, const RoundKeys rk, int G, int *counter, int *progress, long long *carry,
                   int *err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t hot_bytes = align16r(2 * (size_t)a.C);
  const size_t per_warp = hot_bytes + (size_t)kRowsGRing * a.Cp * sizeof(DT);
  int16_t *hot = reinterpret_cast<int16_t *>(smem + warp * per_warp);
  DT *ring = reinterpret_cast<DT *>(smem + warp * per_warp + hot_bytes);
  const int total = a.R * G;
  const int nsw = a.sweep_end - a.sweep_begin;
  const int seg = (nsw + G - 1) / G;
  while (true) {
    int u = 0;
    if (lane == 0) u = atomicAdd(counter, 1);
    u = __shfl_sync(kFull, u, 0);
    if (u >= total) break;
    const int g = u / a.R, r = u - g * a.R;
    const int sb = a.sweep_begin + min(nsw, g * seg), se = a.sweep_begin + min(nsw, (g + 1) * seg);
    if (g > 0) {
      int ok = 1;
      if (lane == 0) {
        const long long t0 = clock64();
        while (true) {
          int v;
          asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(progress + r) : "memory");
          if (v >= g) break;
          if (clock64() - t0 > kSegmentWaitCycles) { ok = 0; break; }
          __nanosleep(256);
        }
      }
      ok = __shfl_sync(kFull, ok, 0);
      if (!ok) {
        if (lane == 0) {
          atomicExch(err, 1);
          a.E_out[r] = LLONG_MIN;
        }
        return;  // no copy is in flight between segments
      }
    }
    long long best = LLONG_MAX, acc = 0;
    if (g > 0) {
      best = __ldcg(carry + 2 * (size_t)r);
      acc = __ldcg(carry + 2 * (size_t)r + 1);
    }
    const bool last = g == G - 1;
    rows_replica_g<DT, NCH, kRowsGRing>(a, r, a.gstate + (size_t)r * a.nw_pad, hot, ring, lane, sb, se, g == 0, last,
                                        best, acc, rk);
    __syncwarp();
    if (!last && lane == 0) {
      carry[2 * (size_t)r] = best;
      carry[2 * (size_t)r + 1] = acc;
      __threadfence();  // the bitsets (atomics in L2), best and acc before the flag
      asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(progress + r), "r"(g + 1) : "memory");
    }
  }
}

// Widest rows (NCH = 4) keep three 16-register fields per lane: they get up to
// 255 registers by capping the CTA at 8 replicas.
template <int NCH>
constexpr int rows_max_warps() { return NCH >= 4 ? 8 : kMaxWarpsPerCta; }

template <typename DT, int NCH, int DMODE>
__global__ void __launch_bounds__(rows_max_warps<NCH>() * 32) k_sweep_rows(const StructArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int C = a.C, Cp = a.Cp;
  unsigned char *p = smem;
  const void *d = a.d;
  if (DMODE == 1) {
    const int nv = (int)((size_t)C * Cp * sizeof(DT) / 16);
    const int4 *src = static_cast<const int4 *>(a.d);
    int4 *dst = reinterpret_cast<int4 *>(p);
    for (int v = threadIdx.x; v < nv; v += blockDim.x) dst[v] = __ldg(src + v);
    d = p;
    p += align16r((size_t)C * Cp * sizeof(DT));
  } else if (DMODE == 2) {
    const DT *src = static_cast<const DT *>(a.d);
    int *dst = reinterpret_cast<int *>(p);
    for (int e = threadIdx.x; e < C * Cp; e += blockDim.x) dst[e] = (int)__ldg(src + e);
    d = p;
    p += align16r((size_t)C * Cp * 4);
  }
  const size_t per_warp = 4 * (size_t)a.nw_pad + align16r(2 * (size_t)C);
  uint32_t *st = reinterpret_cast<uint32_t *>(p + warp * per_warp);
  int16_t *hot1 = reinterpret_cast<int16_t *>(p + warp * per_warp + 4 * (size_t)a.nw_pad);
  __syncthreads();
  const int r = blockIdx.x * W + warp;
  if (r >= a.R) return;  // no CTA-wide barrier after this point
  rows_replica<DT, NCH, DMODE, DMODE == 0 ? 2 : 1>(a, r, st, hot1, d, lane);
}

// Batched persistent sweep: many fields of uneven size in one launch.  Each
// warp takes (field, replica) units from a global counter until none are left
// and runs the same chain as k_sweep_rows for that replica; units are ordered
// largest field first so the tail is made of short units.  Taking a unit is
// one atomicAdd: no warp ever waits on another.  The distance matrices are
// read from L2 (all fields of a batch together are a few MB).
template <int NCH>
__global__ void __launch_bounds__(rows_max_warps<NCH>() * 32)
    k_sweep_batch(const StructArgs *fields, const int2 *units, int n_units, int *counter, int nw_pad_max,
                  int Cmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t per_warp = 4 * (size_t)nw_pad_max + align16r(2 * (size_t)Cmax);
  uint32_t *st = reinterpret_cast<uint32_t *>(smem + warp * per_warp);
  int16_t *hot1 = reinterpret_cast<int16_t *>(smem + warp * per_warp + 4 * (size_t)nw_pad_max);
  while (true) {
    int u = 0;
    if (lane == 0) u = atomicAdd(counter, 1);
    u = __shfl_sync(kFull, u, 0);
    if (u >= n_units) break;
    const int2 unit = units[u];
    const StructArgs a = fields[unit.x];
    rows_replica<int16_t, NCH, 0, 1>(a, unit.y, st, hot1, a.d, lane);
    __syncwarp();
  }
}

constexpr size_t kSmemLimitRows = 227 * 1024;

// The batched launch with each field's distance matrix staged in shared
// memory: a CTA takes a unit of W replicas of one field (W = its warps), copies
// the field's int16 d into shared memory, runs one replica per warp against it
// and, once every warp is done, takes the next unit.  The autotuner times it
// against k_sweep_batch (d read from L2, units of one replica per warp).
template <int NCH>
__global__ void __launch_bounds__(rows_max_warps<NCH>() * 32)
    k_sweep_batch_staged(const StructArgs *fields, const int2 *units, int n_units, int *counter, int nw_pad_max,
                         int Cmax, int Cpmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_unit;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int16_t *dsm = reinterpret_cast<int16_t *>(smem);
  const size_t dbytes = align16r((size_t)Cmax * Cpmax * 2);
  const size_t per_warp = 4 * (size_t)nw_pad_max + align16r(2 * (size_t)Cmax);
  uint32_t *st = reinterpret_cast<uint32_t *>(smem + dbytes + warp * per_warp);
  int16_t *hot1 = reinterpret_cast<int16_t *>(smem + dbytes + warp * per_warp + 4 * (size_t)nw_pad_max);
  while (true) {
    if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
    __syncthreads();
    const int u = s_unit;
    if (u >= n_units) break;  // the same u in every thread
    const int2 unit = units[u];
    const StructArgs a = fields[unit.x];
    const int nv = (int)((size_t)a.C * a.Cp * 2 / 16);  // Cp is a multiple of 8
    const int4 *src = static_cast<const int4 *>(a.d);
    for (int v = threadIdx.x; v < nv; v += blockDim.x) reinterpret_cast<int4 *>(dsm)[v] = __ldg(src + v);
    __syncthreads();
    const int r = unit.y + warp;
    if (r < a.R) rows_replica<int16_t, NCH, 1, 1>(a, r, st, hot1, dsm, lane);
    __syncthreads();  // every warp is done with d and s_unit before the next unit
  }
}



template <typename DT, int NCH, int DMODE>
cudaError_t launch_r(const StructArgs &a, int W, size_t smem, cudaStream_t st) {
  auto k = k_sweep_rows<DT, NCH, DMODE>;
  std::lock_guard<std::mutex> lk(launch_mutex());
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<(a.R + W - 1) / W, W * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename DT, int NCH>
cudaError_t launch_r2(const StructArgs &a, int dmode, int W, size_t smem, cudaStream_t st) {
  if (dmode == 2) return launch_r<DT, NCH, 2>(a, W, smem, st);
  if (dmode == 1) return launch_r<DT, NCH, 1>(a, W, smem, st);
  return launch_r<DT, NCH, 0>(a, W, smem, st);
}

}  // namespace

size_t rows_state_words(int C) {
  const int Cw = (C + 31) / 32;
  return (size_t)(C * Cw + 3) / 4 * 4;
}

// Shared memory of the row kernel: d (mode 1: as stored, mode 2: widened to
// int32) + per replica its row bitsets and single-cell cache.
size_t rows_smem(int C, bool d_i16, int W, int dmode) {
  const int Cp = (C + 7) / 8 * 8;
  size_t dbytes = 0;
  if (dmode == 1) dbytes = align16r((size_t)C * Cp * (d_i16 ? 2 : 4));
  if (dmode == 2) dbytes = align16r((size_t)C * Cp * 4);
  return dbytes + (size_t)W * (4 * rows_state_words(C) + align16r(2 * (size_t)C));
}

bool rows_supported(int C, bool d_i16, int W) {
  const int wmax = C <= 256 ? kMaxWarpsPerCta : 8;
  return C <= 512 && W >= 1 && W <= wmax && rows_smem(C, d_i16, W, 0) <= kSmemLimitRows;
}

size_t batch_smem(int Cmax, int W) {
  return (size_t)W * (4 * rows_state_words(Cmax) + align16r(2 * (size_t)Cmax));
}

bool batch_supported(int Cmax, int W) {
  const int wmax = Cmax <= 256 ? kMaxWarpsPerCta : 8;
  return Cmax >= 2 && Cmax <= 512 && W >= 1 && W <= wmax && batch_smem(Cmax, W) <= kSmemLimitRows;
}

template <int NCH>
static cudaError_t prep_batch(int W, size_t smem, int *blocks_per_sm) {
  auto k = k_sweep_batch<NCH>;
  std::lock_guard<std::mutex> lk(launch_mutex());
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, W * 32, smem);
}

cudaError_t batch_prepare(int Cmax, int W, int *blocks_per_sm) {
  if (!batch_supported(Cmax, W)) return cudaErrorInvalidValue;
  const size_t smem = batch_smem(Cmax, W);
  if (Cmax <= 128) return prep_batch<1>(W, smem, blocks_per_sm);
  if (Cmax <= 256) return prep_batch<2>(W, smem, blocks_per_sm);
  return prep_batch<4>(W, smem, blocks_per_sm);
}

size_t batch_staged_smem(int Cmax, int W) {
  const int Cpmax = (Cmax + 7) / 8 * 8;
  return align16r((size_t)Cmax * Cpmax * 2) + batch_smem(Cmax, W);
}

bool batch_staged_supported(int Cmax, int W) {
  const int wmax = Cmax <= 256 ? kMaxWarpsPerCta : 8;
  return Cmax >= 2 && Cmax <= 512 && W >= 1 && W <= wmax && batch_staged_smem(Cmax, W) <= kSmemLimitRows;
}

template <int NCH>
static cudaError_t prep_batch_staged(int W, size_t smem, int *blocks_per_sm) {
  auto k = k_sweep_batch_staged<NCH>;
  std::lock_guard<std::mutex> lk(launch_mutex());
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, W * 32, smem);
}

cudaError_t batch_staged_prepare(int Cmax, int W, int *blocks_per_sm) {
  if (!batch_staged_supported(Cmax, W)) return cudaErrorInvalidValue;
  const size_t smem = batch_staged_smem(Cmax, W);
  if (Cmax <= 128) return prep_batch_staged<1>(W, smem, blocks_per_sm);
  if (Cmax <= 256) return prep_batch_staged<2>(W, smem, blocks_per_sm);
  return prep_batch_staged<4>(W, smem, blocks_per_sm);
}

cudaError_t launch_batch_staged(const StructArgs *fields, const int2 *units, int n_units, int *counter, int Cmax,
                                int W, int blocks, cudaStream_t st) {
  if (!batch_staged_supported(Cmax, W) || blocks < 1) return cudaErrorInvalidValue;
  const size_t smem = batch_staged_smem(Cmax, W);
  const int nwp = (int)rows_state_words(Cmax);
  const int Cpmax = (Cmax + 7) / 8 * 8;
  if (Cmax <= 128)
    k_sweep_batch_staged<1><<<blocks, W * 32, smem, st>>>(fields, units, n_units, counter, nwp, Cmax, Cpmax);
  else if (Cmax <= 256)
    k_sweep_batch_staged<2><<<blocks, W * 32, smem, st>>>(fields, units, n_units, counter, nwp, Cmax, Cpmax);
  else
    k_sweep_batch_staged<4><<<blocks, W * 32, smem, st>>>(fields, units, n_units, counter, nwp, Cmax, Cpmax);
  return cudaGetLastError();
}

cudaError_t launch_batch(const StructArgs *fields, const int2 *units, int n_units, int *counter, int Cmax,
                         int W, int blocks, cudaStream_t st) {
  if (!batch_supported(Cmax, W) || blocks < 1) return cudaErrorInvalidValue;
  const size_t smem = batch_smem(Cmax, W);
  const int nwp = (int)rows_state_words(Cmax);
  if (Cmax <= 128) k_sweep_batch<1><<<blocks, W * 32, smem, st>>>(fields, units, n_units, counter, nwp, Cmax);
  else if (Cmax <= 256) k_sweep_batch<2><<<blocks, W * 32, smem, st>>>(fields, units, n_units, counter, nwp, Cmax);
  else k_sweep_batch<4><<<blocks, W * 32, smem, st>>>(fields, units, n_units, counter, nwp, Cmax);
  return cudaGetLastError();
}

namespace {

int rows_dmode(int C, bool d_i16, int W) {
  if (rows_smem(C, d_i16, W, 2) <= kSmemLimitRows) return 2;
  if (rows_smem(C, d_i16, W, 1) <= kSmemLimitRows) return 1;
  return 0;
}

template <typename DT, int NCH, int DMODE>
cudaError_t occ_r(int W, size_t smem, int *blocks) {
  auto k = k_sweep_rows<DT, NCH, DMODE>;
  std::lock_guard<std::mutex> lk(launch_mutex());
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, W * 32, smem);
}

template <typename DT, int NCH>
cudaError_t occ_r2(int dmode, int W, size_t smem, int *blocks) {
  if (dmode == 2) return occ_r<DT, NCH, 2>(W, smem, blocks);
  if (dmode == 1) return occ_r<DT, NCH, 1>(W, smem, blocks);
  return occ_r<DT, NCH, 0>(W, smem, blocks);
}

// CTAs of W replicas that fit on one SM at once (0 when none or on error).
int rows_blocks_per_sm(int C, bool d_i16, int W) {
  const int dmode = rows_dmode(C, d_i16, W);
  const size_t smem = rows_smem(C, d_i16, W, dmode);
  const int NCH = C <= 128 ? 1 : (C <= 256 ? 2 : 4);
  int b = 0;
  cudaError_t e;
  if (d_i16) e = NCH == 1 ? occ_r2<int16_t, 1>(dmode, W, smem, &b)
                          : (NCH == 2 ? occ_r2<int16_t, 2>(dmode, W, smem, &b) : occ_r2<int16_t, 4>(dmode, W, smem, &b));
  else e = NCH == 1 ? occ_r2<int32_t, 1>(dmode, W, smem, &b)
                    : (NCH == 2 ? occ_r2<int32_t, 2>(dmode, W, smem, &b) : occ_r2<int32_t, 4>(dmode, W, smem, &b));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return b;
}

}  // namespace

// ---- the global-spins row kernel (fields of 257..512 cells)
size_t rows_g_words(int C) {
  const int Cw = (C + 31) / 32;
  return (size_t)(C * Cw + 3) / 4 * 4;
}

size_t rows_g_smem(int C, bool d_i16, int W) {
  const int Cp = (C + 7) / 8 * 8;
  return (size_t)W * (align16r(2 * (size_t)C) + (size_t)kRowsGRing * Cp * (d_i16 ? 2 : 4));
}

bool rows_g_supported(int C, bool d_i16, int W) {
  return C > 256 && C <= 512 && W >= 1 && W <= kRowsGMaxWarps && rows_g_smem(C, d_i16, W) <= kSmemLimitRows;
}

namespace {

template <typename DT>
cudaError_t occ_g(int W, size_t smem, int *blocks) {
  auto k = k_sweep_rows_g<DT, 4>;
  std::lock_guard<std::mutex> lk(launch_mutex());
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, W * 32, smem);
}

}  // namespace

int rows_g_auto_warps(int C, bool d_i16, int R) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 4;
  }
  static std::mutex mu;
  static std::map<std::tuple<int, int, bool, int>, int> memo;
  const auto key = std::make_tuple(dev, C, d_i16, R);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
  }
  // the most replicas resident at once; among equals the larger CTA
  int best_w = 1;
  long long best = -1;
  for (int W = 1; W <= kRowsGMaxWarps; ++W) {
    if (!rows_g_supported(C, d_i16, W)) continue;
    int b = 0;
    const cudaError_t e = d_i16 ? occ_g<int16_t>(W, rows_g_smem(C, d_i16, W), &b)
                                : occ_g<int32_t>(W, rows_g_smem(C, d_i16, W), &b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    const long long resident = std::min<long long>(R, (long long)sms * b * W);
    if (resident >= best) {
      best = resident;
      best_w = W;
    }
  }
  std::lock_guard<std::mutex> lk(mu);
  memo[key] = best_w;
  return best_w;
}

cudaError_t launch_rows_g(const StructArgs &a_in, bool d_i16, int W, int *counter, int *progress, long long *carry,
                          int *err, cudaStream_t st, LaunchInfo *info) {
  StructArgs a = a_in;
  if (!rows_g_supported(a.C, d_i16, W) || a.gstate == nullptr || !counter || !progress || !carry || !err)
    return cudaErrorInvalidValue;
  a.nw_pad = (int32_t)rows_g_words(a.C);
  const size_t smem = rows_g_smem(a.C, d_i16, W);
  int dev = 0, sms = 0, bps = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = d_i16 ? occ_g<int16_t>(W, smem, &bps) : occ_g<int32_t>(W, smem, &bps);
  if (e != cudaSuccess) return e;
  if (bps < 1) return cudaErrorInvalidConfiguration;
  // more chains than fit at once: cut the sweeps into segments of ~500 so the
  // launch ends on short units instead of a partial wave of whole chains
  const long long capacity = (long long)bps * sms * W;
  const int nsw = a.sweep_end - a.sweep_begin;
  const int G = (a.R > capacity && nsw >= 1000) ? std::min(64, nsw / 500) : 1;
  const long long warps_needed = (long long)a.R * G;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((long long)bps * sms, (warps_needed + W - 1) / W));
  if (info) {
    info->warps_per_cta = W;
    info->blocks = blocks;
    info->smem = smem;
    info->variant = G > 1 ? "rows,spins:global,d:L2 ring,segments" : "rows,spins:global,d:L2 ring";
  }
  // the ten rounds' Philox keys, launch constants
  RoundKeys rk;
  for (int i = 0; i < 10; ++i) {
    rk.k[2 * i] = a.key0 + (uint32_t)i * 0x9E3779B9u;
    rk.k[2 * i + 1] = a.key1 + (uint32_t)i * 0xBB67AE85u;
  }
  std::lock_guard<std::mutex> lk(launch_mutex());
  if (d_i16) {
    auto k = k_sweep_rows_g<int16_t, 4>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k<<<blocks, W * 32, smem, st>>>(a, rk, G, counter, progress, carry, err);
  } else {
    auto k = k_sweep_rows_g<int32_t, 4>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k<<<blocks, W * 32, smem, st>>>(a, rk, G, counter, progress, carry, err);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

int rows_auto_warps(int C, bool d_i16, int R) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 4;
  }
  static std::mutex mu;
  static std::map<std::tuple<int, int, bool, int>, int> memo;
  const auto key = std::make_tuple(dev, C, d_i16, R);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
  }
  // the most replicas resident at once (a sequential chain per warp: the
  // kernel is latency-bound, so resident chains are its throughput); among
  // equals the default of 4 replicas per CTA, then the smaller CTA
  int best_w = 4;
  long long best = -1;
  for (int W = 1; W <= kMaxWarpsPerCta; ++W) {
    if (!rows_supported(C, d_i16, W)) continue;
    const long long resident = std::min<long long>(R, (long long)sms * rows_blocks_per_sm(C, d_i16, W) * W);
    if (resident > best || (resident == best && W == 4)) {
      best = resident;
      best_w = W;
    }
  }
  if (!rows_supported(C, d_i16, best_w)) best_w = 1;
  std::lock_guard<std::mutex> lk(mu);
  memo[key] = best_w;
  return best_w;
}

cudaError_t launch_rows(const StructArgs &a_in, bool d_i16, int W, cudaStream_t st, LaunchInfo *info) {
  StructArgs a = a_in;
  a.nw_pad = (int32_t)rows_state_words(a.C);
  if (!rows_supported(a.C, d_i16, W)) return cudaErrorInvalidValue;
  const int dmode = rows_dmode(a.C, d_i16, W);
  const size_t smem = rows_smem(a.C, d_i16, W, dmode);
  if (smem > kSmemLimitRows) return cudaErrorInvalidValue;
  const int NCH = a.C <= 128 ? 1 : (a.C <= 256 ? 2 : 4);
  if (info) {
    info->warps_per_cta = W;
    info->blocks = (a.R + W - 1) / W;
    info->smem = smem;
    info->variant = dmode == 2 ? "rows,d:smem32" : (dmode == 1 ? "rows,d:smem" : "rows,d:global");
  }
  if (d_i16) {
    if (NCH == 1) return launch_r2<int16_t, 1>(a, dmode, W, smem, st);
    if (NCH == 2) return launch_r2<int16_t, 2>(a, dmode, W, smem, st);
    return launch_r2<int16_t, 4>(a, dmode, W, smem, st);
  }
  if (NCH == 1) return launch_r2<int32_t, 1>(a, dmode, W, smem, st);
  if (NCH == 2) return launch_r2<int32_t, 2>(a, dmode, W, smem, st);
  return launch_r2<int32_t, 4>(a, dmode, W, smem, st);
}

}  // namespace qp

namespace qp {
namespace chk {
QP_CHECK_ACCESSOR(rows)
}  // namespace chk
}  // namespace qp
