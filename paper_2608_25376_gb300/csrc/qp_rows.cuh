// Device helpers of the row-parallel structured sweep (qp_sweep_rows.cu:
// the single-field and the batched persistent kernels): distance-row loads,
// row fields, the single-cell cache and the evaluation of one row chunk.
// Included inside namespace qp::{anon}.
#pragma once

__host__ __device__ constexpr size_t align16r(size_t x) { return (x + 15) & ~size_t(15); }

// d modes: 0 = global memory (DT), 1 = shared memory (DT), 2 = shared memory widened to int32
template <typename DT, int DMODE>
__device__ __forceinline__ void drow4(const void *d, int Cp, int C, int h, int i, bool ok, int (&v)[4]) {
  v[0] = v[1] = v[2] = v[3] = 0;
  if (!ok) return;
  h = QP_IX(h, C, 2);  // the four entries i..i+3 < Cp of row h
  i = QP_IX(i, Cp - 3, 2);
  if (DMODE == 2) {
    const int4 q = *reinterpret_cast<const int4 *>(static_cast<const int *>(d) + (size_t)h * Cp + i);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if (sizeof(DT) == 2) {
    const uint2 *p = reinterpret_cast<const uint2 *>(static_cast<const DT *>(d) + (size_t)h * Cp + i);
    const uint2 q = DMODE == 1 ? *p : __ldg(p);
    v[0] = (int)(short)(q.x & 0xFFFFu);
    v[1] = (int)q.x >> 16;
    v[2] = (int)(short)(q.y & 0xFFFFu);
    v[3] = (int)q.y >> 16;
  } else {
    const int4 *p = reinterpret_cast<const int4 *>(static_cast<const DT *>(d) + (size_t)h * Cp + i);
    const int4 q = DMODE == 1 ? *p : __ldg(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
}

template <typename DT, int NCH, int DMODE>
__device__ __forceinline__ void add_drow(const void *d, int Cp, int C, int h, int lane, int dlt,
                                         int (&F)[NCH][4]) {
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int i = 128 * c + 4 * lane;
    int v[4];
    drow4<DT, DMODE>(d, Cp, C, h, i, i < C, v);
#pragma unroll
    for (int j = 0; j < 4; ++j) F[c][j] += dlt * v[j];
  }
}

template <typename DT, int NCH, int DMODE>
__device__ __forceinline__ void set_drow(const void *d, int Cp, int C, int h, int lane, int (&F)[NCH][4]) {
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int i = 128 * c + 4 * lane;
    drow4<DT, DMODE>(d, Cp, C, h, i, i < C, F[c]);
  }
}

// A word of a replica's spins: from shared memory, or, with SG (spins in
// global memory, flipped by atomics in L2), from L2 past the L1 cache, which
// could still hold the line as it was before the flip.
template <bool SG>
__device__ __forceinline__ uint32_t spin_word(const uint32_t *p) {
  if (SG) return __ldcg(p);
  return *p;
}

// F += sum over the set bits h of one row of d[h][.]; returns the number of bits
// and, in *one, the cell when there is exactly one (else -1).
template <typename DT, int NCH, int DMODE, bool SG = false>
__device__ __forceinline__ int scan_row_field(const uint32_t *row, int Cw, const void *d, int Cp, int C,
                                              int lane, int (&F)[NCH][4], int *one) {
  const uint32_t word = lane < Cw ? spin_word<SG>(row + lane) : 0u;
  const int cnt = __reduce_add_sync(kFull, __popc(word));
  uint32_t bal = __ballot_sync(kFull, word != 0u);
  int last = -1;
  while (bal) {
    const int w = __ffs(bal) - 1;
    bal &= bal - 1;
    uint32_t wd = __shfl_sync(kFull, word, w);
    while (wd) {
      const int h = (w << 5) + __ffs(wd) - 1;
      wd &= wd - 1;
      last = h;
      add_drow<DT, NCH, DMODE>(d, Cp, C, h, lane, 1, F);
    }
  }
  *one = cnt == 1 ? last : -1;
  return cnt;
}

// F_u, the field of row u: the d row of its single hot cell (the per-row cache
// hot1) or, when the row does not hold exactly one cell, a scan of its bits.
// F must be zero on entry.
template <typename DT, int NCH, int DMODE>
__device__ __forceinline__ void row_field(const uint32_t *st, int Cw, const int16_t *hot1, int u, const void *d,
                                          int Cp, int C, int lane, int (&F)[NCH][4]) {
  const int h = hot1[u];
  if (h >= 0) add_drow<DT, NCH, DMODE>(d, Cp, C, h, lane, 1, F);
  else { int one; scan_row_field<DT, NCH, DMODE>(st + u * Cw, Cw, d, Cp, C, lane, F, &one); }
}

// The single hot cell of a row, or -1 if the row does not hold exactly one.
template <bool SG = false>
__device__ __forceinline__ int row_single(const uint32_t *row, int Cw, int lane) {
  const uint32_t word = lane < Cw ? spin_word<SG>(row + lane) : 0u;
  const int cnt = __reduce_add_sync(kFull, __popc(word));
  if (cnt != 1) return -1;
  const uint32_t bal = __ballot_sync(kFull, word != 0u);
  const int w = __ffs(bal) - 1;
  const uint32_t wd = __shfl_sync(kFull, word, w);
  return (w << 5) + __ffs(wd) - 1;
}

template <int NCH>
__device__ __forceinline__ void zero(int (&F)[NCH][4]) {
#pragma unroll
  for (int c = 0; c < NCH; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) F[c][j] = 0;
}

__device__ __forceinline__ int sel4(const int (&v)[4], int j) {
  return j == 0 ? v[0] : (j == 1 ? v[1] : (j == 2 ? v[2] : v[3]));
}

// The whole row as one test.  With base = B f + 2A c_i, a proposal can matter
// (dE < len) only if base < lo = len - 2A(r-1) (x = 0) or base > hi =
// 2A(3-r) - len (x = 1); the lane's columns outside [lo, hi] are a superset
// of its proposals that matter (columns outside the field carry base = 2A,
// inside [lo, hi] when r = 1 and len < 2A).  The range test is one unsigned
// compare, exact because base >= 0 and lo < 2^31 (so base - lo never wraps
// into [0, hi - lo]); an empty range (hi < lo) passes every column.
template <int NCH>
__device__ __forceinline__ bool row_pretest(const int (&P)[NCH][4], const int (&N)[NCH][4], const int (&tAc)[NCH][4],
                                            int B, int twoA, int rt, int len, int C) {
  const int lo = len - twoA * (rt - 1), hi = twoA * (3 - rt) - len;
  if (hi < lo) return true;
  const unsigned W = (unsigned)(hi - lo), ulo = (unsigned)lo;
  bool maybe = false;
  if (B == 1) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      if (128 * c >= C) break;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        maybe |= (unsigned)P[c][j] + (unsigned)N[c][j] + (unsigned)tAc[c][j] - ulo > W;
    }
  } else {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      if (128 * c >= C) break;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        maybe |= (unsigned)B * ((unsigned)P[c][j] + (unsigned)N[c][j]) + (unsigned)tAc[c][j] - ulo > W;
    }
  }
  return maybe;
}

// row_pretest with the column term kept shifted, tAc = 2A c_i - len: base -
// lo = B f + tAc + 2A(r-1), one add fewer per column when r = 1 (the common
// case: a row that holds exactly one cell).  Same result as row_pretest.
// W1 = hi - lo for r = 1, i.e. 4A - 2 len (fixed through a sweep; used when
// len <= 2A, else every column passes).
template <int NCH>
__device__ __forceinline__ bool row_pretest_shifted(const int (&P)[NCH][4], const int (&N)[NCH][4],
                                                    const int (&tAc)[NCH][4], int B, int twoA, int rt, int len,
                                                    unsigned W1) {
  bool maybe = false;
  if (B == 1 && rt == 1) {
    if (len > twoA) return true;
#pragma unroll
    for (int c = 0; c < NCH; ++c)
#pragma unroll
      for (int j = 0; j < 4; ++j) maybe |= (unsigned)P[c][j] + (unsigned)N[c][j] + (unsigned)tAc[c][j] > W1;
  } else {
    const int lo = len - twoA * (rt - 1), hi = twoA * (3 - rt) - len;
    if (hi < lo) return true;
    const unsigned W = (unsigned)(hi - lo);
    const unsigned adj = (unsigned)(twoA * (rt - 1));
#pragma unroll
    for (int c = 0; c < NCH; ++c)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        maybe |= (unsigned)B * ((unsigned)P[c][j] + (unsigned)N[c][j]) + (unsigned)tAc[c][j] + adj > W;
  }
  return maybe;
}

// The proposals of one 128-wide row chunk when at least one of them can be
// accepted or needs a draw: evaluate against the current row sum, take the
// first accepted one, apply it, resume after it.  Returns whether any flip was
// applied.  SG: the row's bits are in global memory (flipped by a fire-and-
// forget atomic XOR, so the warp never waits on the write).
template <typename DT, int NCH, int DMODE, bool SG = false, typename KEY = PhiloxKey>
__device__ __forceinline__ bool row_chunk(int c, int t, int s, int tC, const int (&base)[4], const int (&de0)[4],
                                       int &xnc, int validc,
                                       int (&tAc)[4], int &rt, int (&Cu)[NCH][4], uint32_t *row, long long &E,
                                       long long &acc, int &viol, const void *d, int Cp, int C, int lane, int twoA,
                                       int len, unsigned lenm1, float cT, int dq, uint32_t Q, const uint32_t *thr,
                                       uint32_t rg, const KEY &key, int tshift = 0) {
  const int ib = 128 * c + 4 * lane;
  const int delta = tC & 3;
  int cand = validc;
  bool h0 = false, h1 = false, flipped = false;
  uint4 u0 = make_uint4(0, 0, 0, 0), u1 = make_uint4(0, 0, 0, 0);
  int dE[4] = {de0[0], de0[1], de0[2], de0[3]};  // for the row sum on entry
  while (true) {
    int accm = 0, need = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned dm1 = (unsigned)(dE[j] - 1);
      accm |= (int)(dm1 >> 31) << j;   // dE <= 0
      need |= (int)(dm1 < lenm1) << j;  // 1 <= dE < len
    }
    accm &= cand;
    need &= cand;
    if (__ballot_sync(kFull, need)) {
      // lane L's proposals lie in counter blocks b0 and (when delta != 0) b0 + 1,
      // which is lane L+1's b0: every lane computes its own block once and
      // takes the next one from its right neighbour; lane 31 computes its
      // second block itself when it needs it.
      const int m0 = (1 << (4 - delta)) - 1;
      const uint32_t b0 = (uint32_t)((tC + ib) >> 2);
      if (!h0) {
        u0 = philox4x32_10(make_uint4(b0, (uint32_t)s, rg, kRngTag), key);
        u1.x = __shfl_down_sync(kFull, u0.x, 1);
        u1.y = __shfl_down_sync(kFull, u0.y, 1);
        u1.z = __shfl_down_sync(kFull, u0.z, 1);
        u1.w = __shfl_down_sync(kFull, u0.w, 1);
        h0 = true;
      }
      if (lane == 31 && (need & ~m0) && !h1) {
        u1 = philox4x32_10(make_uint4(b0 + 1, (uint32_t)s, rg, kRngTag), key);
        h1 = true;
      }
      // the lane's four draws: words delta..delta+3 of the blocks (u0, u1); delta
      // is the same for the whole row, so the branch is uniform
      uint32_t uw[4];
      switch (delta) {
        case 0: uw[0] = u0.x; uw[1] = u0.y; uw[2] = u0.z; uw[3] = u0.w; break;
        case 1: uw[0] = u0.y; uw[1] = u0.z; uw[2] = u0.w; uw[3] = u1.x; break;
        case 2: uw[0] = u0.z; uw[1] = u0.w; uw[2] = u1.x; uw[3] = u1.y; break;
        default: uw[0] = u0.w; uw[1] = u1.x; uw[2] = u1.y; uw[3] = u1.z; break;
      }
      // dE >= dq gives thr[dE] <= thr[dq] = Q, so u >= Q rejects outright: the
      // proposals still open after that test (branch-free), then their exact
      // tests, which few proposals reach
      int open = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) open |= (int)((dE[j] < dq) | (uw[j] < Q)) << j;
      open &= need;
      if (open) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (((open >> j) & 1) && accept_draw(uw[j], dE[j], cT, thr, len)) accm |= 1 << j;
      }
    }
    const uint32_t bal = __ballot_sync(kFull, accm);
    if (bal == 0) break;
    const int L = __ffs(bal) - 1;
    const int jl = accm ? __ffs(accm) - 1 : 0;
    const int xl = (xnc >> jl) & 1;
    const int tc = sel4(tAc, jl) + tshift;  // 2A c_i
    const int pk0 = jl | (xl << 2) | ((tc == twoA) << 3) | ((tc + (1 - 2 * xl) * twoA == twoA) << 4);
    const int de = __shfl_sync(kFull, sel4(dE, jl), L);
    const int pk = __shfl_sync(kFull, pk0, L);
    const int jj = pk & 3, dlt = 1 - 2 * ((pk >> 2) & 1);
    E += de;
    ++acc;
    rt += dlt;
    viol += ((pk >> 4) & 1 ? 0 : 1) - ((pk >> 3) & 1 ? 0 : 1);
    flipped = true;
    if (lane == L) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j == jj) tAc[j] += dlt * twoA;
      xnc ^= 1 << jj;
      const int wi = QP_IX(4 * c + (L >> 3), (C + 31) >> 5, 3);
      if (SG) atomicXor(row + wi, 1u << (4 * (L & 7) + jj));
      else row[wi] ^= 1u << (4 * (L & 7) + jj);
    }
    add_drow<DT, NCH, DMODE>(d, Cp, C, 128 * c + 4 * L + jj, lane, dlt, Cu);
    cand &= lane < L ? 0 : (lane > L ? 0xF : (0xF << (jj + 1)) & 0xF);
    __syncwarp();
    // the row sum moved: every later dE of the row moves with it
    const int k0 = twoA * (rt - 1), k1 = twoA * (3 - rt);
#pragma unroll
    for (int j = 0; j < 4; ++j) dE[j] = ((xnc >> j) & 1) ? k1 - base[j] : base[j] + k0;
  }
  return flipped;
}


// The initial state of replica r (given or all zero, with row 0 and column s
// clamped: x_{0,s} = 1), its single-cell cache (the cell when a row holds
// exactly one, -1 when it holds none, -2 when it holds several), 2A x column
// sums, the mask of proposable columns, its energy by Eqs. 3-6 and its
// violation count.
// keep_bits: the bitsets already hold the state (a later segment of the
// same chain): only the derived quantities are rebuilt from them.
template <typename DT, int NCH, int DMODE, bool SG = false>
__device__ __forceinline__ void rows_init(const StructArgs &a, int r, uint32_t *st, int16_t *hot1, const void *d,
                                          int lane, int (&tAc)[NCH][4], int (&validc)[NCH], long long &E_out,
                                          int &viol_out, bool keep_bits = false) {
  const int C = a.C, Cp = a.Cp, s0 = a.start, A = a.A, B = a.B;
  const int twoA = 2 * A;
  const int Cw = (C + 31) >> 5;
  const int n = C * C;
  // ---- initial state: given or all zero; row 0 and column s clamped (x_{0,s} = 1)
  const uint8_t *init = a.init ? a.init + (size_t)r * n : nullptr;
  for (int e = keep_bits ? C * Cw : lane; e < C * Cw; e += 32) {
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

  // ---- column sums, per-row single cells, penalties and H_dist (Eqs. 3-6)
  int cs[NCH][4];
  zero<NCH>(cs);
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    validc[c] = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = 128 * c + 4 * lane + j;
      if (i < C && i != s0) validc[c] |= 1 << j;
    }
  }
  long long hd = 0, pen_rows = 0;
  int viol = 0;
  {
    int Fn[NCH][4];
    for (int t = 0; t < C; ++t) {
      const uint32_t *row = st + t * Cw;
      int rsum = 0, xb[NCH];
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const int ib = 128 * c + 4 * lane;
        xb[c] = ib < C ? (int)((spin_word<SG>(row + 4 * c + (lane >> 3)) >> (4 * (lane & 7))) & 0xFu) : 0;
        rsum += __popc(xb[c]);
#pragma unroll
        for (int j = 0; j < 4; ++j) cs[c][j] += (xb[c] >> j) & 1;
      }
      rsum = __reduce_add_sync(kFull, rsum);
      pen_rows += (long long)(1 - rsum) * (1 - rsum);
      viol += rsum != 1;
      const int h1 = row_single<SG>(row, Cw, lane);
      if (lane == 0) hot1[t] = (int16_t)(rsum == 1 ? h1 : (rsum == 0 ? -1 : -2));
      if (t + 1 < C) {
        zero<NCH>(Fn);
        int one;
        scan_row_field<DT, NCH, DMODE, SG>(st + (t + 1) * Cw, Cw, d, Cp, C, lane, Fn, &one);
#pragma unroll
        for (int c = 0; c < NCH; ++c)
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if ((xb[c] >> j) & 1) hd += Fn[c][j];
      }
    }
  }
  __syncwarp();
  long long pen_cols = 0;
  int viol_cols = 0;
#pragma unroll
  for (int c = 0; c < NCH; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (128 * c + 4 * lane + j < C) {
        pen_cols += (long long)(1 - cs[c][j]) * (1 - cs[c][j]);
        viol_cols += cs[c][j] != 1;
      }
  E_out = (long long)B * warp_sum64(hd) + (long long)A * (pen_rows + warp_sum64(pen_cols));
  viol_out = viol + __reduce_add_sync(kFull, viol_cols);
  // columns outside the field get 2A (as if visited once): the row kernel's
  // whole-row pre-test then never passes on them in a one-hot row
#pragma unroll
  for (int c = 0; c < NCH; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) tAc[c][j] = 128 * c + 4 * lane + j < C ? twoA * cs[c][j] : twoA;

}
