// Kernels of the learned warm start: a per-cell bf16 MLP (features -> 3 x
// Linear(256)+ReLU -> Linear(256) step logits), trained with softmax
// cross-entropy on the annealer's own best paths.
//
// The forward pass of all four layers runs as one kernel (k_mlp_forward, the
// activations of a 128-cell tile kept in shared memory between layers).
// Every other matrix product (dX = dY W, dW = dY^T X, and the forward as four
// separate launches when asked) runs on one tcgen05
// kernel: D[M x N] (+)= A[M x K] B[N x K]^T with bf16 operands (both K-major,
// i.e. K contiguous) and fp32 accumulation in tensor memory.  A CTA owns a
// 128 x N tile (N <= 256, multiple of 16) and walks K in chunks of 64 through
// two shared-memory stages: one thread has the tensor-memory-access engine
// load each operand chunk (one 2-D tile copy per operand, 128-byte swizzle,
// zeros outside the matrix) with its byte count on the stage's "full"
// mbarrier, issues the 128 x N x 16 MMAs of the chunk once it has landed and
// commits them to the stage's "done" mbarrier, which frees the stage for the
// chunk after next; the load of chunk c+1 overlaps the MMAs of chunk c.
// Every wait is bounded.  The epilogue reads the accumulator back with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = rows of the tile), applies
// bias/ReLU/masking and stages the rows in the freed stages, so that the
// stores (and the ReLU reference loads) cover whole sectors.  Split-K partial
// tiles are added into an fp32 output with atomics.
#include <cuda.h>  // CUtensorMap and the tile-encoder types; the encoder comes from the runtime
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "qp_mlp.h"

namespace qp {
namespace mlp {
namespace {

constexpr int kTileM = 128;
constexpr int kChunkK = 64;
constexpr int kTmemCols = 256;
constexpr size_t kSmemA = kTileM * kChunkK * 2;  // 16 KB per stage
constexpr size_t kSmemB = 256 * kChunkK * 2;     // 32 KB per stage
constexpr int kStages = 2;
// Two stages (96 KB) plus 1 KB to align them to the 1024-byte swizzle
// pattern; 100 KB keeps at most two CTAs (2 x 256 TMEM columns = all 512) on
// an SM, so tcgen05.alloc never has to wait long.
constexpr size_t kGemmSmem = 100 * 1024;
static_assert(kStages * (kSmemA + kSmemB) + 1024 <= kGemmSmem, "GEMM stages exceed the shared-memory budget");
constexpr long long kWaitCycles = 1000000000LL;  // ~0.5 s at 2 GHz, then give up
// Epilogue staging: per warp 32 rows of 64 fp32 plus 16 bytes against bank conflicts.
constexpr int kEpiRowFloats = 64 + 4;
constexpr int kEpiRowBytes = kEpiRowFloats * 4;
static_assert(4 * 32 * kEpiRowBytes <= kStages * (kSmemA + kSmemB), "epilogue staging exceeds the stages");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05) of a K-major operand tile that
// the tile copy wrote with 128-byte swizzle: row r is 128 bytes (64 bf16 along
// K) at r * 128 with its 16-byte pieces permuted within each 8-row, 1024-byte
// group.  Start address >> 4 in bits 0-13, leading-dimension offset field 1
// (not used by swizzled K-major tiles), stride-dimension offset 1024 >> 4 (one
// 8-row group) in 32-45, descriptor version 1 in 46-47, base offset 0 (tiles
// are 1024-byte aligned), layout type 2 = 128-byte swizzle in bits 61-63.  The
// k-th 16-element step of a chunk starts 32k bytes into the tile.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// 2-D tile copy global -> shared of box (x, y) = (k0, row0) of `map`, its bytes
// counted on `mbar`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Instruction descriptor of kind::f16: fp32 D (bits 4-5 = 1), bf16 A and B
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of an mbarrier, giving up after kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(mbar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(128)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs g) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[kStages], done[kStages];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail_flag;
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTileM;
  const int N = g.N;
  const int kbeg = blockIdx.z * g.k_per_split;
  const int kend = min(g.K, kbeg + g.k_per_split);
  const int nchunks = kend > kbeg ? (kend - kbeg + kChunkK - 1) / kChunkK : 0;

  if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), kTmemCols);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&done[s]), 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    fail_flag = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int issued = nchunks;
  if (tid == 0 && nchunks > 0) {
    const uint32_t idesc = idesc_bf16(kTileM, N);
    const uint32_t bytes = (uint32_t)(kSmemA + (size_t)N * kChunkK * 2);  // both boxes, zeros included
    uint32_t sa[kStages], sb[kStages];
    for (int s = 0; s < kStages; ++s) {
      sa[s] = smem_u32(smem + s * kSmemA);
      sb[s] = smem_u32(smem + kStages * kSmemA + s * kSmemB);
    }
    // completions issued and seen per barrier; the k-th completion has parity k & 1
    int full_issued[kStages] = {0, 0}, full_seen[kStages] = {0, 0};
    int done_issued[kStages] = {0, 0}, done_seen[kStages] = {0, 0};
    bool ok = true;
    auto load = [&](int c) {
      const int s = c & 1;
      mbar_expect_tx(smem_u32(&full[s]), bytes);
      tma_load_2d(sa[s], &tmA, kbeg + c * kChunkK, m0, smem_u32(&full[s]));
      tma_load_2d(sb[s], &tmB, kbeg + c * kChunkK, 0, smem_u32(&full[s]));
      ++full_issued[s];
    };
    load(0);
    for (int c = 0; c < nchunks && ok; ++c) {
      const int s = c & 1;
      if (c + 1 < nchunks) {
        const int s1 = (c + 1) & 1;
        if (done_seen[s1] < done_issued[s1]) {  // the MMAs of chunk c-1 still read stage s1
          ok = mbar_wait(smem_u32(&done[s1]), done_seen[s1] & 1);
          if (!ok) break;
          ++done_seen[s1];
        }
        load(c + 1);
      }
      ok = mbar_wait(smem_u32(&full[s]), full_seen[s] & 1);
      if (!ok) break;
      ++full_seen[s];
      tc_fence_after();
      const int k0 = kbeg + c * kChunkK;
      const int ksteps = min(4, (kend - k0 + 15) / 16);
      for (int kk = 0; kk < ksteps; ++kk) {
        const uint64_t ad = smem_desc_sw128(sa[s] + kk * 32);
        const uint64_t bd = smem_desc_sw128(sb[s] + kk * 32);
        mma_bf16(tmem, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(smem_u32(&done[s]));
      ++done_issued[s];
    }
    // the accumulator is complete once every commit has landed; after a
    // failed wait, let whatever is still in flight land (bounded) before the
    // CTA frees its shared and tensor memory
    for (int s = 0; s < kStages; ++s) {
      while (done_seen[s] < done_issued[s]) {
        if (!mbar_wait(smem_u32(&done[s]), done_seen[s] & 1)) { ok = false; break; }
        ++done_seen[s];
      }
      while (full_seen[s] < full_issued[s]) {
        if (!mbar_wait(smem_u32(&full[s]), full_seen[s] & 1)) { ok = false; break; }
        ++full_seen[s];
      }
    }
    if (!ok) fail_flag = 1;
  }
  __syncthreads();
  tc_fence_after();
  if (!fail_flag && issued > 0) {
    // The stages are free now (every copy landed, every MMA complete): each
    // warp stages its 32 accumulator rows, 64 columns at a time, in shared
    // memory, then writes them out two rows per instruction so that every
    // global access covers whole sectors.
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    float *stg = reinterpret_cast<float *>(smem + (size_t)warp * 32 * kEpiRowBytes);
    const int row0 = m0 + warp * 32;
    const bool bias = g.bias && (g.mode == kEpiBiasRelu || g.mode == kEpiBiasF32);
    for (int c0 = 0; c0 < N; c0 += 64) {
      const int nb = min(64, N - c0);  // a multiple of 16
      for (int cc = 0; cc < nb; cc += 16) {
        float v[16];
        tmem_ld16(lane_base + c0 + cc, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float x = v[i] + (bias ? g.bias[c0 + cc + i] : 0.0f);
          if (g.mode == kEpiBiasRelu) x = fmaxf(x, 0.0f);
          v[i] = x;
        }
#pragma unroll
        for (int i = 0; i < 16; i += 4)
          *reinterpret_cast<float4 *>(stg + lane * kEpiRowFloats + cc + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
      }
      __syncwarp();
      const int cl = 4 * (lane & 15);  // this lane's 4 columns of the block
      // the ReLU reference of the lane's 16 (row, 4-column) pieces, all loads in flight at once
      uint2 rref[16];
      if (g.mode == kEpiReluMask) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int row = row0 + 2 * q + (lane >> 4);
          rref[q] = (cl < nb && row < g.M)
                        ? *reinterpret_cast<const uint2 *>(g.relu_ref + (size_t)row * g.ldr + c0 + cl)
                        : make_uint2(0u, 0u);
        }
      }
#pragma unroll
      for (int rr = 0; rr < 32; rr += 2) {
        const int r = rr + (lane >> 4), row = row0 + r;
        if (cl >= nb || row >= g.M) continue;
        const float4 x = *reinterpret_cast<const float4 *>(stg + r * kEpiRowFloats + cl);
        const size_t col = (size_t)(c0 + cl);
        if (g.mode == kEpiBiasF32) {
          *reinterpret_cast<float4 *>(g.out_f32 + (size_t)row * g.ldo + col) = x;
        } else if (g.mode == kEpiPartialF32) {
          *reinterpret_cast<float4 *>(g.out_f32 + (size_t)blockIdx.z * g.M * g.ldo + (size_t)row * g.ldo + col) = x;
        } else {
          float a = x.x, b = x.y, c = x.z, e = x.w;
          if (g.mode == kEpiReluMask) {  // gradient through the ReLU of the stored activation
            const uint2 rq = rref[rr >> 1];
            const __nv_bfloat162 r01 = *reinterpret_cast<const __nv_bfloat162 *>(&rq.x);
            const __nv_bfloat162 r23 = *reinterpret_cast<const __nv_bfloat162 *>(&rq.y);
            a = __low2float(r01) > 0.0f ? a : 0.0f;
            b = __high2float(r01) > 0.0f ? b : 0.0f;
            c = __low2float(r23) > 0.0f ? c : 0.0f;
            e = __high2float(r23) > 0.0f ? e : 0.0f;
          }
          const __nv_bfloat162 o01 = __floats2bfloat162_rn(a, b), o23 = __floats2bfloat162_rn(c, e);
          uint2 oq;
          oq.x = *reinterpret_cast<const uint32_t *>(&o01);
          oq.y = *reinterpret_cast<const uint32_t *>(&o23);
          *reinterpret_cast<uint2 *>(g.out_bf16 + (size_t)row * g.ldo + col) = oq;
        }
      }
      __syncwarp();
    }
  }
  if (fail_flag && tid == 0 && g.err) atomicExch(g.err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ----------------------------------------------------------------------------- fused forward
// The whole network for one 128-row tile in one CTA.  The tile's activations
// stay in shared memory (K-major, 256 columns: 64 KB, four 128 x 64 blocks in
// the 128-byte swizzle layout a tile copy would write) as the A operand of
// every layer.  The weights (N = 256 rows, K-major) come in
// 64-column chunks by tensor-map tile copies (128-byte swizzle) through four
// 32 KB stages: 13 chunks in all (one for the 16-feature layer, four for each
// other layer), chunk j in stage j % 4, its copy issued as soon as the MMAs
// of chunk j - 4 are complete, so the next layer's weights land while the
// current layer's epilogue runs.  One thread issues each chunk's MMAs as soon
// as its weights have landed and only then waits for the chunk before it, so
// the tensor pipe is never drained between chunks.  The accumulator (128 x
// 256 fp32, 256 TMEM columns) is read back by the epilogue (bias from shared
// memory, ReLU, bf16), which writes the next layer's input over the
// activations once the layer's MMAs are complete; when the hidden
// activations are asked for (training keeps them for the backward pass) the
// CTA copies them to global memory in full sectors while the next layer's
// MMAs run.  The last layer's fp32 logits are staged per warp in shared
// memory and written in 512-byte rows.  Eight warps: warp w reads TMEM lanes
// 32 (w mod 4) .. +31 (its rows) and accumulator columns 128 (w / 4) .. +127.
// Every wait is bounded; TMEM is always freed.
constexpr int kFwdLayers = 4;
constexpr int kFwdChunks = 13;
constexpr int kFwdStages = 4;
constexpr size_t kActBytes = (size_t)kTileM * 256 * 2;
constexpr size_t kWStage = 256 * kChunkK * 2;  // 32 KB
constexpr size_t kBiasBytes = (size_t)kFwdLayers * 256 * 4;
constexpr int kFwdThreads = 256;
constexpr int kZRow = 512 + 16;  // staged half logit row: 128 fp32 + 16 bytes against bank conflicts
constexpr size_t kFwdSmem = 1024 + kActBytes + kFwdStages * kWStage + kBiasBytes;
static_assert((kFwdThreads / 32) * 32 * kZRow <= kActBytes + kFwdStages * kWStage,
              "logit staging exceeds the free buffers");
static_assert(kFwdSmem <= 227 * 1024, "fused forward exceeds the shared-memory budget");

struct FwdTmaps {
  CUtensorMap w[kFwdLayers];
};

// Byte offset of the 16-byte segment `seg` (8 columns) of row r in the
// activation tile: block seg / 8 (64 columns, 16 KB), row r at 128 r, its
// 16-byte pieces permuted by the 128-byte swizzle (piece index XOR r mod 8).
__device__ __forceinline__ uint32_t act_offset(int r, int seg) {
  return (uint32_t)((seg >> 3) * (kTileM * 128) + r * 128 + (((seg & 7) ^ (r & 7)) << 4));
}

// 64 consecutive fp32 columns of this thread's TMEM lane; the wait is in the
// same statement, so no use of the registers can be scheduled before it.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
}

__global__ void __launch_bounds__(kFwdThreads)
    k_mlp_forward(const __grid_constant__ FwdTmaps tm, const __grid_constant__ FwdArgs g) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[kFwdStages], done[kFwdStages];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail_flag;
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *act = smem;
  uint8_t *wst = smem + kActBytes;
  float *bias_s = reinterpret_cast<float *>(wst + kFwdStages * kWStage);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, half = warp >> 2;  // TMEM lane quarter, accumulator column half
  const int trow = quad * 32 + lane;            // the tile row this thread reads back
  const int m0 = blockIdx.x * kTileM;

  if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), kTmemCols);
  if (tid == 0) {
    for (int s = 0; s < kFwdStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&done[s]), 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int l = 0; l < kFwdLayers; ++l)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm.w[l])) : "memory");
    fail_flag = 0;
  }
  // the biases, and layer 1's input: the tile's 16 features (bf16) into core-matrix columns 0..15
  for (int i = tid; i < kFwdLayers * 256; i += kFwdThreads) bias_s[i] = g.bias[i >> 8][i & 255];
  if (tid < kTileM) {
    const uint4 *src = reinterpret_cast<const uint4 *>(g.x0 + (size_t)(m0 + tid) * 16);
    const uint4 a = src[0], b = src[1];
    *reinterpret_cast<uint4 *>(act + act_offset(tid, 0)) = a;
    *reinterpret_cast<uint4 *>(act + act_offset(tid, 1)) = b;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16(kTileM, 256);
  const uint32_t act_a = smem_u32(act);
  const uint32_t wst_a = smem_u32(wst);
  // chunk j: layer 0 for j = 0, else layer 1 + (j - 1) / 4, K columns 64 ((j - 1) % 4) ...
  auto layer_of = [](int j) { return j == 0 ? 0 : 1 + (j - 1) / 4; };
  auto chunk_in_layer = [](int j) { return j == 0 ? 0 : (j - 1) % 4; };
  uint32_t done_seen = 0;  // bit j: the MMAs of chunk j have been waited for
  uint32_t full_seen = 0;  // bit j: the weights of chunk j have been waited for
  int issued = 0;          // chunks whose tile copy has been issued (in order)
  int committed = 0;       // chunks whose MMAs have been committed (in order)
  auto issue = [&](int j) {
    const int s = j % kFwdStages;
    mbar_expect_tx(smem_u32(&full[s]), (uint32_t)kWStage);
    tma_load_2d(wst_a + s * (uint32_t)kWStage, &tm.w[layer_of(j)], chunk_in_layer(j) * kChunkK, 0,
                smem_u32(&full[s]));
    ++issued;
  };
  // chunk j is the (j / 4)-th use of stage j % 4, hence phase parity (j / 4) & 1;
  // chunk j + 4 is issued only after the MMAs of chunk j completed, so no wait
  // ever looks at a phase two completions old
  auto wait_done = [&](int j) -> bool {
    if ((done_seen >> j) & 1u) return true;
    if (!mbar_wait(smem_u32(&done[j % kFwdStages]), (j / kFwdStages) & 1)) return false;
    done_seen |= 1u << j;
    return true;
  };
  auto wait_full = [&](int j) -> bool {
    if ((full_seen >> j) & 1u) return true;
    if (!mbar_wait(smem_u32(&full[j % kFwdStages]), (j / kFwdStages) & 1)) return false;
    full_seen |= 1u << j;
    return true;
  };
  // after chunk j's MMAs are complete its stage takes chunk j + 4
  auto refill = [&](int j) {
    if (j + kFwdStages < kFwdChunks && issued == j + kFwdStages) issue(j + kFwdStages);
  };
  if (tid == 0)
    for (int j = 0; j < kFwdStages; ++j) issue(j);

  int j0 = 0;  // first chunk of the current layer
  for (int l = 0; l < kFwdLayers; ++l) {
    const int nch = l == 0 ? 1 : 4;  // weight chunks of the layer
    bool ok = true;
    if (tid == 0 && !fail_flag) {
      for (int c = 0; c < nch && ok; ++c) {
        const int j = j0 + c, s = j % kFwdStages;
        ok = wait_full(j);
        if (!ok) break;
        tc_fence_after();
        const int ksteps = l == 0 ? 1 : 4;
        for (int kk = 0; kk < ksteps; ++kk) {
          const uint64_t ad = smem_desc_sw128(act_a + (uint32_t)c * (kTileM * 128) + kk * 32);
          const uint64_t bd = smem_desc_sw128(wst_a + s * (uint32_t)kWStage + kk * 32);
          mma_bf16(tmem, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(smem_u32(&done[s]));
        ++committed;
        if (c > 0) {  // the chunk before is complete once this one is queued behind it
          ok = wait_done(j - 1);
          if (ok) refill(j - 1);
        }
      }
    }
    // the previous layer's activations to global memory (16 rows x 64 bytes
    // per warp instruction) while this layer's MMAs read them
    if (l > 0 && g.h[l - 1]) {
      __nv_bfloat16 *hg = g.h[l - 1];
      for (int it = warp; it < 128; it += kFwdThreads / 32) {  // 16 row groups x 8 quads of segments
        const int r = (it >> 3) * 8 + (lane & 7), seg = (it & 7) * 4 + (lane >> 3);
        const uint4 u = *reinterpret_cast<const uint4 *>(act + act_offset(r, seg));
        *reinterpret_cast<uint4 *>(hg + (size_t)(m0 + r) * 256 + seg * 8) = u;
      }
    }
    if (tid == 0 && !fail_flag) {
      if (ok) ok = wait_done(j0 + nch - 1);  // the layer's accumulator is complete
      if (ok) refill(j0 + nch - 1);
      if (!ok) fail_flag = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (fail_flag) break;
    __syncwarp();  // the warp-wide tcgen05.ld below needs the whole warp converged
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
    const float4 *bl = reinterpret_cast<const float4 *>(bias_s + l * 256);
    if (l < kFwdLayers - 1) {
      // accumulator row trow -> + bias, ReLU, bf16 -> the next layer's input
      for (int q = half * 2; q < half * 2 + 2; ++q) {
        uint32_t r[64];
        tmem_ld64(lane_base + q * 64, r);
#pragma unroll
        for (int p = 0; p < 8; ++p) {  // 8 columns = one 16-byte segment
          const float4 b0 = bl[q * 16 + 2 * p], b1 = bl[q * 16 + 2 * p + 1];
          const float x[8] = {__uint_as_float(r[8 * p]) + b0.x,     __uint_as_float(r[8 * p + 1]) + b0.y,
                              __uint_as_float(r[8 * p + 2]) + b0.z, __uint_as_float(r[8 * p + 3]) + b0.w,
                              __uint_as_float(r[8 * p + 4]) + b1.x, __uint_as_float(r[8 * p + 5]) + b1.y,
                              __uint_as_float(r[8 * p + 6]) + b1.z, __uint_as_float(r[8 * p + 7]) + b1.w};
          uint32_t w[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(fmaxf(x[2 * i], 0.0f), fmaxf(x[2 * i + 1], 0.0f));
            w[i] = *reinterpret_cast<const uint32_t *>(&b2);
          }
          *reinterpret_cast<uint4 *>(act + act_offset(trow, q * 8 + p)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
      // the new activations are the next layer's A operand (read by the async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    } else {
      // logits: every MMA is complete and every copy consumed, so the
      // activation and weight buffers are free; each warp stages its 32 half rows
      uint8_t *zw = smem + (size_t)warp * 32 * kZRow;
      for (int q = half * 2; q < half * 2 + 2; ++q) {
        uint32_t r[64];
        tmem_ld64(lane_base + q * 64, r);
#pragma unroll
        for (int p = 0; p < 16; ++p) {
          const float4 b = bl[q * 16 + p];
          *reinterpret_cast<float4 *>(zw + (size_t)lane * kZRow + ((q - half * 2) * 16 + p) * 16) =
              make_float4(__uint_as_float(r[4 * p]) + b.x, __uint_as_float(r[4 * p + 1]) + b.y,
                          __uint_as_float(r[4 * p + 2]) + b.z, __uint_as_float(r[4 * p + 3]) + b.w);
        }
      }
      __syncwarp();
      for (int rr = 0; rr < 32; ++rr) {
        float *zg = g.z + (size_t)(m0 + quad * 32 + rr) * 256 + half * 128;
        *reinterpret_cast<float4 *>(zg + lane * 4) = *reinterpret_cast<const float4 *>(zw + (size_t)rr * kZRow + lane * 16);
      }
    }
    j0 += nch;
  }
  if (tid == 0) {
    // let every copy and MMA still in flight land (bounded) before the CTA exits
    for (int j = 0; j < issued; ++j) wait_full(j);
    for (int j = 0; j < committed; ++j) wait_done(j);
    if (fail_flag && g.err) atomicExch(g.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// Softmax cross-entropy over the valid steps t < steps[m] of each cell row;
// rows with label < 0 are padding.  dZ = (softmax - onehot) * inv_rows (bf16),
// loss_rows[m] = -log p[label] (0 for padding).  One warp per row, 8 columns
// per lane.
__global__ void k_softmax_ce(const float *Z, int ldz, const int32_t *label, const int32_t *steps, int M,
                             float inv_rows, __nv_bfloat16 *dZ, int ldd, float *loss_rows) {
  const int lane = threadIdx.x & 31;
  const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (m >= M) return;
  const int y = label[m], T = steps[m];
  float v[8];
  float mx = -INFINITY;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int t = lane * 8 + i;
    v[i] = (y >= 0 && t < T) ? Z[(size_t)m * ldz + t] : -INFINITY;
    mx = fmaxf(mx, v[i]);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    v[i] = (y >= 0 && lane * 8 + i < T) ? expf(v[i] - mx) : 0.0f;
    s += v[i];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __nv_bfloat16 *d = dZ + (size_t)m * ldd;
#pragma unroll
  for (int i = 0; i < 8; i += 2) {
    const int t = lane * 8 + i;
    float g0 = 0.0f, g1 = 0.0f;
    if (y >= 0) {
      g0 = (v[i] / s - (t == y ? 1.0f : 0.0f)) * inv_rows;
      g1 = (v[i + 1] / s - (t + 1 == y ? 1.0f : 0.0f)) * inv_rows;
    }
    *reinterpret_cast<__nv_bfloat162 *>(d + t) = __floats2bfloat162_rn(g0, g1);
  }
  if (y < 0) {
    if (lane == 0) loss_rows[m] = 0.0f;
  } else if (lane == (y >> 3)) {
    const float py = v[y & 7] / s;
    loss_rows[m] = -logf(fmaxf(py, 1e-30f));
  }
}

// partial[slab][n] = sum of Y[m][n] over the slab's rows, in row order.
__global__ void k_colsum(const __nv_bfloat16 *Y, int ld, int M, int N, float *partial) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int rows_per = (M + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * rows_per, r1 = min(M, r0 + rows_per);
  float s = 0.0f;
  for (int m = r0; m < r1; ++m) s += __bfloat162float(Y[(size_t)m * ld + n]);
  partial[(size_t)blockIdx.y * N + n] = s;
}

// out[i] = sum_{z < Z} ws[z * n + i], z in increasing order.
__global__ void k_sum_splits(const float *ws, int Z, int n, float *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f;
  for (int z = 0; z < Z; ++z) s += ws[(size_t)z * n + i];
  out[i] = s;
}

// out[0] = sum of v[0 .. n-1] in a fixed order: thread j sums j, j+256, ...;
// then thread 0 adds the 256 partial sums in order.
__global__ void __launch_bounds__(256) k_sum_ordered(const float *v, int n, float *out) {
  __shared__ float part[256];
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += 256) s += v[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int j = 0; j < 256; ++j) t += part[j];
    out[0] = t;
  }
}

// out[c][r] = in[r][c] for a bf16 R x C matrix (32 x 32 tiles).
__global__ void k_transpose(const __nv_bfloat16 *in, int R, int Cc, int ldi, __nv_bfloat16 *out, int ldo) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = blockIdx.y * 32 + j;
    tile[j][threadIdx.x] = (r < R && c < Cc) ? in[(size_t)r * ldi + c] : __float2bfloat16(0.0f);
  }
  __syncthreads();
  const int r2 = blockIdx.y * 32 + threadIdx.x;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c2 = blockIdx.x * 32 + j;
    if (c2 < Cc && r2 < R) out[(size_t)c2 * ldo + r2] = tile[threadIdx.x][j];
  }
}

// Adam on an fp32 master copy; writes the bf16 weight (rows x cols, row-major)
// and, when wt != null, its transpose.
__global__ void k_adam(float *w, float *m, float *v, const float *g, int rows, int cols, float lr, float b1,
                       float b2, float eps, float c1, float c2, __nv_bfloat16 *wb, __nv_bfloat16 *wt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const float gr = g[e];
  const float mm = b1 * m[e] + (1.0f - b1) * gr;
  const float vv = b2 * v[e] + (1.0f - b2) * gr * gr;
  m[e] = mm;
  v[e] = vv;
  const float upd = lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  const float nw = w[e] - upd;
  w[e] = nw;
  if (wb) {
    const __nv_bfloat16 b = __float2bfloat16(nw);
    wb[e] = b;
    if (wt) wt[(size_t)(e % cols) * rows + e / cols] = b;
  }
}

__global__ void k_f32_to_bf16(const float *in, __nv_bfloat16 *out, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = __float2bfloat16(in[e]);
}

}  // namespace

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tile-map encoder, looked up once through the runtime.
EncodeTiled encoder() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// Row-major bf16 matrix [rows x K] with row stride ld (elements) as tiles of
// 64 (K) x box_rows, 128-byte swizzle, zeros outside the matrix.
bool tile_map(CUtensorMap *map, const __nv_bfloat16 *base, int rows, int K, int ld, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) || ((size_t)ld * 2) % 16) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kChunkK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int gemm_splits(int K, int splits) {
  int kps = (K + splits - 1) / splits;
  kps = (kps + kChunkK - 1) / kChunkK * kChunkK;
  return (K + kps - 1) / kps;
}

cudaError_t sum_splits(const float *ws, int splits, int n, float *out, cudaStream_t st) {
  k_sum_splits<<<(n + 255) / 256, 256, 0, st>>>(ws, splits, n, out);
  return cudaGetLastError();
}

cudaError_t gemm(const GemmArgs &g, int splits, cudaStream_t st) {
  if (g.N < 16 || g.N > 256 || (g.N & 15) || (g.K & 15) || (g.lda & 7) || (g.ldb & 7) || (g.ldo & 3) ||
      (g.mode == kEpiReluMask && (g.ldr & 3)) || splits < 1)
    return cudaErrorInvalidValue;
  // set on every call: the attribute belongs to the current device
  if (cudaError_t e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
      e != cudaSuccess)
    return e;
  alignas(64) CUtensorMap ta, tb;
  if (!tile_map(&ta, g.A, g.M, g.K, g.lda, kTileM) || !tile_map(&tb, g.B, g.N, g.K, g.ldb, g.N))
    return cudaErrorInvalidValue;
  GemmArgs a = g;
  int kps = (g.K + splits - 1) / splits;
  kps = (kps + kChunkK - 1) / kChunkK * kChunkK;
  a.k_per_split = kps;
  const int zs = (g.K + kps - 1) / kps;
  dim3 grid((g.M + kTileM - 1) / kTileM, 1, zs);
  k_gemm_tc<<<grid, 128, kGemmSmem, st>>>(ta, tb, a);
  return cudaGetLastError();
}

cudaError_t forward(const FwdArgs &g, const __nv_bfloat16 *const w[4], cudaStream_t st) {
  if (g.Mp <= 0 || (g.Mp % kTileM) || !g.x0 || !g.z) return cudaErrorInvalidValue;
  if (cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
      e != cudaSuccess)
    return e;
  alignas(64) FwdTmaps tm;
  for (int l = 0; l < kFwdLayers; ++l) {
    const int K = l == 0 ? 16 : 256;
    if (!g.bias[l] || !tile_map(&tm.w[l], w[l], 256, K, K, 256)) return cudaErrorInvalidValue;
  }
  k_mlp_forward<<<g.Mp / kTileM, kFwdThreads, kFwdSmem, st>>>(tm, g);
  return cudaGetLastError();
}

cudaError_t softmax_ce(const float *Z, int ldz, const int32_t *label, const int32_t *steps, int M, float inv_rows,
                       __nv_bfloat16 *dZ, int ldd, float *loss_rows, float *loss_sum, cudaStream_t st) {
  k_softmax_ce<<<(M + 7) / 8, 256, 0, st>>>(Z, ldz, label, steps, M, inv_rows, dZ, ldd, loss_rows);
  k_sum_ordered<<<1, 256, 0, st>>>(loss_rows, M, loss_sum);
  return cudaGetLastError();
}

cudaError_t colsum(const __nv_bfloat16 *Y, int ld, int M, int N, float *partial, float *out, cudaStream_t st) {
  dim3 grid((N + 127) / 128, kColsumSlabs);
  k_colsum<<<grid, 128, 0, st>>>(Y, ld, M, N, partial);
  return sum_splits(partial, kColsumSlabs, N, out, st);
}

cudaError_t transpose(const __nv_bfloat16 *in, int R, int Cc, int ldi, __nv_bfloat16 *out, int ldo,
                      cudaStream_t st) {
  dim3 grid((Cc + 31) / 32, (R + 31) / 32), block(32, 8);
  k_transpose<<<grid, block, 0, st>>>(in, R, Cc, ldi, out, ldo);
  return cudaGetLastError();
}

cudaError_t adam(float *w, float *m, float *v, const float *g, int rows, int cols, float lr, float b1, float b2,
                 float eps, int step, __nv_bfloat16 *wb, __nv_bfloat16 *wt, cudaStream_t st) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  const int n = rows * cols;
  k_adam<<<(n + 255) / 256, 256, 0, st>>>(w, m, v, g, rows, cols, lr, b1, b2, eps, c1, c2, wb, wt);
  return cudaGetLastError();
}

cudaError_t to_bf16(const float *in, __nv_bfloat16 *out, int n, cudaStream_t st) {
  k_f32_to_bf16<<<(n + 255) / 256, 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace qp
