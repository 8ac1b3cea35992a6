// Device helpers shared by the sweep kernels: Philox4x32-10, the acceptance
// test, warp reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifndef QP_DEVICE_CHECKS
#define QP_DEVICE_CHECKS 0
#endif

namespace qp {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

// Device bounds checks, compiled in only with QP_DEVICE_CHECKS=1 (the checked
// build of the library).  QP_IX(i, n, site) is i when 0 <= i < n; otherwise
// the first failure of the translation unit's kernels is recorded as
// (site << 24) | (i mod 2^24) and the access goes to element 0, so a wrong
// index cannot reach memory outside its array.  Sites: 1 threshold table,
// 2 distance row, 3 spin word, 4 row of S, 5 repair distance, 6 hot-cell list.
// In the release build QP_IX(i, n, site) is i.
#if QP_DEVICE_CHECKS
static __device__ unsigned int g_check_word;
__device__ __forceinline__ long long check_ix(long long i, long long n, unsigned site) {
  if (i >= 0 && i < n) return i;
  atomicCAS(&g_check_word, 0u, (site << 24) | ((unsigned)i & 0xFFFFFFu));
  return 0;
}
#define QP_IX(i, n, site) ((decltype(i))::qp::dev::check_ix((long long)(i), (long long)(n), (site)))
// Host accessor of the translation unit's word: returns it and clears it.
#define QP_CHECK_ACCESSOR(fn)                                                        \
  uint32_t fn() {                                                                    \
    unsigned v = 0;                                                                  \
    if (cudaMemcpyFromSymbol(&v, ::qp::dev::g_check_word, sizeof v) != cudaSuccess) \
      return 0xFFFFFFFFu;                                                            \
    const unsigned z = 0;                                                            \
    cudaMemcpyToSymbol(::qp::dev::g_check_word, &z, sizeof z);                      \
    return v;                                                                        \
  }
#else
#define QP_IX(i, n, site) (i)
#define QP_CHECK_ACCESSOR(fn) \
  uint32_t fn() { return 0; }
#endif

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 S-box with
// the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    // each 32x32 -> 64-bit product as one wide multiply (both halves at once)
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The same generator with its key given as the seed's two words (round keys
// computed on the fly) or as the ten rounds' keys k0 + i W0, k1 + i W1
// computed once (launch constants, read straight from the kernel's argument
// block by the XORs).
struct PhiloxKey {
  uint32_t k0, k1;
};
struct RoundKeys {
  uint32_t k[20];  // k[2i] = k0 + i 0x9E3779B9, k[2i+1] = k1 + i 0xBB67AE85
};
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKey &key) {
  return philox4x32_10(c, key.k0, key.k1);
}
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys &rk) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ rk.k[2 * i], lo1, hi0 ^ c.w ^ rk.k[2 * i + 1], lo0);
  }
  return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4 &u, int j) {
  return j == 0 ? u.x : (j == 1 ? u.y : (j == 2 ? u.z : u.w));
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Relative margin of the float acceptance estimate.  The estimate
// v = 2^(32 - dE * log2(e)/T) carries a relative error below 1e-5: the product
// dE * c and the subtraction round to 2^-24 relative on an exponent of at most
// 64 in magnitude (3.8e-6 absolute, 2.7e-6 relative in 2^x), c = log2(e)/T is
// rounded to float (1.9e-6), exp2f is within 2 ulp (2.4e-7) and u -> float
// rounds to 6e-8.  The margin is 2^-12 = 2.4e-4, 40x that sum.
constexpr float kAcceptMargin = 1.0f / 4096.0f;

// Proposal with 1 <= dE < len: accept iff u < thr[dE], thr[dE] =
// floor(2^32 exp(-dE/T)) from the host table.  When u lies outside the band
// v(1 -/+ margin) -/+ 2 around the float estimate the answer is the table's
// (u < v(1-m) - 2 implies u < V - 1, hence u < floor(V); u > v(1+m) + 2
// implies u >= floor(V)); inside the band the table itself is read.
__device__ __forceinline__ bool accept_draw(uint32_t u, int dE, float c, const uint32_t *thr, int len) {
  const float v = exp2f(32.0f - (float)dE * c);
  const float uf = __uint2float_rn(u);
  if (uf < fmaf(v, -kAcceptMargin, v) - 2.0f) return true;
  if (uf > fmaf(v, kAcceptMargin, v) + 2.0f) return false;
  return u < __ldg(thr + QP_IX(dE, len, 1));
}

// ---- bulk copies global -> shared with mbarrier completion
constexpr long long kBulkWaitCycles = 1000000000LL;  // ~0.5 s at 2 GHz, then give up

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init1(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One thread asks for `bytes` (a multiple of 16, both addresses 16-byte
// aligned) from global `src` into shared `dst`; the copy engine counts the
// bytes on the mbarrier.  The proxy fence orders the thread's (and, after a
// __syncwarp, its warp's) earlier reads of dst before the asynchronous write.
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

// Wait for phase `parity` of the mbarrier, giving up after kBulkWaitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > kBulkWaitCycles) return false;
  }
}

}  // namespace dev
}  // namespace qp
