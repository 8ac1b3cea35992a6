// Self-test of the bounded mbarrier wait that guards every asynchronous copy
// in the library (the dense sweep's row copies): one warp waits on a phase
// that nothing will ever complete and must come back with "timed out" after
// the wait's bound instead of hanging, leaving the context usable.
#include "qp_device.cuh"
#include "qp_internal.h"

namespace qp {
namespace {

__global__ void k_selftest_wait(int32_t *timed_out, long long *cycles) {
  __shared__ __align__(8) uint64_t mbar;
  const uint32_t m = dev::smem_addr(&mbar);
  if (threadIdx.x == 0) {
    dev::mbar_init1(m);
    dev::mbar_init_fence();
  }
  __syncwarp();
  const long long t0 = clock64();
  // no thread arrives and no copy is issued: phase 0 never completes
  const bool done = dev::mbar_wait_bounded(m, 0);
  const long long t1 = clock64();
  if (threadIdx.x == 0) {
    *timed_out = done ? 0 : 1;
    *cycles = t1 - t0;
  }
}

}  // namespace
}  // namespace qp

extern "C" qp_status qp_selftest_wait(int32_t *timed_out, double *waited_ms) {
  using namespace qp;
  if (!timed_out) return set_error(QP_EINVAL, "timed_out is NULL");
  int32_t *d_flag = nullptr;
  long long *d_cyc = nullptr;
  if (cudaMalloc(&d_flag, 4) != cudaSuccess || cudaMalloc(&d_cyc, 8) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_flag);
    return set_error(QP_ENOMEM, "qp_selftest_wait: allocation failed");
  }
  k_selftest_wait<<<1, 32>>>(d_flag, d_cyc);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int32_t flag = -1;
  long long cyc = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flag, d_flag, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&cyc, d_cyc, 8, cudaMemcpyDeviceToHost);
  int dev = 0, khz = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  cudaFree(d_flag);
  cudaFree(d_cyc);
  if (e != cudaSuccess) return set_error(QP_ECUDA, cudaGetErrorString(e));
  *timed_out = flag;
  if (waited_ms) *waited_ms = khz > 0 ? (double)cyc / (double)khz : -1.0;
  return QP_OK;
}
