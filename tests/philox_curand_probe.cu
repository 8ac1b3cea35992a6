// Test helper: cuRAND's Philox4x32-10 (an independent implementation of the
// generator the annealer draws from) evaluated on the GPU for given counters
// and keys, so the oracle's generator can be compared with it.
#include <cuda_runtime.h>
#include <curand_philox4x32_x.h>

__global__ void k_curand_philox(const uint4 *ctr, const uint2 *key, uint4 *out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

// ctr: n x 4 words, key: n x 2 words, out: n x 4 words (host).  0 on success.
extern "C" int curand_philox_batch(const unsigned *ctr, const unsigned *key, unsigned *out, int n) {
  uint4 *dc = nullptr, *dout = nullptr;
  uint2 *dk = nullptr;
  int rc = 1;
  if (cudaMalloc(&dc, sizeof(uint4) * n) == cudaSuccess && cudaMalloc(&dk, sizeof(uint2) * n) == cudaSuccess &&
      cudaMalloc(&dout, sizeof(uint4) * n) == cudaSuccess &&
      cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice) == cudaSuccess &&
      cudaMemcpy(dk, key, sizeof(uint2) * n, cudaMemcpyHostToDevice) == cudaSuccess) {
    k_curand_philox<<<(n + 255) / 256, 256>>>(dc, dk, dout, n);
    if (cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
        cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost) == cudaSuccess)
      rc = 0;
  }
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return rc;
}
