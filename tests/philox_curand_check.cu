// Test helper (built by tests/test_gpu_philox.py): the library's device Philox4x32-10
// and cuRAND's raw Philox4x32-10 on the same counters and keys, word for word.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

#include "../paper_1807_09896_gb300/csrc/dpd_common.cuh"

__global__ void k_both(const uint32_t* ctr, const uint32_t* key, int n, uint32_t* ours, uint32_t* theirs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t c0 = ctr[4 * i], c1 = ctr[4 * i + 1], c2 = ctr[4 * i + 2], c3 = ctr[4 * i + 3];
  const uint32_t k0 = key[2 * i], k1 = key[2 * i + 1];
  const uint4 r = curand_Philox4x32_10(make_uint4(c0, c1, c2, c3), make_uint2(k0, k1));
  dpd::philox4x32_10(c0, c1, c2, c3, k0, k1);
  ours[4 * i] = c0;
  ours[4 * i + 1] = c1;
  ours[4 * i + 2] = c2;
  ours[4 * i + 3] = c3;
  theirs[4 * i] = r.x;
  theirs[4 * i + 1] = r.y;
  theirs[4 * i + 2] = r.z;
  theirs[4 * i + 3] = r.w;
}

extern "C" int philox_both(const uint32_t* ctr, const uint32_t* key, int n, uint32_t* ours, uint32_t* theirs) {
  uint32_t *dc = nullptr, *dk = nullptr, *d1 = nullptr, *d2 = nullptr;
  const size_t m = n > 0 ? (size_t)n : 1;
  cudaError_t e = cudaMalloc(&dc, 16 * m);
  if (e == cudaSuccess) e = cudaMalloc(&dk, 8 * m);
  if (e == cudaSuccess) e = cudaMalloc(&d1, 16 * m);
  if (e == cudaSuccess) e = cudaMalloc(&d2, 16 * m);
  if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, 16 * m, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dk, key, 8 * m, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n > 0) {
    k_both<<<(n + 255) / 256, 256>>>(dc, dk, n, d1, d2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(ours, d1, 16 * m, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(theirs, d2, 16 * m, cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(d1);
  cudaFree(d2);
  return (int)e;
}
