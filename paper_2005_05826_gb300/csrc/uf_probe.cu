// uf_probe.cu -- uf_probe_l2_atomics: the rate of random 64-bit atomic adds
// into a small (L2-resident) array, the ceiling the stripe-region scatter's
// atomics are measured against.  Each thread adds 1 to iters pseudo-random
// words (a multiplicative hash of its index and step), with no other memory
// traffic, so the L2 atomic units are the only bound.
#include <cuda_runtime.h>

#include <cstdint>

#include "uf_runtime.h"

namespace {

__global__ void k_atomic_probe(unsigned long long *__restrict__ buf, uint32_t mask, int iters) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t h = t * 2654435761u + 12345u;
  for (int i = 0; i < iters; i++) {
    h = h * 1664525u + 1013904223u;  // an LCG step per add (Numerical Recipes constants)
    atomicAdd(buf + ((h ^ (h >> 15)) & mask), 1ull);
  }
}

}  // namespace

extern "C" __attribute__((visibility("default"))) uf_status uf_probe_l2_atomics(int64_t bytes, double *adds_per_second) {
  using namespace ufg::rt;
  if (!adds_per_second) return fail(UF_EINVAL, "adds_per_second is NULL");
  *adds_per_second = 0.0;
  const int64_t words = bytes / 8;
  if (words < 1024 || words > ((int64_t)1 << 31) || (words & (words - 1)))
    return fail(UF_EINVAL, "bytes must be 8 x a power of two between 1024 and 2^31 words");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(UF_ECUDA, "no CUDA device");
  unsigned long long *buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaMalloc(&buf, (size_t)words * 8);
  if (err == cudaSuccess) err = cudaMemset(buf, 0, (size_t)words * 8);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  const int threads = 256, blocks = sms * 8, iters = 256;
  float ms = 0.f;
  if (err == cudaSuccess) {
    k_atomic_probe<<<blocks, threads>>>(buf, (uint32_t)(words - 1), iters);  // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < 8; r++) k_atomic_probe<<<blocks, threads>>>(buf, (uint32_t)(words - 1), iters);
    cudaEventRecord(e1);
    err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  if (err != cudaSuccess) return fail(UF_ECUDA, "atomic probe: %s", cudaGetErrorString(err));
  if (!(ms > 0.f)) return fail(UF_ECUDA, "atomic probe: no elapsed time");
  *adds_per_second = 8.0 * blocks * threads * (double)iters / (ms / 1e3);
  return UF_OK;
}
