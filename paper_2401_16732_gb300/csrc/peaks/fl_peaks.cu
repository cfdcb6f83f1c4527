// Roofline ceilings measured on the running GPU, for the throughput
// measurements (not part of the homomorphic-convolution path).
//
// fl_measure_butterfly_rate: the lazy Gentleman-Sande butterfly of the
// inverse NTT (the same gs_bfly the transforms use: one Shoup product, sums
// and conditional subtractions on 30-bit residues), issued from registers
// with no memory traffic: every thread runs 16 independent butterfly chains,
// so the rate is bounded by the SM's integer pipes and issue, the ceiling of
// any kernel made of these butterflies.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../../include/flpeaks.h"
#include "../fl_device.cuh"

namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(256) k_bfly_rate(int iters, uint32_t q, uint32_t w, uint32_t wsh,
                                                   uint32_t* __restrict__ sink) {
  const uint32_t two_q = 2 * q;
  uint32_t x[kChains], y[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    x[k] = (threadIdx.x * 7919u + k * 104729u + blockIdx.x) % q;
    y[k] = (threadIdx.x * 6007u + k * 7907u + blockIdx.x * 3u) % q;
  }
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) fl::gs_bfly(x[k], y[k], w, wsh, q, two_q);
  }
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc ^= x[k] + y[k];
  if (acc == 0xFFFFFFFFu) sink[blockIdx.x] = acc;  // keeps the chains live; never true for residues
}

}  // namespace

extern "C" int fl_measure_butterfly_rate(int iters, double* butterflies_per_s) {
  if (!butterflies_per_s || iters < 1) return -1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return -3;
  const uint32_t q = 1073692673u, w = 123456789u;  // a 30-bit NTT prime and a twiddle below it
  const uint32_t wsh = (uint32_t)(((uint64_t)w << 32) / q);
  uint32_t* sink = nullptr;
  if (cudaMalloc(&sink, (size_t)sms * 4 * sizeof(uint32_t)) != cudaSuccess) return -4;
  const int blocks = sms * 4;  // 4 CTAs x 256 threads per SM: the register file's limit at 64 registers
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = 0;
  if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) rc = -3;
  if (!rc) {
    k_bfly_rate<<<blocks, 256>>>(iters / 8 + 1, q, w, wsh, sink);  // warm-up
    cudaEventRecord(e0);
    k_bfly_rate<<<blocks, 256>>>(iters, q, w, wsh, sink);
    cudaEventRecord(e1);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
      rc = -3;
    else
      *butterflies_per_s = (double)blocks * 256 * kChains * (double)iters / (ms * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return rc;
}
