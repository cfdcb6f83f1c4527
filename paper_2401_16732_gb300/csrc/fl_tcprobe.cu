// Throughput probe of the warp-level tensor-core instructions a byte-split
// contraction could use on sm_103a (tcgen05 has no integer kind there):
//   kind 0: mma.sync m16n8k32, u8 x u8 -> s32 (exact integer products)
//   kind 1: mma.sync m16n8k16, bf16 x bf16 -> f32 (exact for byte digits while
//           every partial sum stays below 2^24)
// Every warp keeps 8 independent accumulator tiles in registers and issues
// `iters` rounds of 8 MMAs on them; no memory traffic inside the loop.  The
// result is the measured multiply-add rate of the instruction, the ceiling
// of any contraction built on it.
#include <cuda_runtime.h>

#include <cstdint>

namespace fl {

__global__ void __launch_bounds__(256) k_mma_probe_u8(int iters, uint32_t seed, uint32_t* sink) {
  uint32_t a[4], b[2];
#pragma unroll
  for (int j = 0; j < 4; ++j) a[j] = seed * (threadIdx.x + 1 + j);
#pragma unroll
  for (int j = 0; j < 2; ++j) b[j] = seed * (threadIdx.x + 7 + j);
  uint32_t acc[8][4];
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[t][j] = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int t = 0; t < 8; ++t)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+r"(acc[t][0]), "+r"(acc[t][1]), "+r"(acc[t][2]), "+r"(acc[t][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  uint32_t x = 0;
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int j = 0; j < 4; ++j) x ^= acc[t][j];
  if (x == 0x9e3779b9u) sink[threadIdx.x] = x;  // keeps the loop alive; practically never taken
}

__global__ void __launch_bounds__(256) k_mma_probe_bf16(int iters, uint32_t seed, uint32_t* sink) {
  // operands: pairs of small byte-valued bf16 numbers (exact), accumulators f32
  uint32_t a[4], b[2];
  const uint32_t one_two = 0x3f804000u;  // bf16 {2.0, 1.0}
#pragma unroll
  for (int j = 0; j < 4; ++j) a[j] = one_two;
#pragma unroll
  for (int j = 0; j < 2; ++j) b[j] = one_two;
  float acc[8][4];
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[t][j] = 0.f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int t = 0; t < 8; ++t)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  uint32_t x = seed;
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int j = 0; j < 4; ++j) x ^= __float_as_uint(acc[t][j]);
  if (x == 0x9e3779b9u) sink[threadIdx.x] = x;
}

cudaError_t probe_mma_rate(int kind, int blocks, int iters, float* ms, double* macs) {
  uint32_t* sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, 256 * sizeof(uint32_t));
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
    cudaEventRecord(e0);
    if (kind == 0) k_mma_probe_u8<<<blocks, 256>>>(iters, 0x12345u, sink);
    else k_mma_probe_bf16<<<blocks, 256>>>(iters, 0x12345u, sink);
    cudaEventRecord(e1);
  }
  e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) cudaEventElapsedTime(ms, e0, e1);
  const double per_mma = kind == 0 ? 16.0 * 8 * 32 : 16.0 * 8 * 16;
  *macs = (double)blocks * (256 / 32) * iters * 8 * per_mma;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return e;
}

}  // namespace fl
