// Roofline ceilings measured on the running GPU, for the throughput
// measurements (not part of the homomorphic-convolution path).
//
// fl_measure_butterfly_rate: the lazy Gentleman-Sande butterfly of the
// inverse NTT (the same gs_bfly the transforms use: one Shoup product, sums
// and conditional subtractions on 30-bit residues), issued from registers
// with no memory traffic: every thread runs 16 independent butterfly chains,
// so the rate is bounded by the SM's integer pipes and issue, the ceiling of
// any kernel made of these butterflies.
//
// fl_measure_tc_f16_rate: tcgen05.mma kind::f16 (fp16 operands, fp32
// accumulators in tensor memory) of shape M128 x N x K16, issued back to back
// by one thread of one CTA per SM on operands resident in shared memory (the
// canonical no-swizzle K-major layout), every MMA accumulating into the same
// tensor-memory columns: the instruction's own rate, without operand traffic.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

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

constexpr int kTcK = 64;                     // K extent of the resident operands (4 MMAs of K16)
constexpr int kTcSmem = 120 * 1024;          // > half of the SM's shared memory: one CTA per SM
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// shared-memory matrix descriptor without swizzle: start, leading byte offset
// (next 8 x 16-byte core matrix along K), stride byte offset (next 8 rows),
// descriptor version 1 at bit 46
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}
// kind::f16 instruction descriptor: fp32 D, fp16 A and B, both K-major
__host__ __device__ constexpr uint32_t f16_idesc(int m, int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// wait for phase 0 of the mbarrier, at most kWaitNs; false if it ran out
__device__ __forceinline__ bool wait_phase0(uint64_t* bar) {
  const unsigned long long t0 = now_ns();
  for (unsigned polls = 0; polls < (1u << 24); ++polls) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(su32(bar))
        : "memory");
    if (done) return true;
    if (now_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

template <int N>
__global__ void __launch_bounds__(128, 1) k_tc_rate(int iters, unsigned long long* cycles, unsigned* err) {
  constexpr uint32_t kCols = N < 32 ? 32 : N;  // tensor-memory columns of the M128 x N fp32 accumulator
  constexpr int kc = kTcK / 8;                 // 16-byte K chunks per row
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x;
  // A (128 x 64) and B (N x 64) halves, all 1.0: the values do not change the rate
  for (int e = tid; e < (128 + N) * kTcK / 2; e += 128) reinterpret_cast<uint32_t*>(sm)[e] = 0x3C003C00u;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tbase)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t d = tbase, a0 = su32(sm), b0 = a0 + 128 * kTcK * 2;
  const long long c0 = clock64();
  if (tid == 0) {
    for (int it = 0; it < iters; ++it)
      for (int k = 0; k < kTcK / 16; ++k) {
        const uint64_t ad = sdesc(a0 + 256 * k, 128, kc * 128), bd = sdesc(b0 + 256 * k, 128, kc * 128);
        const uint32_t acc = (it | k) != 0;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(ad), "l"(bd), "r"(f16_idesc(128, N)), "r"(acc)
            : "memory");
      }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&done))
                 : "memory");
  }
  // every MMA of the CTA is complete once the commit's arrival lands; if the
  // bound runs out, record it and wait once more (also bounded) so that no
  // MMA still writes the columns when they are freed
  bool ok = wait_phase0(&done);
  if (!ok) {
    if (tid == 0) atomicOr(err, 1u);
    ok = wait_phase0(&done);
    if (!ok && tid == 0) atomicOr(err, 2u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid == 0) cycles[blockIdx.x] = (unsigned long long)(clock64() - c0);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(d), "r"(kCols) : "memory");
}

template <int N>
int tc_rate(int sms, int iters, double* flops_per_s, double* cycles_per_mma) {
  unsigned long long* cyc = nullptr;
  unsigned* err = nullptr;
  if (cudaMalloc(&cyc, (size_t)sms * sizeof *cyc) != cudaSuccess) return -4;
  if (cudaMalloc(&err, sizeof *err) != cudaSuccess) {
    cudaFree(cyc);
    return -4;
  }
  int rc = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMemset(err, 0, sizeof *err) || cudaEventCreate(&e0) || cudaEventCreate(&e1) ||
      cudaFuncSetAttribute(k_tc_rate<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem))
    rc = -3;
  if (!rc) {
    k_tc_rate<N><<<sms, 128, kTcSmem>>>(iters / 8 + 1, cyc, err);  // warm-up
    cudaEventRecord(e0);
    k_tc_rate<N><<<sms, 128, kTcSmem>>>(iters, cyc, err);
    cudaEventRecord(e1);
    float ms = 0.f;
    unsigned e = 0;
    std::vector<unsigned long long> c(sms);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f ||
        cudaMemcpy(&e, err, sizeof e, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(c.data(), cyc, c.size() * sizeof c[0], cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = -3;
    } else if (e) {
      rc = -5;
    } else {
      const double mmas = (double)iters * (kTcK / 16);
      *flops_per_s = (double)sms * mmas * 2.0 * 128 * N * 16 / (ms * 1e-3);
      unsigned long long cmax = 0;
      for (unsigned long long v : c) cmax = v > cmax ? v : cmax;
      if (cycles_per_mma) *cycles_per_mma = (double)cmax / mmas;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(cyc);
  cudaFree(err);
  return rc;
}

}  // namespace

extern "C" int fl_measure_tc_f16_rate(int n, int iters, double* flops_per_s, double* cycles_per_mma) {
  if (!flops_per_s || iters < 1 || iters > (1 << 20) || (n != 64 && n != 128 && n != 256)) return -1;
  int dev = 0, sms = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev))
    return -3;
  if (major != 10 || minor != 3) return -2;  // the library's device code is built for sm_103a only
  switch (n) {
    case 64: return tc_rate<64>(sms, iters, flops_per_s, cycles_per_mma);
    case 128: return tc_rate<128>(sms, iters, flops_per_s, cycles_per_mma);
    default: return tc_rate<256>(sms, iters, flops_per_s, cycles_per_mma);
  }
}

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
