// Direct form of the convolution on the GPU: Algorithm 1's DRot + CMult,
// with no NTT and the int8 filters as they are.
//
// For output ciphertext (image b, output channel i, band), component c and
// limb l:
//   y[u] = sum_{j, ky, kx} w[i][j][ky][kx] * (x^-e * ct_g)[u],
//   e = ky*Wp + kx + (j mod c_n)*P,  g = band*G + j / c_n,
// where multiplication by x^-e is the DRot of Eq. 2 (a negacyclic shift:
// (x^-e * a)[u] = a[u+e] for u+e < N, -a[u+e-N] otherwise).  Products are
// accumulated exactly in signed 64 bits (lazy reduction, Sec. 6.1) and
// reduced once per output coefficient.  The result is the same polynomial
// the NTT route computes.
//
// One CTA per (image/band, CI output channels, component x limb).  The
// input polynomial of each packed group goes through shared memory, and
// every thread keeps CI x 4 accumulators (its 4 coefficients of one 1024-wide
// chunk, for CI output channels) in registers.  Each shared-memory read
// feeds CI multiply-adds.
#include <cuda_runtime.h>

#include "fl_device.cuh"
#include "fl_launch.h"

namespace fl {

constexpr int kDirectThreads = 256;
constexpr int kDirectCI = 4;

template <int LOGN, bool MASK>
__global__ void __launch_bounds__(kDirectThreads)
    k_direct(const int8_t* __restrict__ w, const uint32_t* __restrict__ ct, uint32_t* __restrict__ out,
             const uint32_t* __restrict__ r, GeomDims g, CtxConst cc) {
  constexpr int N = 1 << LOGN, CI = kDirectCI, CHUNK = 4 * kDirectThreads;
  extern __shared__ uint32_t sm[];
  const int kk = g.k * g.k, KW = g.Cin * kk;
  int8_t* ws = reinterpret_cast<int8_t*>(sm + N);  // [CI][Cin][k][k]
  const int tid = threadIdx.x;
  const int bb = blockIdx.x, i0 = blockIdx.y * CI, cl = blockIdx.z, L = cc.L;
  const int b = bb / g.bands, band = bb % g.bands;
  const int c = cl / L, l = cl % L;
  const LimbConst lc = cc.limb[l];
  const int nci = min(CI, g.Cout - i0);
  for (int x = tid; x < CI * KW; x += kDirectThreads) {
    const int ci = x / KW;
    ws[x] = ci < nci ? w[(size_t)(i0 + ci) * KW + x % KW] : (int8_t)0;
  }
  const size_t row_stride = (size_t)2 * L * N;  // words between consecutive ciphertexts
  const uint32_t* in0 = ct + ((size_t)b * g.n_in + (size_t)band * g.G) * row_stride + ((size_t)c * L + l) * N;
  // |acc| <= Cin*k^2 * 128 * 2^30 < 2^51 (the host caps Cin*k^2 at 2^14); OFF > 2^51 makes it non-negative
  const uint64_t OFF = (uint64_t)lc.q << 22;

#pragma unroll 1
  for (int ch = 0; ch < N / CHUNK; ++ch) {
    long long acc[CI][4];
#pragma unroll
    for (int ci = 0; ci < CI; ++ci)
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[ci][m] = 0;
    const int u0 = ch * CHUNK + tid;
#pragma unroll 1
    for (int gg = 0; gg < g.G; ++gg) {
      __syncthreads();  // previous group's reads (and the weight fill) are done
      const uint4* src = reinterpret_cast<const uint4*>(in0 + (size_t)gg * row_stride);
      for (int v = tid; v < N / 4; v += kDirectThreads) reinterpret_cast<uint4*>(sm)[v] = __ldg(src + v);
      __syncthreads();
      const int jn = min(g.c_n, g.Cin - gg * g.c_n);
#pragma unroll 1
      for (int jj = 0; jj < jn; ++jj) {
        const int j = gg * g.c_n + jj;
#pragma unroll 1
        for (int ky = 0; ky < g.k; ++ky) {
#pragma unroll 1
          for (int kx = 0; kx < g.k; ++kx) {
            const int e = ky * g.Wp + kx + jj * g.P;
            const int t = j * kk + ky * g.k + kx;
            int wv[CI];
#pragma unroll
            for (int ci = 0; ci < CI; ++ci) wv[ci] = ws[ci * KW + t];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              const int idx = u0 + m * kDirectThreads + e;
              const int xv = (int)sm[idx & (N - 1)];
              const int xs = idx >= N ? -xv : xv;  // the wrap of x^-e
#pragma unroll
              for (int ci = 0; ci < CI; ++ci) acc[ci][m] += (long long)wv[ci] * xs;
            }
          }
        }
      }
    }
#pragma unroll
    for (int ci = 0; ci < CI; ++ci) {
      if (ci >= nci) break;
      const size_t oc = (size_t)b * g.n_out + (size_t)(i0 + ci) * g.bands + band;
      uint32_t* o = out + oc * row_stride + ((size_t)c * L + l) * N;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int u = u0 + m * kDirectThreads;
        uint32_t y = barrett64((uint64_t)(acc[ci][m] + (long long)OFF), lc.q, lc.mu);
        if (MASK && c == 0) y = csub(csub(y + shoup_mul(__ldg(r + oc * N + u), lc.delta, lc.delta_sh, lc.q), lc.two_q), lc.q);
        o[u] = y;
      }
    }
  }
}

size_t direct_smem_bytes(int logn, int Cin, int k) {
  return ((size_t)4 << logn) + (((size_t)kDirectCI * Cin * k * k + 15) & ~(size_t)15);
}

template <int LOGN>
static cudaError_t direct_setup() {
  cudaError_t e;
  const int lim = 227 * 1024;
  if ((e = cudaFuncSetAttribute(k_direct<LOGN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaFuncSetAttribute(k_direct<LOGN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

cudaError_t launch_direct_setup(int logn) {
  switch (logn) {
    case 11: return direct_setup<11>();
    case 12: return direct_setup<12>();
    case 13: return direct_setup<13>();
    case 14: return direct_setup<14>();
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_direct(int logn, int B, const GeomDims& g, const int8_t* w, const uint32_t* ct, uint32_t* out,
                          const uint32_t* r, const CtxConst& cc, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  const size_t smem = direct_smem_bytes(logn, g.Cin, g.k);
  dim3 grid(B * g.bands, (g.Cout + kDirectCI - 1) / kDirectCI, 2 * cc.L);
#define FL_DIRECT_CASE(LG)                                                                             \
  case LG:                                                                                             \
    if (r) k_direct<LG, true><<<grid, kDirectThreads, smem, st>>>(w, ct, out, r, g, cc);               \
    else k_direct<LG, false><<<grid, kDirectThreads, smem, st>>>(w, ct, out, r, g, cc);                \
    break;
  switch (logn) {
    FL_DIRECT_CASE(11)
    FL_DIRECT_CASE(12)
    FL_DIRECT_CASE(13)
    FL_DIRECT_CASE(14)
    default: return cudaErrorInvalidValue;
  }
#undef FL_DIRECT_CASE
  return cudaGetLastError();
}

}  // namespace fl
