// On-the-fly weights: the convolution of fl_he_conv2d without the encoded
// NTT-domain weights.  Each CTA rebuilds the weight polynomials W_{i,g} it
// needs from the int8 filters in shared memory and forward-transforms them
// there, so the only weight state is the filter tensor itself.  This
// removes the NTT-weight footprint that the paper's Table 3 warns about
// (Cout*G*L*N*4 bytes per layer: 1.88 GiB for ResNet-18 at N = 8192, 56.7 GiB
// for ResNet-50 at N = 16384).  The price is one extra forward NTT per
// (image, output channel, limb, g).
//
// Per CTA (image/band bb, output channel i, limb l), 2 * N/32 threads, three
// padded polynomials of shared memory (two accumulators and one weight):
//   for g < G:  scatter the c_n*k^2 taps of W_{i,g} (x^-e = -x^(N-e)),
//               forward NTT (first N/32 threads),
//               acc_c += W_hat * C_hat[band*G+g][c]   (mod q_l, both c)
//   inverse NTT of both accumulators (+ Delta*r on c0), as in k_conv_intt.
#include <cuda_runtime.h>

#include "fl_device.cuh"
#include "fl_launch.h"

namespace fl {

template <int LOGN>
__global__ void __launch_bounds__(2 * ((1 << LOGN) / 32), minb_two_polys<LOGN>())
    k_conv_otf(const int8_t* __restrict__ w, const uint32_t* __restrict__ c_hat, uint32_t* __restrict__ out,
               const uint32_t* __restrict__ r, GeomDims gd, const uint32_t* __restrict__ tw, CtxConst cc) {
  constexpr int N = 1 << LOGN, T = N / 32, T2 = 2 * T, SW = Geo<LOGN>::SMEM_WORDS;
  constexpr int R1 = Plan<LOGN>::R1, R2 = Plan<LOGN>::R2;
  extern __shared__ uint32_t sm[];
  uint32_t* s0 = sm;
  uint32_t* s1 = sm + SW;
  uint32_t* sw = sm + 2 * SW;
  const int tid = threadIdx.x, L = cc.L;
  const int bb = blockIdx.x, i = blockIdx.y, l = blockIdx.z;
  const int b = bb / gd.bands, band = bb % gd.bands;
  const LimbConst lc = cc.limb[l];
  const uint32_t q = lc.q;
  const uint32_t* tw_l = tw + (size_t)l * TwLayout<LOGN>::LIMB_WORDS;
  const uint2* f = reinterpret_cast<const uint2*>(tw_l) + TW_FWD * N;
  const uint4* tg = reinterpret_cast<const uint4*>(tw_l + TwLayout<LOGN>::PAIRS_WORDS) + TW_FWD * 16 * T;
  const size_t ct_words = (size_t)2 * L * N;
  const uint32_t* C = c_hat + ((size_t)b * gd.n_in + (size_t)band * gd.G) * ct_words + (size_t)l * N;
  const int kk = gd.k * gd.k;
  const int8_t* wi = w + (size_t)i * gd.Cin * kk;

  for (int u = tid; u < SW; u += T2) s0[u] = s1[u] = 0;
#pragma unroll 1
  for (int g = 0; g < gd.G; ++g) {
    __syncthreads();  // the previous g's products are done reading sw
    for (int u = tid; u < SW; u += T2) sw[u] = 0;
    __syncthreads();
    const int taps = min(gd.c_n, gd.Cin - g * gd.c_n) * kk;
    for (int t = tid; t < taps; t += T2) {
      const int jj = t / kk, tap = t % kk;
      const int e = (tap / gd.k) * gd.Wp + tap % gd.k + jj * gd.P;  // 0 <= e < N, distinct per (i, g)
      const int wv = wi[(size_t)(g * gd.c_n + jj) * kk + tap];
      // tap value times N^-1 mod q_l (the inverse NTT below leaves that factor out)
      const uint32_t raw = e == 0 ? (wv >= 0 ? (uint32_t)wv : q - (uint32_t)(-wv))
                                  : (wv > 0 ? q - (uint32_t)wv : (uint32_t)(-wv));
      sw[e == 0 ? 0 : pad(N - e)] = csub(shoup_mul(raw, lc.n_inv, lc.n_inv_sh, q), q);
    }
    __syncthreads();
    if (tid < T) fwd_pass<LOGN, T, 0, R1, false>(sw, nullptr, f, q, lc.two_q, tid);
    __syncthreads();
    if (tid < T) {
      fwd_pass<LOGN, T, R1, R2, false>(sw, nullptr, f, q, lc.two_q, tid);
    }
    __syncthreads();
    if (tid < T) {
      uint32_t v[32];
      uint32_t* p = sw + tid * ROW;
      lds_row(p, v);
      pass32<false>(v, tg, T, tid, q, lc.two_q);
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = csub(csub(v[k], lc.two_q), q);  // [0, q)
      sts_row(p, v);
    }
    __syncthreads();
    const uint4* X0 = reinterpret_cast<const uint4*>(C + (size_t)g * ct_words);
    const uint4* X1 = reinterpret_cast<const uint4*>(C + (size_t)g * ct_words + (size_t)L * N);
    for (int v = tid; v < N / 4; v += T2) {
      const uint4 x0 = __ldg(X0 + v), x1 = __ldg(X1 + v);
      const int pu = pad(4 * v);
      const uint32_t xs0[4] = {x0.x, x0.y, x0.z, x0.w}, xs1[4] = {x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint64_t wv = sw[pu + j];
        s0[pu + j] = csub(s0[pu + j] + barrett64(wv * xs0[j], q, lc.mu), q);
        s1[pu + j] = csub(s1[pu + j] + barrett64(wv * xs1[j], q, lc.mu), q);
      }
    }
  }
  __syncthreads();

  const int h = tid >= T, lt = tid - h * T;
  const size_t oct = (size_t)b * gd.n_out + (size_t)i * gd.bands + band;
  uint32_t* op = out + oct * ct_words + (size_t)h * L * N + (size_t)l * N;
  const uint32_t* rr = (r && h == 0) ? r + oct * N : nullptr;
  intt_from_smem_unscaled<LOGN>(h ? s1 : s0, tw_l, lc, lt, MaskStore{op, rr, lc});
}

template <int LOGN>
static cudaError_t otf_setup() {
  const int smem = 3 * Geo<LOGN>::SMEM_WORDS * 4;
  return cudaFuncSetAttribute(k_conv_otf<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_otf_setup(int logn) {
  switch (logn) {
    case 11: return otf_setup<11>();
    case 12: return otf_setup<12>();
    case 13: return otf_setup<13>();
    case 14: return otf_setup<14>();
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_conv_otf(int logn, int B, const GeomDims& gd, const int8_t* w, const uint32_t* c_hat,
                            uint32_t* out, const uint32_t* r, const uint32_t* tw, const CtxConst& cc,
                            cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  const int N = 1 << logn;
  const size_t smem = (size_t)3 * padded_words(N) * 4;
  dim3 grid(B * gd.bands, gd.Cout, cc.L);
  switch (logn) {
    case 11: k_conv_otf<11><<<grid, N / 16, smem, st>>>(w, c_hat, out, r, gd, tw, cc); break;
    case 12: k_conv_otf<12><<<grid, N / 16, smem, st>>>(w, c_hat, out, r, gd, tw, cc); break;
    case 13: k_conv_otf<13><<<grid, N / 16, smem, st>>>(w, c_hat, out, r, gd, tw, cc); break;
    case 14: k_conv_otf<14><<<grid, N / 16, smem, st>>>(w, c_hat, out, r, gd, tw, cc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fl
