// Server side of the x^2 + x activation protocol (Sec. 5.2) and the batch
// (SIMD) encoding it needs (Sec. 2.2).
//
// Batch encoding over Z_t[x]/(x^N+1), t prime with t = 1 mod 2N: slot k of
// a plaintext m holds m(psi_t^(2k+1)) mod t, psi_t a primitive 2N-th root of
// unity mod t.  The forward negacyclic NTT mod t (fl_device.cuh, run on the
// tables of t) leaves m(psi_t^(2k+1)) at output position brev(k), so decoding
// is one NTT and a bit-reversal gather, and encoding one inverse NTT of the
// slots scattered to bit-reversed positions.
//
// Protocol, with z = a + r the client's masked activations (one vector of N
// values per ciphertext), X = z^2 + z and Y = 2rz + v:
//   offline   prep rows: NTT(N^-1 * lift(encode(2r))) per limb, encode(v), and the
//             direct-encoded constant r^2 - r + v (Sec. 6.3 keeps r, v and
//             r^2 precomputed)
//   round 1   <2rz + v>_batch = PMult(<z>_batch, encode(2r)) + encode(v)
//   round 2   <a^2 + a>      = <X> - <Y> + (r^2 - r + v), direct encoding
//
//   k_batch_decode   forward NTT mod t + gather, one CTA per plaintext
//   k_batch_encode   scatter + inverse NTT mod t, one CTA per plaintext;
//                    writes the plaintext in [0, t) or its centred lift to
//                    every ciphertext limb
//   k_x2x_const      r^2 - r + v mod t, elementwise
//   k_x2x_round1     forward NTT of both components, NTT-domain product with
//                    the prepared 2r, inverse NTT and + Delta*encode(v), one
//                    CTA per (ciphertext, limb); the product sits between the
//                    forward radix-32 pass and the inverse one in registers
//   k_x2x_round2     <X> - <Y> + Delta*(r^2 - r + v), elementwise (HBM-bound)
//   k_repack         a plain vector from a convolution's output layout to the
//                    next layer's zero-padded input layout
#include <cuda_runtime.h>

#include "fl_device.cuh"
#include "fl_launch.h"

namespace fl {

__device__ __forceinline__ int brev_n(int k, int logn) { return (int)(__brev((unsigned)k) >> (32 - logn)); }

// slots[c][k] = m_c(psi_t^(2k+1)); m values in [0, t).
template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 32, minb_one_poly<LOGN>())
    k_batch_decode(const uint32_t* __restrict__ m, uint32_t* __restrict__ slots, const uint32_t* __restrict__ tw_t,
                   LimbConst tc) {
  constexpr int N = 1 << LOGN, T = N / 32;
  extern __shared__ uint32_t sm[];
  const int c = blockIdx.x, tid = threadIdx.x;
  ntt_forward_to_smem<LOGN>(sm, m + (size_t)c * N, tw_t, tc, tid);
  __syncthreads();
  uint32_t* out = slots + (size_t)c * N;
  for (int k = tid; k < N; k += T) out[k] = sm[pad(brev_n(k, LOGN))];
}

// Plaintext c = encode(scale * slots[c] mod t).  lift_L == 0: written in
// [0, t) to dst + c*dst_stride.  lift_L > 0: the centred representative in
// (-t/2, t/2], times N^-1, is written mod q_l to dst + c*dst_stride + l*N,
// l < lift_L (the plaintext as a polynomial of R_q, the form PMult
// multiplies by, pre-scaled for round 1's unscaled inverse NTT).
template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 32, minb_one_poly<LOGN>())
    k_batch_encode(const uint32_t* __restrict__ slots, uint32_t scale, uint32_t* __restrict__ dst,
                   long long dst_stride, int lift_L, const uint32_t* __restrict__ tw_t, LimbConst tc,
                   CtxConst cc) {
  constexpr int N = 1 << LOGN, T = N / 32;
  extern __shared__ uint32_t sm[];
  const int c = blockIdx.x, tid = threadIdx.x;
  const uint32_t t = tc.q;
  const uint32_t* in = slots + (size_t)c * N;
  for (int k = tid; k < N; k += T) sm[pad(brev_n(k, LOGN))] = barrett64((uint64_t)__ldg(in + k) * scale, t, tc.mu);
  __syncthreads();
  uint32_t* o = dst + (size_t)c * dst_stride;
  const uint32_t half = t >> 1;
  intt_from_smem<LOGN>(sm, tw_t, tc, tid, [&](uint32_t v, int u) {
    const uint32_t m = csub(v, t);  // [0, t)
    if (lift_L == 0) {
      o[u] = m;
    } else {
      // centred lift, times N^-1 mod q_l (round 1's inverse NTT leaves that factor out)
      for (int l = 0; l < lift_L; ++l) {
        const LimbConst& lq = cc.limb[l];
        const uint32_t lifted = m > half ? lq.q - (t - m) : m;
        o[(size_t)l * N + u] = csub(shoup_mul(lifted, lq.n_inv, lq.n_inv_sh, lq.q), lq.q);
      }
    }
  });
}

// dst[c][u] = r^2 - r + v mod t (r, v < 2^32; reduced mod t first).
__global__ void k_x2x_const(const uint32_t* __restrict__ r, const uint32_t* __restrict__ v,
                            uint32_t* __restrict__ dst, long long dst_stride, int n, int N, LimbConst tc) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * N) return;
  const size_t c = idx / N, u = idx % N;
  const uint32_t t = tc.q;
  const uint32_t rr = barrett64(__ldg(r + idx), t, tc.mu), vv = barrett64(__ldg(v + idx), t, tc.mu);
  // rr^2 + (t - rr) + vv < 2^34 + 2^21 fits the 64-bit Barrett reduction
  dst[c * dst_stride + u] = barrett64((uint64_t)rr * rr + (t - rr) + vv, t, tc.mu);
}

// Round 1.  Grid (n, L), 2 * N/32 threads: threads [0, T) take c0, [T, 2T) c1.
// prep row layout per ciphertext: [L] NTT-domain 2r, [1] encode(v), [1] const.
template <int LOGN>
__global__ void __launch_bounds__(2 * ((1 << LOGN) / 32), minb_two_polys<LOGN>())
    k_x2x_round1(const uint32_t* __restrict__ prep, const uint32_t* ct, uint32_t* out,
                 const uint32_t* __restrict__ tw, CtxConst cc) {
  constexpr int N = 1 << LOGN, T = N / 32, SW = Geo<LOGN>::SMEM_WORDS;
  constexpr int R1 = Plan<LOGN>::R1, R2 = Plan<LOGN>::R2;
  extern __shared__ uint32_t sm[];
  const int c = blockIdx.x, l = blockIdx.y, L = cc.L, tid = threadIdx.x;
  const int h = tid >= T, lt = tid - h * T;
  const LimbConst lc = cc.limb[l];
  const uint32_t q = lc.q, two_q = lc.two_q;
  uint32_t* s = sm + h * SW;
  const uint32_t* tw_l = tw + (size_t)l * TwLayout<LOGN>::LIMB_WORDS;
  const uint2* f = reinterpret_cast<const uint2*>(tw_l) + TW_FWD * N;
  const uint2* fi = reinterpret_cast<const uint2*>(tw_l) + TW_INV * N;
  const uint4* tgf = reinterpret_cast<const uint4*>(tw_l + TwLayout<LOGN>::PAIRS_WORDS) + TW_FWD * 16 * T;
  const uint4* tgi = reinterpret_cast<const uint4*>(tw_l + TwLayout<LOGN>::PAIRS_WORDS) + TW_INV * 16 * T;
  const size_t row = ((size_t)c * 2 + h) * L + l;  // component h, limb l of ciphertext c
  const uint32_t* P = prep + ((size_t)c * (L + 2) + l) * N;
  const uint32_t* V = prep + ((size_t)c * (L + 2) + L) * N;

  // both halves run the same passes, so block-wide barriers serve both
  fwd_pass<LOGN, T, 0, R1, true>(s, ct + row * N, f, q, two_q, lt);
  __syncthreads();
  fwd_pass<LOGN, T, R1, R2, false>(s, nullptr, f, q, two_q, lt);
  __syncthreads();
  {
    uint32_t v[32];
    uint32_t* srow = s + lt * ROW;
    lds_row(srow, v);
    pass32<false>(v, tgf, T, lt, q, two_q);
    // NTT-domain entries lt*32 .. lt*32+31 of this component times those of 2r
    const uint4* P4 = reinterpret_cast<const uint4*>(P + lt * 32);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint4 p = __ldg(P4 + j);
      v[4 * j + 0] = red64_2q((uint64_t)v[4 * j + 0] * p.x, lc);
      v[4 * j + 1] = red64_2q((uint64_t)v[4 * j + 1] * p.y, lc);
      v[4 * j + 2] = red64_2q((uint64_t)v[4 * j + 2] * p.z, lc);
      v[4 * j + 3] = red64_2q((uint64_t)v[4 * j + 3] * p.w, lc);
    }
    pass32<true>(v, tgi, T, lt, q, two_q);
    sts_row(srow, v);
  }
  __syncthreads();
  uint32_t* o = out + row * N;
  MaskStore epi{o, h == 0 ? V : nullptr, lc};  // c0 += Delta * encode(v)
  // the prepared 2r carries N^-1, so the transform skips that scaling
  inv_pass<LOGN, T, R1, R2, false, decltype(epi), false>(s, fi, lc, lt, epi);
  __syncthreads();
  inv_pass<LOGN, T, 0, R1, true, decltype(epi), false>(s, fi, lc, lt, epi);
}

// Round 2: out = X - Y, c0 += Delta_l * const.  One thread per 4 coefficients
// of a ciphertext, all limbs and both components.
__global__ void k_x2x_round2(const uint32_t* __restrict__ prep, const uint32_t* X, const uint32_t* Y,
                             uint32_t* out, int n, int N, CtxConst cc) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int N4 = N / 4, L = cc.L;
  if (idx >= (size_t)n * N4) return;
  const size_t c = idx / N4, u4 = idx % N4;
  const uint4 k4 = __ldg(reinterpret_cast<const uint4*>(prep + ((size_t)c * (L + 2) + L + 1) * N) + u4);
  for (int l = 0; l < L; ++l) {
    const LimbConst lc = cc.limb[l];
    const uint32_t q = lc.q, two_q = lc.two_q;
    for (int h = 0; h < 2; ++h) {
      const size_t off = (((size_t)c * 2 + h) * L + l) * N4 + u4;
      const uint4 x = __ldcs(reinterpret_cast<const uint4*>(X) + off);
      const uint4 y = __ldcs(reinterpret_cast<const uint4*>(Y) + off);
      uint4 z;
      z.x = x.x + q - y.x;  // (0, 2q)
      z.y = x.y + q - y.y;
      z.z = x.z + q - y.z;
      z.w = x.w + q - y.w;
      if (h == 0) {
        z.x = csub(z.x + csub(shoup_mul(k4.x, lc.delta, lc.delta_sh, q), q), two_q);  // [0, 2q)
        z.y = csub(z.y + csub(shoup_mul(k4.y, lc.delta, lc.delta_sh, q), q), two_q);
        z.z = csub(z.z + csub(shoup_mul(k4.z, lc.delta, lc.delta_sh, q), q), two_q);
        z.w = csub(z.w + csub(shoup_mul(k4.w, lc.delta, lc.delta_sh, q), q), two_q);
      }
      z.x = csub(z.x, q);
      z.y = csub(z.y, q);
      z.z = csub(z.z, q);
      z.w = csub(z.w, q);
      __stcs(reinterpret_cast<uint4*>(out) + off, z);
    }
  }
}

// dst[b][ci][u] for the next layer's input ciphertext ci: the value of
// channel j at (yy, xx) of the previous layer's output, read from that
// layer's output layout (channel j, band yy / Rout, coefficient
// (s*(yy % Rout))*Wp + s*xx), or 0 at padding and unused coefficients.
__global__ void k_repack(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, GeomDims pv,
                         GeomDims nx, int B, int N) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)B * nx.n_in * N) return;
  const int u = (int)(idx % N);
  const int ci = (int)((idx / N) % nx.n_in);
  const int b = (int)(idx / ((size_t)N * nx.n_in));
  uint32_t val = 0;
  const int band = ci / nx.G, gg = ci % nx.G, jj = u / nx.P;
  if (jj < nx.c_n) {
    const int j = gg * nx.c_n + jj;
    const int rem = u - jj * nx.P;
    const int yy = band * nx.Rout * nx.s + rem / nx.Wp - nx.pad;
    const int xx = rem % nx.Wp - nx.pad;
    if (j < nx.Cin && yy >= 0 && yy < nx.H && xx >= 0 && xx < nx.W) {
      const int pband = yy / pv.Rout, oyl = yy % pv.Rout;
      val = __ldg(src + ((size_t)b * pv.n_out + (size_t)j * pv.bands + pband) * N + (pv.s * oyl) * pv.Wp +
                  pv.s * xx);
    }
  }
  dst[idx] = val;
}

// --------------------------------------------------------------------------
// Launchers
// --------------------------------------------------------------------------
#define FL_ACT_DISPATCH(logn, CALL)                   \
  switch (logn) {                                     \
    case 11: { constexpr int LG = 11; CALL; break; }  \
    case 12: { constexpr int LG = 12; CALL; break; }  \
    case 13: { constexpr int LG = 13; CALL; break; }  \
    case 14: { constexpr int LG = 14; CALL; break; }  \
    default: return cudaErrorInvalidValue;            \
  }

template <int LOGN>
static cudaError_t act_setup() {
  constexpr int SW = Geo<LOGN>::SMEM_WORDS;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_batch_decode<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SW * 4))) return e;
  if ((e = cudaFuncSetAttribute(k_batch_encode<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SW * 4))) return e;
  if ((e = cudaFuncSetAttribute(k_x2x_round1<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * SW * 4)))
    return e;
  return cudaFuncSetAttribute(k_x2x_round1<LOGN>, cudaFuncAttributePreferredSharedMemoryCarveout, 60);
}

cudaError_t launch_act_setup(int logn) { FL_ACT_DISPATCH(logn, return act_setup<LG>()); }

cudaError_t launch_batch_decode(int logn, int n, const uint32_t* m, uint32_t* slots, const uint32_t* tw_t,
                                const LimbConst& tc, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int N = 1 << logn;
  const size_t smem = (size_t)Geo<11>::SMEM_WORDS * 4 << (logn - 11);
  FL_ACT_DISPATCH(logn, (k_batch_decode<LG><<<n, N / 32, smem, st>>>(m, slots, tw_t, tc)));
  return cudaGetLastError();
}

cudaError_t launch_batch_encode(int logn, int n, const uint32_t* slots, uint32_t scale, uint32_t* dst,
                                long long dst_stride, int lift_L, const uint32_t* tw_t, const LimbConst& tc,
                                const CtxConst& cc, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int N = 1 << logn;
  const size_t smem = (size_t)Geo<11>::SMEM_WORDS * 4 << (logn - 11);
  FL_ACT_DISPATCH(logn, (k_batch_encode<LG><<<n, N / 32, smem, st>>>(slots, scale, dst, dst_stride, lift_L, tw_t,
                                                                      tc, cc)));
  return cudaGetLastError();
}

cudaError_t launch_x2x_const(const uint32_t* r, const uint32_t* v, uint32_t* dst, long long dst_stride, int n, int N,
                             const LimbConst& tc, cudaStream_t st) {
  const size_t total = (size_t)n * N;
  if (total == 0) return cudaSuccess;
  k_x2x_const<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(r, v, dst, dst_stride, n, N, tc);
  return cudaGetLastError();
}

cudaError_t launch_x2x_round1(int logn, int n, const uint32_t* prep, const uint32_t* ct, uint32_t* out,
                              const uint32_t* tw, const CtxConst& cc, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int N = 1 << logn;
  const size_t smem = (size_t)2 * Geo<11>::SMEM_WORDS * 4 << (logn - 11);
  dim3 grid(n, cc.L);
  FL_ACT_DISPATCH(logn, (k_x2x_round1<LG><<<grid, N / 16, smem, st>>>(prep, ct, out, tw, cc)));
  return cudaGetLastError();
}

cudaError_t launch_x2x_round2(const uint32_t* prep, const uint32_t* X, const uint32_t* Y, uint32_t* out, int n,
                              int N, const CtxConst& cc, cudaStream_t st) {
  const size_t total = (size_t)n * N / 4;
  if (total == 0) return cudaSuccess;
  k_x2x_round2<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(prep, X, Y, out, n, N, cc);
  return cudaGetLastError();
}

cudaError_t launch_repack(const uint32_t* src, uint32_t* dst, const GeomDims& pv, const GeomDims& nx, int B, int N,
                          cudaStream_t st) {
  const size_t total = (size_t)B * nx.n_in * N;
  if (total == 0) return cudaSuccess;
  k_repack<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(src, dst, pv, nx, B, N);
  return cudaGetLastError();
}

}  // namespace fl
