// CUDA kernels of the HE-convolution path and their launchers.
//
//   k_ntt_fwd     forward negacyclic NTT, out of place (row a3; also keygen,
//                 encryption and weight encoding)
//   k_ntt_inv     inverse NTT, in place (test entry point)
//   k_conv_intt   per-slot contraction mod q_l + inverse NTT + optional mask
//                 epilogue: rows a4, a5, a6 fused, one CTA per output
//                 (image/band, output channel, limb), both components
//   k_pmul_intt   NTT-domain product with the secret key + inverse NTT +
//                 encryption / decryption epilogue (row a1, client side)
//   k_dec_round   exact RNS scale-and-round for decryption
//   k_mask        standalone mask addition (row a6)
//   k_w_scatter   weight polynomial construction (row a2)
#include <cuda_runtime.h>

#include "fl_device.cuh"
#include "fl_launch.h"

namespace fl {


// --------------------------------------------------------------------------
// Forward NTT: one CTA per polynomial row.  Row r of the source starts at
// src + ((r / src_per) * src_stride + r % src_per) * N (same for dst), and
// uses limb (r / limb_div) % L.
// --------------------------------------------------------------------------
template <int LOGN, int R1 = Plan<LOGN>::R1>
__global__ void __launch_bounds__((1 << LOGN) / 32, minb_one_poly<LOGN>())
    k_ntt_fwd(const uint32_t* __restrict__ src, int src_per, int src_stride, uint32_t* dst,
              int dst_per, int dst_stride, int limb_div, const uint32_t* __restrict__ tw,
              CtxConst cc) {
  constexpr int N = 1 << LOGN, T = N / 32;
  extern __shared__ uint32_t sm[];
  const int r = blockIdx.x, tid = threadIdx.x;
  pdl_trigger();  // a dependent conv grid may be scheduled once every CTA is running
  const int l = (r / limb_div) % cc.L;
  const LimbConst lc = cc.limb[l];
  const uint32_t* x = src + ((size_t)(r / src_per) * src_stride + r % src_per) * N;
  uint32_t* y = dst + ((size_t)(r / dst_per) * dst_stride + r % dst_per) * N;
  ntt_forward_to_smem<LOGN, R1>(sm, x, tw + (size_t)l * TwLayout<LOGN>::LIMB_WORDS, lc, tid);
  __syncthreads();
  for (int v = tid; v < N / 4; v += T) {
    const uint4 o = *reinterpret_cast<const uint4*>(sm + pad(4 * v));  // 4 slots of one row
    reinterpret_cast<uint4*>(y)[v] = o;
  }
}

// Inverse NTT in place on contiguous rows [n][L][N].
template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 32, minb_one_poly<LOGN>())
    k_ntt_inv(uint32_t* data, const uint32_t* __restrict__ tw, CtxConst cc) {
  constexpr int N = 1 << LOGN, T = N / 32;
  extern __shared__ uint32_t sm[];
  const int r = blockIdx.x, tid = threadIdx.x;
  const int l = r % cc.L;
  const LimbConst lc = cc.limb[l];
  uint32_t* x = data + (size_t)r * N;
  for (int i = tid; i < N; i += T) sm[pad(i)] = x[i];
  __syncthreads();
  intt_from_smem<LOGN>(sm, tw + (size_t)l * TwLayout<LOGN>::LIMB_WORDS, lc, tid,
                       [&](uint32_t v, int u) { x[u] = csub(v, lc.q); });
}

// --------------------------------------------------------------------------
// Fused contraction + inverse NTT (+ mask).  Grid (B*bands, Cout, L).
//   Y_c[u] = sum_g W[l][i][g][u] * C[b][band*G+g][c][l][u]  mod q_l
// accumulated in 64 bits (products < 2^60; a fold every 16 terms),
// reduced once, inverse-transformed in shared memory and stored with
// streaming stores; c0 optionally gets + Delta_l * r[u].
// --------------------------------------------------------------------------
// One output item: image/band bb, output channel i, limb l.  2 * N/32
// threads, two padded polynomials of shared memory at `sm`.  r may be null
// (no mask).
template <int LOGN, bool WALK>
__device__ __forceinline__ void conv_item(const uint32_t* __restrict__ w_hat, const uint32_t* __restrict__ c_hat,
                                          uint32_t* __restrict__ out, const uint32_t* __restrict__ r,
                                          const ConvDims& cd, int bb, int i, int l, const uint32_t* __restrict__ tw,
                                          const CtxConst& cc, uint32_t* sm) {
  constexpr int N = 1 << LOGN, T = N / 32, T2 = 2 * T, SW = Geo<LOGN>::SMEM_WORDS;
  uint32_t* s0 = sm;
  uint32_t* s1 = sm + SW;
  const int tid = threadIdx.x, L = cc.L;
  const int b = bb / cd.bands, band = bb % cd.bands;
  const LimbConst lc = cc.limb[l];
  const size_t ct_words = (size_t)2 * L * N;
  const uint4* W = reinterpret_cast<const uint4*>(w_hat + ((size_t)l * cd.Cout + i) * cd.G * N);
  const uint32_t* C = c_hat + ((size_t)b * cd.n_in + (size_t)band * cd.G) * ct_words + (size_t)l * N;

  // contraction: each thread owns 4 consecutive slots of both components, so
  // every weight word is loaded once and used twice; the 64-bit accumulators
  // are folded after every 16 terms.  Two forms of the same loop, identical
  // in result: WALK advances the operand pointers by additions, the other
  // indexes from fixed bases.  They differ only in what the compiler makes of
  // them under the 64-register cap; each kernel takes the one that measures
  // faster in it (WALK in k_conv_intt, where it also halves the spills).
  const int G = cd.G;
#pragma unroll 1
  for (int v = tid; v < N / 4; v += T2) {
    uint64_t a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0};
    if (WALK) {
      const size_t ct4 = ct_words / 4;
      const uint4* wp = W + v;
      const uint4* xp0 = reinterpret_cast<const uint4*>(C) + v;
      const uint4* xp1 = reinterpret_cast<const uint4*>(C + (size_t)L * N) + v;
#pragma unroll 1
      for (int g0 = 0; g0 < G; g0 += 16) {
        if (g0) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            a0[j] = red64(a0[j], lc);
            a1[j] = red64(a1[j], lc);
          }
        }
        const int g1 = min(G, g0 + 16);
#pragma unroll 2
        for (int g = g0; g < g1; ++g) {
          const uint4 w = __ldg(wp);
          const uint4 x0 = __ldg(xp0);
          const uint4 x1 = __ldg(xp1);
          wp += N / 4;
          xp0 += ct4;
          xp1 += ct4;
          a0[0] += (uint64_t)w.x * x0.x;
          a0[1] += (uint64_t)w.y * x0.y;
          a0[2] += (uint64_t)w.z * x0.z;
          a0[3] += (uint64_t)w.w * x0.w;
          a1[0] += (uint64_t)w.x * x1.x;
          a1[1] += (uint64_t)w.y * x1.y;
          a1[2] += (uint64_t)w.z * x1.z;
          a1[3] += (uint64_t)w.w * x1.w;
        }
      }
    } else {
#pragma unroll 2
      for (int g = 0; g < cd.G; ++g) {
        const uint4 w = __ldg(W + (size_t)g * (N / 4) + v);
        const uint4 x0 = __ldg(reinterpret_cast<const uint4*>(C + g * ct_words) + v);
        const uint4 x1 = __ldg(reinterpret_cast<const uint4*>(C + g * ct_words + (size_t)L * N) + v);
        a0[0] += (uint64_t)w.x * x0.x;
        a0[1] += (uint64_t)w.y * x0.y;
        a0[2] += (uint64_t)w.z * x0.z;
        a0[3] += (uint64_t)w.w * x0.w;
        a1[0] += (uint64_t)w.x * x1.x;
        a1[1] += (uint64_t)w.y * x1.y;
        a1[2] += (uint64_t)w.z * x1.z;
        a1[3] += (uint64_t)w.w * x1.w;
        if (((g + 1) & 15) == 0 && g + 1 < cd.G) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            a0[j] = red64(a0[j], lc);
            a1[j] = red64(a1[j], lc);
          }
        }
      }
    }
    const int pu = pad(4 * v);  // the 4 slots share one row: one 128-bit store per component
    *reinterpret_cast<uint4*>(s0 + pu) =
        make_uint4(red64_2q(a0[0], lc), red64_2q(a0[1], lc), red64_2q(a0[2], lc), red64_2q(a0[3], lc));
    *reinterpret_cast<uint4*>(s1 + pu) =
        make_uint4(red64_2q(a1[0], lc), red64_2q(a1[1], lc), red64_2q(a1[2], lc), red64_2q(a1[3], lc));
  }
  __syncthreads();

  // inverse NTTs: threads [0, T) transform c0, [T, 2T) transform c1
  const int h = tid >= T, lt = tid - h * T;
  const size_t oct = (size_t)b * cd.n_out + (size_t)i * cd.bands + band;
  uint32_t* op = out + oct * ct_words + (size_t)h * L * N + (size_t)l * N;
  const uint32_t* rr = (r && h == 0) ? r + oct * N : nullptr;
  // the encoded weights carry N^-1, so the transform skips that scaling
  intt_from_smem_unscaled<LOGN>(h ? s1 : s0, tw + (size_t)l * TwLayout<LOGN>::LIMB_WORDS, lc, lt,
                                MaskStore{op, rr, lc});
}

// Fused contraction + inverse NTT (+ mask).  Grid (B*bands, Cout, L).
//   Y_c[u] = sum_g W[l][i][g][u] * C[b][band*G+g][c][l][u]  mod q_l
// accumulated in 64 bits (products < 2^60; a fold every 16 terms),
// reduced once, inverse-transformed in shared memory and stored with
// streaming stores; c0 optionally gets + Delta_l * r[u].
template <int LOGN, bool MASK>
__global__ void __launch_bounds__(2 * ((1 << LOGN) / 32), minb_two_polys<LOGN>())
    k_conv_intt(const uint32_t* __restrict__ w_hat, const uint32_t* __restrict__ c_hat,
                uint32_t* __restrict__ out, const uint32_t* __restrict__ r, ConvDims cd,
                const uint32_t* __restrict__ tw, CtxConst cc) {
  extern __shared__ uint32_t sm[];
  pdl_wait();  // the NTT-domain inputs come from the previous grid in the stream
  conv_item<LOGN, true>(w_hat, c_hat, out, MASK ? r : nullptr, cd, blockIdx.x, blockIdx.y, blockIdx.z, tw, cc, sm);
}

// The same items for every layer of a stack, pulled from one queue by
// persistent CTAs (grid = resident CTAs): no wave tails per layer, no gaps
// between launches.  ctl[0] is the queue head, zeroed before the launch.
template <int LOGN>
__global__ void __launch_bounds__(2 * ((1 << LOGN) / 32), minb_two_polys<LOGN>())
    k_conv_queue(StackArgs a, unsigned long long* __restrict__ ctl, const uint32_t* __restrict__ tw, CtxConst cc) {
  extern __shared__ uint32_t sm[];
  __shared__ long long s_item;
  pdl_wait();  // the NTT-domain inputs (and the zeroed queue head) come from earlier work in the stream
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(ctl, 1ull);
    __syncthreads();  // also: every thread is done with the previous item's shared memory
    const long long it = s_item;
    if (it >= a.n_items) break;
    // claims alternate between the two ends of the item list: even claims walk
    // forward from the first layers, odd claims backward from the last ones,
    // so the CTAs sharing an SM tend to mix contraction-heavy (large G) and
    // transform-heavy (small G) items; each end keeps consecutive items together
    const long long pos = (it & 1) ? a.n_items - 1 - (it >> 1) : (it >> 1);
    const Item x = decode(a, pos);
    const StackLayer& y = a.layer[x.li];
    const ConvDims cd{y.Cout, y.G, y.n_in, y.n_out, y.bands};
    conv_item<LOGN, false>(y.w_hat, y.c_hat, y.out, y.r, cd, x.bb, x.i, x.l, tw, cc, sm);
  }
}

// --------------------------------------------------------------------------
// Client side: NTT-domain product with the secret key + inverse NTT.
// Grid (n, L).  MODE_DEC: xhat = ws row [n][L][N] (NTT of c1); result
// [c0 + c1*s] written back to the same ws row.  MODE_ENC: xhat = c0 slot of
// ct (holds NTT(a)); result c0 = Delta*m - a*s - e written to that slot.
// --------------------------------------------------------------------------
enum { MODE_DEC = 0, MODE_ENC = 1 };

__device__ __forceinline__ uint32_t packed_input(const int32_t* __restrict__ x, const GeomDims& g,
                                                 int b, int ci, int u) {
  // Coefficient u of input ciphertext ci = band*G + gg of image b: channel
  // j = gg*c_n + u/P, padded row band*Rout*s + (u%P)/Wp, padded column (u%P)%Wp.
  const int band = ci / g.G, gg = ci % g.G;
  const int jj = u / g.P;
  if (jj >= g.c_n) return 0;
  const int j = gg * g.c_n + jj;
  if (j >= g.Cin) return 0;
  const int rem = u - jj * g.P;
  const int yy = band * g.Rout * g.s + rem / g.Wp - g.pad;
  const int xx = rem % g.Wp - g.pad;
  if (yy < 0 || yy >= g.H || xx < 0 || xx >= g.W) return 0;
  return (uint32_t)x[(((size_t)b * g.Cin + j) * g.H + yy) * g.W + xx];
}

template <int LOGN, int MODE>
__global__ void __launch_bounds__((1 << LOGN) / 32, minb_one_poly<LOGN>())
    k_pmul_intt(uint32_t* __restrict__ ws, uint32_t* __restrict__ ct,
                const uint32_t* __restrict__ sk, const int32_t* __restrict__ x,
                const int32_t* __restrict__ e, GeomDims gd, const uint32_t* __restrict__ tw,
                CtxConst cc) {
  constexpr int N = 1 << LOGN, T = N / 32;
  extern __shared__ uint32_t sm[];
  const int n = blockIdx.x, l = blockIdx.y, L = cc.L, tid = threadIdx.x;
  const LimbConst lc = cc.limb[l];
  uint32_t* row = MODE == MODE_DEC ? ws + ((size_t)n * L + l) * N : ct + ((size_t)n * 2 * L + l) * N;
  const uint32_t* s = sk + (size_t)l * N;
  for (int i = tid; i < N; i += T) {
    uint64_t p = (uint64_t)row[i] * __ldg(s + i);
    sm[pad(i)] = barrett64(p, lc.q, lc.mu);
  }
  __syncthreads();
  if (MODE == MODE_DEC) {
    const uint32_t* c0 = ct + ((size_t)n * 2 * L + l) * N;
    intt_from_smem<LOGN>(sm, tw + (size_t)l * TwLayout<LOGN>::LIMB_WORDS, lc, tid, [&](uint32_t v, int u) {
      row[u] = csub(csub(v + __ldg(c0 + u), lc.two_q), lc.q);
    });
  } else {
    const int b = n / gd.n_in, ci = n % gd.n_in;
    intt_from_smem<LOGN>(sm, tw + (size_t)l * TwLayout<LOGN>::LIMB_WORDS, lc, tid, [&](uint32_t v, int u) {
      // Delta*m - a*s - e  (v = a*s in [0, 2q))
      uint32_t m = packed_input(x, gd, b, ci, u);
      uint32_t dm = csub(shoup_mul(m, lc.delta, lc.delta_sh, lc.q), lc.q);  // [0, q)
      int32_t ev = __ldg(e + (size_t)n * N + u);
      uint32_t em = ev >= 0 ? (uint32_t)ev : lc.q - (uint32_t)(-ev);  // e mod q, |e| < 2^20
      uint32_t as = csub(v, lc.q);
      uint32_t r = dm + lc.two_q - as - em;  // (0, 3q): dm, as, em all in [0, q)
      row[u] = csub(csub(r, lc.two_q), lc.q);
    });
  }
}

// Exact scale-and-round: x = [c0 + c1 s]_q from its residues x_l.
// y_l = x_l * (q/q_l)^-1 mod q_l, so t*x/q = sum_l y_l*t/q_l - k*t for an
// integer k.  With y_l*t = a_l*q_l + b_l: m = (sum a_l + round(S)) mod t,
// S = sum b_l/q_l = (sum b_l*(q/q_l)) / q, rounded exactly in 128-bit
// integers (q odd, so S is never a half-integer).
__global__ void k_dec_round(const uint32_t* __restrict__ ws, uint32_t* __restrict__ m, int n, int N,
                            DecConst dc) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * N) return;
  const size_t c = idx / N, u = idx % N;
  typedef unsigned __int128 u128;
  u128 num = 0;
  uint64_t asum = 0;
  for (int l = 0; l < dc.L; ++l) {
    const uint32_t q = dc.q[l];
    uint32_t xl = ws[(c * dc.L + l) * N + u];
    uint32_t y = (uint32_t)(((uint64_t)xl * dc.inv[l]) % q);
    uint64_t yt = (uint64_t)y * dc.t;
    uint64_t a = yt / q;
    uint64_t bl = yt - a * q;
    asum += a;
    num += (u128)bl * (((u128)dc.Qhi[l] << 64) | dc.Qlo[l]);
  }
  const u128 Q = ((u128)dc.qhi << 64) | dc.qlo;
  const u128 two = num << 1;
  uint32_t rnd = 0;
  for (int j = 0; j < dc.L; ++j)
    if (two >= (u128)(2 * j + 1) * Q) ++rnd;
  m[idx] = (uint32_t)((asum + rnd) % dc.t);
}

// Noise of decryption (Appendix A): v = [c0 + c1 s - Delta m]_q, centred, for
// every coefficient; ws holds the phase residues [c0 + c1 s]_{q_l} [n][L][N].
// The residues of v are lifted to Z_q by CRT in 128 bits; the largest |v|
// (as a double: exact below 2^53) goes to *out through an atomic maximum on
// its bit pattern (non-negative doubles order like their bits).
__global__ void k_noise(const uint32_t* __restrict__ ws, const uint32_t* __restrict__ m, int n, int N,
                        DecConst dc, CtxConst cc, unsigned long long* out) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * N) return;
  const size_t c = idx / N, u = idx % N;
  typedef unsigned __int128 u128;
  const u128 Q = ((u128)dc.qhi << 64) | dc.qlo;
  const uint64_t msg = m[idx];
  u128 V = 0;
  for (int l = 0; l < dc.L; ++l) {
    const uint64_t q = dc.q[l];
    const uint64_t x = ws[(c * dc.L + l) * N + u];
    const uint64_t dm = (cc.limb[l].delta * (msg % q)) % q;
    const uint64_t v = (x + q - dm) % q;
    const uint64_t y = (v * dc.inv[l]) % q;
    V += (u128)y * (((u128)dc.Qhi[l] << 64) | dc.Qlo[l]);
  }
  while (V >= Q) V -= Q;
  const u128 a = (V << 1) > Q ? Q - V : V;  // |centred v|
  const double d = (double)(uint64_t)(a >> 64) * 18446744073709551616.0 + (double)(uint64_t)a;
  atomicMax(out, (unsigned long long)__double_as_longlong(d));
}

__global__ void k_extract(const uint32_t* __restrict__ m, int32_t* __restrict__ y, GeomDims g, int B,
                          int N) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)B * g.Cout * g.Ho * g.Wo;
  if (idx >= total) return;
  size_t r = idx;
  const int ox = r % g.Wo; r /= g.Wo;
  const int oy = r % g.Ho; r /= g.Ho;
  const int i = r % g.Cout;
  const int b = (int)(r / g.Cout);
  const int band = oy / g.Rout, oyl = oy % g.Rout;
  const uint32_t* poly = m + ((size_t)b * g.n_out + (size_t)i * g.bands + band) * N;
  y[idx] = (int32_t)poly[(g.s * oyl) * g.Wp + g.s * ox];
}

// c0 <- c0 + Delta_l * r  for cts [n][2][L][N]; one thread per 4 coefficients.
__global__ void k_mask(uint32_t* __restrict__ ct, const uint32_t* __restrict__ r, int n, int N,
                       CtxConst cc) {
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int L = cc.L;
  const size_t per_ct = (size_t)L * N / 4;
  if (v >= (size_t)n * per_ct) return;
  const size_t c = v / per_ct, rem = v % per_ct;
  const int l = (int)(rem / (N / 4));
  const size_t u4 = rem % (N / 4);
  const LimbConst lc = cc.limb[l];
  uint4* p = reinterpret_cast<uint4*>(ct + (c * 2 * L + l) * N) + u4;
  const uint4 rv = __ldg(reinterpret_cast<const uint4*>(r + c * N) + u4);
  uint4 x = *p;
  x.x = csub(csub(x.x + shoup_mul(rv.x, lc.delta, lc.delta_sh, lc.q), lc.two_q), lc.q);
  x.y = csub(csub(x.y + shoup_mul(rv.y, lc.delta, lc.delta_sh, lc.q), lc.two_q), lc.q);
  x.z = csub(csub(x.z + shoup_mul(rv.z, lc.delta, lc.delta_sh, lc.q), lc.two_q), lc.q);
  x.w = csub(csub(x.w + shoup_mul(rv.w, lc.delta, lc.delta_sh, lc.q), lc.two_q), lc.q);
  *p = x;
}

// Online encryption (Algorithm 2): c0 <- enc0.c0 + Delta*m, c1 <- enc0.c1.
__global__ void k_enc_online(const uint32_t* __restrict__ enc0, uint32_t* __restrict__ ct,
                             const int32_t* __restrict__ x, GeomDims gd, int n, int N,
                             CtxConst cc) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int L = cc.L;
  if (idx >= (size_t)n * 2 * L * N) return;
  const int u = idx % N;
  const int l = (idx / N) % L;
  const int comp = (idx / ((size_t)L * N)) % 2;
  const int c = (int)(idx / ((size_t)2 * L * N));
  uint32_t v = enc0[idx];
  if (comp == 0) {
    const LimbConst lc = cc.limb[l];
    const uint32_t m = packed_input(x, gd, c / gd.n_in, c % gd.n_in, u);
    v = csub(csub(v + shoup_mul(m, lc.delta, lc.delta_sh, lc.q), lc.two_q), lc.q);
  }
  ct[idx] = v;
}

// Weight polynomial construction: one thread per (l, i, j, ky, kx).  Tap
// w[i][j][ky][kx] (times N^-1 mod q_l) lands on x^-e, e = ky*Wp + kx + (j mod c_n)*P, of W_{i,g},
// g = j / c_n; x^-e = -x^(N-e) for e > 0.  Exponents within one (i, g) are
// distinct, so every coefficient is written at most once (buffer pre-zeroed).
__global__ void k_w_scatter(const int8_t* __restrict__ w, uint32_t* __restrict__ w_hat, GeomDims g,
                            int N, CtxConst cc) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per_l = (size_t)g.Cout * g.Cin * g.k * g.k;
  if (idx >= per_l * cc.L) return;
  const int l = (int)(idx / per_l);
  size_t r = idx % per_l;
  const int kx = r % g.k; r /= g.k;
  const int ky = r % g.k; r /= g.k;
  const int j = r % g.Cin;
  const int i = (int)(r / g.Cin);
  const int gg = j / g.c_n, jj = j % g.c_n;
  const int e = ky * g.Wp + kx + jj * g.P;
  const int wv = w[(((size_t)i * g.Cin + j) * g.k + ky) * g.k + kx];
  const uint32_t q = cc.limb[l].q;
  int pos;
  uint32_t val;
  if (e == 0) {
    pos = 0;
    val = wv >= 0 ? (uint32_t)wv : q - (uint32_t)(-wv);
  } else {
    pos = N - e;
    val = wv > 0 ? q - (uint32_t)wv : (uint32_t)(-wv);
  }
  // times N^-1, which the hot path's inverse NTT then leaves out
  const LimbConst& lc = cc.limb[l];
  val = csub(shoup_mul(val, lc.n_inv, lc.n_inv_sh, q), q);
  w_hat[(((size_t)l * g.Cout + i) * g.G + gg) * N + pos] = val;
}

// Secret key expansion: s (ternary int8) -> residues [L][N].
__global__ void k_sk_expand(const int8_t* __restrict__ s, uint32_t* __restrict__ out, int N,
                            CtxConst cc) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)cc.L * N) return;
  const int l = (int)(idx / N);
  const int sv = s[idx % N];
  const uint32_t q = cc.limb[l].q;
  out[idx] = sv >= 0 ? (uint32_t)sv : q - (uint32_t)(-sv);
}

// --------------------------------------------------------------------------
// Launchers
// --------------------------------------------------------------------------
static inline int blocks_for(size_t n, int t) { return (int)((n + t - 1) / t); }

template <int LOGN>
static cudaError_t setup_smem() {
  constexpr int SW = Geo<LOGN>::SMEM_WORDS;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_ntt_fwd<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SW * 4))) return e;
  for (int r1 = 3; r1 <= 5; ++r1) {  // the other instantiated pass plans
    if (r1 == Plan<LOGN>::R1 || !plan_available(LOGN, r1)) continue;
    FL_PLAN_DISPATCH(LOGN, r1, (e = cudaFuncSetAttribute(k_ntt_fwd<LG, R1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SW * 4)));
    if (e) return e;
  }
  if ((e = cudaFuncSetAttribute(k_ntt_inv<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SW * 4))) return e;
  if ((e = cudaFuncSetAttribute(k_conv_intt<LOGN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * SW * 4))) return e;
  if ((e = cudaFuncSetAttribute(k_conv_intt<LOGN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * SW * 4))) return e;
  if ((e = cudaFuncSetAttribute(k_conv_queue<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * SW * 4))) return e;
  if ((e = cudaFuncSetAttribute(k_conv_queue<LOGN>, cudaFuncAttributePreferredSharedMemoryCarveout, 60))) return e;
  if ((e = cudaFuncSetAttribute(k_pmul_intt<LOGN, MODE_DEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, SW * 4))) return e;
  if ((e = cudaFuncSetAttribute(k_pmul_intt<LOGN, MODE_ENC>, cudaFuncAttributeMaxDynamicSharedMemorySize, SW * 4))) return e;
  // every kernel here is sized for ~135 KiB of shared memory per SM; the
  // rest of the unified L1 is left to the twiddle tables
  const int carve = 60;
  if ((e = cudaFuncSetAttribute(k_conv_intt<LOGN, false>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
  if ((e = cudaFuncSetAttribute(k_conv_intt<LOGN, true>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
  if ((e = cudaFuncSetAttribute(k_ntt_fwd<LOGN>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
  return cudaSuccess;
}

size_t twiddle_limb_words(int logn) { return (size_t)TwLayout<11>::LIMB_WORDS << (logn - 11); }

cudaError_t launch_setup(int logn) {
  switch (logn) {
    case 11: return setup_smem<11>();
    case 12: return setup_smem<12>();
    case 13: return setup_smem<13>();
    case 14: return setup_smem<14>();
  }
  return cudaErrorInvalidValue;
}

#define FL_DISPATCH(logn, CALL)            \
  switch (logn) {                          \
    case 11: { constexpr int LG = 11; CALL; break; } \
    case 12: { constexpr int LG = 12; CALL; break; } \
    case 13: { constexpr int LG = 13; CALL; break; } \
    case 14: { constexpr int LG = 14; CALL; break; } \
    default: return cudaErrorInvalidValue;  \
  }

cudaError_t launch_ntt_fwd(int logn, int rows, const uint32_t* src, int src_per, int src_stride,
                           uint32_t* dst, int dst_per, int dst_stride, int limb_div,
                           const uint32_t* tw, const CtxConst& cc, cudaStream_t st, int r1) {
  if (rows == 0) return cudaSuccess;
  const int N = 1 << logn;
  const size_t smem = (size_t)padded_words(N) * 4;
  FL_PLAN_DISPATCH(logn, r1, (k_ntt_fwd<LG, R1><<<rows, N / 32, smem, st>>>(src, src_per, src_stride, dst, dst_per,
                                                                            dst_stride, limb_div, tw, cc)));
  return cudaGetLastError();
}

cudaError_t launch_ntt_inv(int logn, int rows, uint32_t* data, const uint32_t* tw, const CtxConst& cc,
                           cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  const int N = 1 << logn;
  const size_t smem = (size_t)padded_words(N) * 4;
  FL_DISPATCH(logn, (k_ntt_inv<LG><<<rows, N / 32, smem, st>>>(data, tw, cc)));
  return cudaGetLastError();
}

template <int LOGN, bool MASK>
static cudaError_t conv_intt_launch(dim3 grid, size_t smem, bool pdl, const uint32_t* w_hat, const uint32_t* c_hat,
                                    uint32_t* out, const uint32_t* r, const ConvDims& cd, const uint32_t* tw,
                                    const CtxConst& cc, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(2 * (1 << LOGN) / 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_conv_intt<LOGN, MASK>, w_hat, c_hat, out, r, cd, tw, cc);
}

// pdl: the previous operation in `st` is the forward NTT of these inputs
// (programmatic dependent launch; the kernel waits for it before reading).
cudaError_t launch_conv_intt(int logn, int B, const ConvDims& cd, const uint32_t* w_hat,
                             const uint32_t* c_hat, uint32_t* out, const uint32_t* r,
                             const uint32_t* tw, const CtxConst& cc, cudaStream_t st, bool pdl) {
  const int N = 1 << logn;
  const size_t smem = (size_t)2 * padded_words(N) * 4;
  dim3 grid(B * cd.bands, cd.Cout, cc.L);
  cudaError_t e = cudaSuccess;
  if (r) {
    FL_DISPATCH(logn, (e = conv_intt_launch<LG, true>(grid, smem, pdl, w_hat, c_hat, out, r, cd, tw, cc, st)));
  } else {
    FL_DISPATCH(logn, (e = conv_intt_launch<LG, false>(grid, smem, pdl, w_hat, c_hat, out, r, cd, tw, cc, st)));
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int LOGN>
static cudaError_t conv_queue_launch(const StackArgs& a, unsigned long long* ctl, const uint32_t* tw,
                                     const CtxConst& cc, int sms, cudaStream_t st) {
  const size_t smem = (size_t)2 * Geo<LOGN>::SMEM_WORDS * 4;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_queue<LOGN>, 2 * (1 << LOGN) / 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const long long slots = (long long)sms * per_sm;
  const int grid = (int)(a.n_items < slots ? a.n_items : slots);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(2 * (1 << LOGN) / 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_conv_queue<LOGN>, a, ctl, tw, cc);
}

// The queue head ctl[0] must be zero when the kernel starts: the caller
// zeroes it earlier in `st` (before the stack's input NTT, so that the kernel
// can follow the NTT as a programmatic dependent launch).
cudaError_t launch_conv_queue(int logn, const StackArgs& a, unsigned long long* ctl, const uint32_t* tw,
                              const CtxConst& cc, int sms, cudaStream_t st) {
  if (a.n_items == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  FL_DISPATCH(logn, e = conv_queue_launch<LG>(a, ctl, tw, cc, sms, st));
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_pmul_intt(int logn, int mode, int n, uint32_t* ws, uint32_t* ct, const uint32_t* sk,
                             const int32_t* x, const int32_t* e, const GeomDims& gd,
                             const uint32_t* tw, const CtxConst& cc, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int N = 1 << logn;
  const size_t smem = (size_t)padded_words(N) * 4;
  dim3 grid(n, cc.L);
  if (mode == MODE_DEC) {
    FL_DISPATCH(logn, (k_pmul_intt<LG, MODE_DEC><<<grid, N / 32, smem, st>>>(ws, ct, sk, x, e, gd, tw, cc)));
  } else {
    FL_DISPATCH(logn, (k_pmul_intt<LG, MODE_ENC><<<grid, N / 32, smem, st>>>(ws, ct, sk, x, e, gd, tw, cc)));
  }
  return cudaGetLastError();
}

cudaError_t launch_dec_round(const uint32_t* ws, uint32_t* m, int n, int N, const DecConst& dc,
                             cudaStream_t st) {
  const size_t total = (size_t)n * N;
  if (total == 0) return cudaSuccess;
  k_dec_round<<<blocks_for(total, 256), 256, 0, st>>>(ws, m, n, N, dc);
  return cudaGetLastError();
}

cudaError_t launch_noise(const uint32_t* ws, const uint32_t* m, int n, int N, const DecConst& dc, const CtxConst& cc,
                         unsigned long long* out, cudaStream_t st) {
  const size_t total = (size_t)n * N;
  if (total == 0) return cudaSuccess;
  k_noise<<<blocks_for(total, 256), 256, 0, st>>>(ws, m, n, N, dc, cc, out);
  return cudaGetLastError();
}

cudaError_t launch_extract(const uint32_t* m, int32_t* y, const GeomDims& g, int B, int N,
                           cudaStream_t st) {
  const size_t total = (size_t)B * g.Cout * g.Ho * g.Wo;
  if (total == 0) return cudaSuccess;
  k_extract<<<blocks_for(total, 256), 256, 0, st>>>(m, y, g, B, N);
  return cudaGetLastError();
}

cudaError_t launch_mask(uint32_t* ct, const uint32_t* r, int n, int N, const CtxConst& cc,
                        cudaStream_t st) {
  const size_t total = (size_t)n * cc.L * N / 4;
  if (total == 0) return cudaSuccess;
  k_mask<<<blocks_for(total, 256), 256, 0, st>>>(ct, r, n, N, cc);
  return cudaGetLastError();
}

cudaError_t launch_enc_online(const uint32_t* enc0, uint32_t* ct, const int32_t* x, const GeomDims& gd,
                              int n, int N, const CtxConst& cc, cudaStream_t st) {
  const size_t total = (size_t)n * 2 * cc.L * N;
  if (total == 0) return cudaSuccess;
  k_enc_online<<<blocks_for(total, 256), 256, 0, st>>>(enc0, ct, x, gd, n, N, cc);
  return cudaGetLastError();
}

cudaError_t launch_w_scatter(const int8_t* w, uint32_t* w_hat, const GeomDims& g, int N,
                             const CtxConst& cc, cudaStream_t st) {
  const size_t total = (size_t)g.Cout * g.Cin * g.k * g.k * cc.L;
  if (total == 0) return cudaSuccess;
  k_w_scatter<<<blocks_for(total, 256), 256, 0, st>>>(w, w_hat, g, N, cc);
  return cudaGetLastError();
}

cudaError_t launch_sk_expand(const int8_t* s, uint32_t* out, int N, const CtxConst& cc,
                             cudaStream_t st) {
  k_sk_expand<<<blocks_for((size_t)cc.L * N, 256), 256, 0, st>>>(s, out, N, cc);
  return cudaGetLastError();
}

}  // namespace fl
