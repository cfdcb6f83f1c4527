// Device-side building blocks of the GB300 HE-convolution path: modular
// arithmetic for 30-bit NTT-friendly primes and the shared-memory negacyclic
// NTT / inverse NTT passes.
//
// Arithmetic (published methods, written from their definitions):
//  * Shoup multiplication by a fixed w < q with w' = floor(w * 2^32 / q):
//    x*w - umulhi(x, w')*q lies in [0, 2q) for every 32-bit x.
//  * Harvey's lazy butterflies (D. Harvey, "Faster arithmetic for
//    number-theoretic transforms", 2014): forward Cooley-Tukey values live in
//    [0, 4q), inverse Gentleman-Sande values in [0, 2q).  q < 2^30 keeps 4q
//    inside 32 bits.
//  * Barrett reduction of a 64-bit accumulator with mu = floor(2^64 / q):
//    the quotient estimate is at most one short, so one conditional
//    subtraction finishes it.
//
// NTT: negacyclic transform over Z_q[x]/(x^N+1) with psi a primitive 2N-th
// root of unity.  Forward = Cooley-Tukey, natural order in, bit-reversed order
// out, twiddles psi^brev(i); inverse = Gentleman-Sande, bit-reversed in,
// natural out, twiddles psi^-brev(i), N^-1 folded into the last stage
// (the merged negacyclic form of Longa and Naehrig, 2016).  The transform
// runs in three passes over shared memory; each thread keeps one radix-2^R
// group in registers for R consecutive stages.  The last forward / first
// inverse pass is radix-32 on 32 consecutive coefficients.  Shared memory is
// padded by one word per 32 so every pass is free of bank conflicts.
#pragma once
#include <cstdint>

#define FL_MAX_L 4

namespace fl {

struct LimbConst {
  uint32_t q, two_q;
  uint32_t n_inv, n_inv_sh;    // N^-1 mod q and its Shoup companion
  uint32_t last_w, last_w_sh;  // psi^-(N/2) * N^-1: last inverse stage
  uint32_t delta, delta_sh;    // Delta mod q (Delta = floor(Q / t))
  uint64_t mu;                 // floor(2^64 / q)
};

struct CtxConst {
  LimbConst limb[FL_MAX_L];
  int L;
  uint32_t t;
};

// Twiddle tables: [L][4][N] words: psi^brev, Shoup(psi^brev),
// psi^-brev, Shoup(psi^-brev).
enum { TW_FWD = 0, TW_FWD_SH = 1, TW_INV = 2, TW_INV_SH = 3 };

__device__ __forceinline__ uint32_t shoup_mul(uint32_t x, uint32_t w, uint32_t wsh, uint32_t q) {
  return x * w - __umulhi(x, wsh) * q;  // [0, 2q)
}

__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t m) { return x >= m ? x - m : x; }

__device__ __forceinline__ uint32_t barrett64(uint64_t x, uint32_t q, uint64_t mu) {
  uint64_t qh = __umul64hi(x, mu);
  uint32_t r = (uint32_t)x - (uint32_t)qh * q;  // true remainder < 2q, exact mod 2^32
  return csub(r, q);
}

__device__ __forceinline__ void ct_bfly(uint32_t& X, uint32_t& Y, uint32_t w, uint32_t wsh,
                                        uint32_t q, uint32_t two_q) {
  uint32_t x = csub(X, two_q);
  uint32_t t = shoup_mul(Y, w, wsh, q);
  X = x + t;
  Y = x - t + two_q;
}

__device__ __forceinline__ void gs_bfly(uint32_t& X, uint32_t& Y, uint32_t w, uint32_t wsh,
                                        uint32_t q, uint32_t two_q) {
  uint32_t x = csub(X + Y, two_q);
  uint32_t y = shoup_mul(X - Y + two_q, w, wsh, q);
  X = x;
  Y = y;
}

__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

template <int LOGN> struct Plan;
template <> struct Plan<11> { static constexpr int R1 = 3, R2 = 3; };
template <> struct Plan<12> { static constexpr int R1 = 4, R2 = 3; };
template <> struct Plan<13> { static constexpr int R1 = 4, R2 = 4; };
template <> struct Plan<14> { static constexpr int R1 = 5, R2 = 4; };

template <int LOGN> struct Geo {
  static constexpr int N = 1 << LOGN;
  static constexpr int T = N / 32;                 // threads per polynomial
  static constexpr int SMEM_WORDS = N + N / 32;    // one padded polynomial
};

// Element k of group gid in the pass over stages [S0, S0+R).
template <int LOGN, int S0, int R>
__device__ __forceinline__ void group_of(int gid, int& blk, int& base) {
  constexpr int N = 1 << LOGN;
  constexpr int TL = N >> (S0 + R);
  static_assert(TL == 1 || TL >= 32, "pass plan keeps passes bank-conflict free");
  if (TL >= 32) {
    blk = gid / TL;
    base = blk * (N >> S0) + gid % TL;
  } else {
    blk = gid;
    base = blk * (N >> S0);
  }
}

// Forward pass over stages [S0, S0+R).  SRC_G: read the group from global
// memory `g` (natural order) instead of shared memory.
template <int LOGN, int S0, int R, bool SRC_G>
__device__ __forceinline__ void fwd_pass(uint32_t* __restrict__ s, const uint32_t* __restrict__ g,
                                         const uint32_t* __restrict__ tw,
                                         const uint32_t* __restrict__ twsh, uint32_t q,
                                         uint32_t two_q, int tid) {
  constexpr int N = 1 << LOGN, T = N / 32, TL = N >> (S0 + R), RAD = 1 << R;
  constexpr int NG = 32 / RAD;
#pragma unroll
  for (int gi = 0; gi < NG; ++gi) {
    int blk, base;
    group_of<LOGN, S0, R>(tid + gi * T, blk, base);
    uint32_t v[RAD];
#pragma unroll
    for (int k = 0; k < RAD; ++k) v[k] = SRC_G ? __ldg(g + base + k * TL) : s[pad(base + k * TL)];
#pragma unroll
    for (int d = 0; d < R; ++d) {
      const int half = RAD >> (d + 1);
#pragma unroll
      for (int k = 0; k < RAD; ++k) {
        if (k & half) continue;
        int ti = (1 << (S0 + d)) + (blk << d) + (k >> (R - d));
        ct_bfly(v[k], v[k + half], __ldg(tw + ti), __ldg(twsh + ti), q, two_q);
      }
    }
#pragma unroll
    for (int k = 0; k < RAD; ++k) s[pad(base + k * TL)] = v[k];
  }
}

// Inverse pass over stages [S0, S0+R), applied from the highest stage down.
// LAST: this pass contains stage 0; fold N^-1 into it and hand each final
// value (in [0, 2q)) with its coefficient index to `epi`, which stores it.
template <int LOGN, int S0, int R, bool LAST, class Epi>
__device__ __forceinline__ void inv_pass(uint32_t* __restrict__ s, const uint32_t* __restrict__ tw,
                                         const uint32_t* __restrict__ twsh, const LimbConst& lc,
                                         int tid, Epi epi) {
  constexpr int N = 1 << LOGN, T = N / 32, TL = N >> (S0 + R), RAD = 1 << R;
  constexpr int NG = 32 / RAD;
  const uint32_t q = lc.q, two_q = lc.two_q;
#pragma unroll
  for (int gi = 0; gi < NG; ++gi) {
    int blk, base;
    group_of<LOGN, S0, R>(tid + gi * T, blk, base);
    uint32_t v[RAD];
#pragma unroll
    for (int k = 0; k < RAD; ++k) v[k] = s[pad(base + k * TL)];
#pragma unroll
    for (int d = R - 1; d >= 0; --d) {
      const int half = RAD >> (d + 1);
#pragma unroll
      for (int k = 0; k < RAD; ++k) {
        if (k & half) continue;
        if (LAST && S0 + d == 0) {
          uint32_t X = v[k], Y = v[k + half];
          v[k] = shoup_mul(X + Y, lc.n_inv, lc.n_inv_sh, q);
          v[k + half] = shoup_mul(X - Y + two_q, lc.last_w, lc.last_w_sh, q);
        } else {
          int ti = (1 << (S0 + d)) + (blk << d) + (k >> (R - d));
          gs_bfly(v[k], v[k + half], __ldg(tw + ti), __ldg(twsh + ti), q, two_q);
        }
      }
    }
    if (LAST) {
#pragma unroll
      for (int k = 0; k < RAD; ++k) epi(v[k], base + k * TL);
    } else {
#pragma unroll
      for (int k = 0; k < RAD; ++k) s[pad(base + k * TL)] = v[k];
    }
  }
}

// Full forward NTT of one polynomial: global `src` -> shared `s`, result in
// shared memory reduced to [0, q).  Caller syncs before reading `s`.
template <int LOGN>
__device__ __forceinline__ void ntt_forward_to_smem(uint32_t* s, const uint32_t* __restrict__ src,
                                                    const uint32_t* __restrict__ tw_l,
                                                    const LimbConst& lc, int tid) {
  constexpr int N = 1 << LOGN, R1 = Plan<LOGN>::R1, R2 = Plan<LOGN>::R2;
  const uint32_t* f = tw_l + TW_FWD * N;
  const uint32_t* fs = tw_l + TW_FWD_SH * N;
  fwd_pass<LOGN, 0, R1, true>(s, src, f, fs, lc.q, lc.two_q, tid);
  __syncthreads();
  fwd_pass<LOGN, R1, R2, false>(s, nullptr, f, fs, lc.q, lc.two_q, tid);
  __syncthreads();
  fwd_pass<LOGN, R1 + R2, 5, false>(s, nullptr, f, fs, lc.q, lc.two_q, tid);
  __syncthreads();
  // reduce [0, 4q) -> [0, q)
  for (int i = tid; i < N; i += N / 32) {
    uint32_t x = s[pad(i)];
    s[pad(i)] = csub(csub(x, lc.two_q), lc.q);
  }
}

// Full inverse NTT of the polynomial in shared memory `s` (values in
// [0, 2q)); every output coefficient goes through `epi(value_in_[0,2q), u)`.
template <int LOGN, class Epi>
__device__ __forceinline__ void intt_from_smem(uint32_t* s, const uint32_t* __restrict__ tw_l,
                                               const LimbConst& lc, int tid, Epi epi) {
  constexpr int N = 1 << LOGN, R1 = Plan<LOGN>::R1, R2 = Plan<LOGN>::R2;
  const uint32_t* f = tw_l + TW_INV * N;
  const uint32_t* fs = tw_l + TW_INV_SH * N;
  inv_pass<LOGN, R1 + R2, 5, false>(s, f, fs, lc, tid, epi);
  __syncthreads();
  inv_pass<LOGN, R1, R2, false>(s, f, fs, lc, tid, epi);
  __syncthreads();
  inv_pass<LOGN, 0, R1, true>(s, f, fs, lc, tid, epi);
}

}  // namespace fl
