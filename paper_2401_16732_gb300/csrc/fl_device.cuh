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
// inverse pass is radix-32 on 32 consecutive coefficients.  In shared memory
// each row of 32 coefficients is padded to 36 words (144 bytes): one row
// covers the 32 banks, and the rows of 8 consecutive threads start in 8
// different bank quads, so both the row-strided passes and the per-thread
// 128-bit accesses of the radix-32 pass are free of bank conflicts.  In the
// row-strided passes a thread takes 32/2^R adjacent columns, loaded and
// stored as one 64- or 128-bit access, sharing one set of twiddles.
#pragma once
#include <cstdint>
#include <type_traits>
#include <utility>

#define FL_MAX_L 4

namespace fl {

struct LimbConst {
  uint32_t q, two_q;
  uint32_t n_inv, n_inv_sh;    // N^-1 mod q and its Shoup companion
  uint32_t last_w, last_w_sh;  // psi^-(N/2) * N^-1: last inverse stage
  uint32_t delta, delta_sh;    // Delta mod q (Delta = floor(Q / t))
  uint64_t mu;                 // floor(2^64 / q)
  uint32_t r32, r32_sh;        // 2^32 mod q and its Shoup companion
};

struct CtxConst {
  LimbConst limb[FL_MAX_L];
  int L;
  uint32_t t;
};

// Twiddle tables, per limb (all in one device allocation):
//  * uint2 [2][N]: (psi^brev(i), Shoup companion) for the forward transform,
//    then (psi^-brev(i), companion) for the inverse; one 8-byte load fetches a
//    twiddle with its companion.  Used by the passes whose twiddles are the
//    same for a whole warp (broadcast loads).
//  * uint4 [2][16][N/32]: the twiddles of the radix-32 pass on contiguous
//    groups (forward last pass, inverse first pass), where every thread needs
//    31 twiddles of its own.  Entry [dir][p][blk] holds the twiddles the
//    thread of group blk consumes in order 2p and 2p+1, so a warp reads 512
//    contiguous bytes per load instead of 31 scattered pairs.
enum { TW_FWD = 0, TW_INV = 1 };
template <int LOGN> struct TwLayout {
  static constexpr int N = 1 << LOGN;
  static constexpr int PAIRS_WORDS = 2 * N * 2;             // uint2 [2][N] in 32-bit words
  static constexpr int GROUPED_WORDS = 2 * 16 * (N / 32) * 4;  // uint4 [2][16][N/32]
  static constexpr int LIMB_WORDS = PAIRS_WORDS + GROUPED_WORDS;
};

__device__ __forceinline__ uint32_t shoup_mul(uint32_t x, uint32_t w, uint32_t wsh, uint32_t q) {
  return x * w - __umulhi(x, wsh) * q;  // [0, 2q)
}

// Programmatic dependent launch.  A grid launched with programmatic stream
// serialization may start while its predecessor in the stream is finishing;
// pdl_wait() blocks until that predecessor has completed and its writes are
// visible (a no-op for an ordinary launch).  pdl_trigger() lets the dependent
// grid be scheduled once every CTA of this grid has passed it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t m) { return min(x, x - m); }  // x < 2m

__device__ __forceinline__ uint32_t barrett64(uint64_t x, uint32_t q, uint64_t mu) {
  uint64_t qh = __umul64hi(x, mu);
  uint32_t r = (uint32_t)x - (uint32_t)qh * q;  // true remainder < 2q, exact mod 2^32
  return csub(r, q);
}

// x mod q for any 64-bit x, in [0, q): with x = hi*2^32 + lo,
// x = hi*(2^32 mod q) + lo (mod q).  One Shoup product on the multiply pipe
// plus conditional subtractions on the ALU pipe (q in (2^29, 2^30), so
// lo < 2^32 < 8q and 4q fits 32 bits).
// red64_2q stops at [0, 2q), the input range of the inverse transform.
__device__ __forceinline__ uint32_t red64_2q(uint64_t x, const LimbConst& lc) {
  const uint32_t q = lc.q, two_q = lc.two_q;
  const uint32_t a = shoup_mul((uint32_t)(x >> 32), lc.r32, lc.r32_sh, q);  // [0, 2q)
  const uint32_t lo = (uint32_t)x;
  const uint32_t b = csub(csub(lo, 2 * two_q), two_q);                      // [0, 2q)
  return csub(a + b, two_q);                                                 // [0, 4q) -> [0, 2q)
}
__device__ __forceinline__ uint32_t red64(uint64_t x, const LimbConst& lc) { return csub(red64_2q(x, lc), lc.q); }

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

// Padded shared-memory position of coefficient i: rows of 32 at a stride of 36 words.
constexpr int ROW = 36;
__host__ __device__ __forceinline__ constexpr int pad(int i) { return i + ((i >> 5) << 2); }
// 32-bit words of one padded polynomial of n coefficients
__host__ __device__ constexpr int padded_words(int n) { return n + n / 8; }

// A padded row (32 consecutive coefficients starting at p, 16-byte aligned)
// to registers and back as eight 128-bit accesses.
__device__ __forceinline__ void lds_row(const uint32_t* p, uint32_t* v) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint4 x = reinterpret_cast<const uint4*>(p)[j];
    v[4 * j] = x.x, v[4 * j + 1] = x.y, v[4 * j + 2] = x.z, v[4 * j + 3] = x.w;
  }
}
__device__ __forceinline__ void sts_row(uint32_t* p, const uint32_t* v) {
#pragma unroll
  for (int j = 0; j < 8; ++j)
    reinterpret_cast<uint4*>(p)[j] = make_uint4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}

// NG consecutive words (NG = 1, 2 or 4, p aligned to 4*NG bytes) as one access.
template <int NG, bool GLOBAL>
__device__ __forceinline__ void ld_n(const uint32_t* p, uint32_t* v) {
  if constexpr (NG == 4) {
    const uint4 x = GLOBAL ? __ldg(reinterpret_cast<const uint4*>(p)) : *reinterpret_cast<const uint4*>(p);
    v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
  } else if constexpr (NG == 2) {
    const uint2 x = GLOBAL ? __ldg(reinterpret_cast<const uint2*>(p)) : *reinterpret_cast<const uint2*>(p);
    v[0] = x.x, v[1] = x.y;
  } else {
    v[0] = GLOBAL ? __ldg(p) : *p;
  }
}
template <int NG>
__device__ __forceinline__ void st_n(uint32_t* p, const uint32_t* v) {
  if constexpr (NG == 4) *reinterpret_cast<uint4*>(p) = make_uint4(v[0], v[1], v[2], v[3]);
  else if constexpr (NG == 2) *reinterpret_cast<uint2*>(p) = make_uint2(v[0], v[1]);
  else *p = v[0];
}

// Streaming (evict-first) global store of NG consecutive words.
template <int NG>
__device__ __forceinline__ void stcs_n(uint32_t* p, const uint32_t* v) {
  if constexpr (NG == 4) __stcs(reinterpret_cast<uint4*>(p), make_uint4(v[0], v[1], v[2], v[3]));
  else if constexpr (NG == 2) __stcs(reinterpret_cast<uint2*>(p), make_uint2(v[0], v[1]));
  else __stcs(p, v[0]);
}

// Epilogues of the inverse transform receive NG adjacent final values at a
// time: through `epi.put<NG>(v, u)` when the epilogue has that vector form,
// else as NG calls `epi(v[j], u + j)`.
template <class E, class = void> struct has_put : std::false_type {};
template <class E>
struct has_put<E, std::void_t<decltype(std::declval<E&>().template put<1>((const uint32_t*)nullptr, 0))>>
    : std::true_type {};

template <int NG, class E>
__device__ __forceinline__ void epi_put(E& epi, const uint32_t* v, int u) {
  if constexpr (has_put<E>::value) {
    epi.template put<NG>(v, u);
  } else {
#pragma unroll
    for (int j = 0; j < NG; ++j) epi(v[j], u + j);
  }
}

// The store that ends every fused convolution item: o[u] = v, plus
// Delta * r[u] when a mask r is given, reduced to [0, q), as streaming stores.
// v is in [0, 2q) and the Shoup product in [0, 2q), so the sum stays below 4q;
// without a mask one conditional subtraction of q suffices.
struct MaskStore {
  uint32_t* o;
  const uint32_t* r;  // nullptr: no mask
  const LimbConst& lc;
  template <int NG>
  __device__ __forceinline__ void put(const uint32_t* v, int u) const {
    uint32_t x[NG];
#pragma unroll
    for (int j = 0; j < NG; ++j) x[j] = v[j];
    if (r) {
      uint32_t m[NG];
      ld_n<NG, true>(r + u, m);
#pragma unroll
      for (int j = 0; j < NG; ++j) x[j] = csub(csub(x[j] + shoup_mul(m[j], lc.delta, lc.delta_sh, lc.q), lc.two_q), lc.q);
    } else {
#pragma unroll
      for (int j = 0; j < NG; ++j) x[j] = csub(x[j], lc.q);
    }
    stcs_n<NG>(o + u, x);
  }
};

// Twiddle m of stage st for block blk of a pass that entered d stages
// earlier: table entry (1 << st) + (blk << d) + m.  For d >= 1 that index is
// even for even m, so twiddles m and m ^ 1 come from one 16-byte load.
__device__ __forceinline__ uint2 tw_at(const uint2* __restrict__ tw, int st, int blk, int d, int m) {
  const int i = (1 << st) + (blk << d);
  if (d == 0) return __ldg(tw + i + m);
  const uint4 t = __ldg(reinterpret_cast<const uint4*>(tw + i + (m & ~1)));
  return (m & 1) ? make_uint2(t.z, t.w) : make_uint2(t.x, t.y);
}

template <int LOGN> struct Plan;
template <> struct Plan<11> { static constexpr int R1 = 3, R2 = 3; };
template <> struct Plan<12> { static constexpr int R1 = 4, R2 = 3; };
template <> struct Plan<13> { static constexpr int R1 = 4, R2 = 4; };
template <> struct Plan<14> { static constexpr int R1 = 5, R2 = 4; };
// Other pass plans of the same transform: the first row-strided pass is
// radix 2^R1, the second 2^(LOGN - 5 - R1), the last radix 32; each row pass
// needs 3 <= R <= 5.  The result is the same canonical transform for every
// plan, so a caller may pick any valid plan (autotuned per workload).
__host__ __device__ constexpr bool plan_ok(int logn, int r1) {
  return r1 >= 3 && r1 <= 5 && logn - 5 - r1 >= 3 && logn - 5 - r1 <= 5;
}

// Resident CTAs per SM the register budget (64 per thread) is sized for:
// 1024 threads per SM.  Kernels on two polynomials run 2 * N/32 threads (one
// group per ciphertext component) on two padded polynomials of shared memory,
// so at N = 8192 two CTAs fit with about 90 KiB of L1 left for the twiddles.
template <int LOGN> constexpr int minb_two_polys() { return (512 >> (LOGN - 5)) > 0 ? (512 >> (LOGN - 5)) : 1; }
template <int LOGN> constexpr int minb_one_poly() { return 1024 >> (LOGN - 5); }

template <int LOGN> struct Geo {
  static constexpr int N = 1 << LOGN;
  static constexpr int T = N / 32;                 // threads per polynomial
  static constexpr int SMEM_WORDS = padded_words(N);  // one padded polynomial
};

// Row-strided pass over stages [S0, S0+R) (TL = N >> (S0+R) >= 32): group
// gid holds coefficients base + k*TL, k < 2^R.  Thread tid of the T = N/32
// threads takes the NG = 32 / 2^R adjacent groups NG*tid .. NG*tid + NG-1:
// one block, NG adjacent columns, i.e. element k of all its groups is one
// NG-word access at pb + k*PSTEP in padded shared memory.
template <int LOGN, int S0, int R>
struct PassGeo {
  static constexpr int N = 1 << LOGN;
  static constexpr int TL = N >> (S0 + R);
  static constexpr int NG = 32 >> R;
  static constexpr int PSTEP = TL + TL / 8;
  static_assert(TL % 32 == 0, "row-strided passes only; the contiguous one is pass32");
  static_assert(NG >= 1 && NG <= 4, "radix 8, 16 or 32");
  __device__ __forceinline__ static void of(int tid, int& blk, int& base, int& pb) {
    const int gid = NG * tid;
    blk = gid / TL;
    base = blk * (N >> S0) + gid % TL;
    pb = pad(base);
  }
};

// Forward pass over stages [S0, S0+R).  SRC_G: read the groups from global
// memory `g` (natural order) instead of shared memory.  T: threads sharing
// this polynomial.  v[k*NG + j] is element k of column j.
template <int LOGN, int T, int S0, int R, bool SRC_G>
__device__ __forceinline__ void fwd_pass(uint32_t* __restrict__ s, const uint32_t* __restrict__ g,
                                         const uint2* __restrict__ tw, uint32_t q, uint32_t two_q,
                                         int tid) {
  using PG = PassGeo<LOGN, S0, R>;
  constexpr int RAD = 1 << R, NG = PG::NG;
  static_assert(NG * T * RAD == PG::N, "one set of groups per thread");
  int blk, base, pb;
  PG::of(tid, blk, base, pb);
  uint32_t v[RAD * NG];
#pragma unroll
  for (int k = 0; k < RAD; ++k) {
    if (SRC_G) ld_n<NG, true>(g + base + k * PG::TL, v + k * NG);
    else ld_n<NG, false>(s + pb + k * PG::PSTEP, v + k * NG);
  }
#pragma unroll
  for (int d = 0; d < R; ++d) {
    const int half = RAD >> (d + 1);
#pragma unroll
    for (int k = 0; k < RAD; ++k) {
      if (k & half) continue;
      const uint2 w = tw_at(tw, S0 + d, blk, d, k >> (R - d));
#pragma unroll
      for (int j = 0; j < NG; ++j) ct_bfly(v[k * NG + j], v[(k + half) * NG + j], w.x, w.y, q, two_q);
    }
  }
#pragma unroll
  for (int k = 0; k < RAD; ++k) st_n<NG>(s + pb + k * PG::PSTEP, v + k * NG);
}

// Inverse pass over stages [S0, S0+R), applied from the highest stage down.
// LAST: this pass contains stage 0; hand each final value (in [0, 2q)) with
// its coefficient index to `epi`, which stores it.  SCALE: fold N^-1 into
// stage 0 (one more Shoup product per butterfly there); without it the
// result is N times the inverse transform, for inputs that already carry the
// factor N^-1 (the encoded weights and the prepared x^2+x plaintexts).
template <int LOGN, int T, int S0, int R, bool LAST, class Epi, bool SCALE = true>
__device__ __forceinline__ void inv_pass(uint32_t* __restrict__ s, const uint2* __restrict__ tw,
                                         const LimbConst& lc, int tid, Epi& epi) {
  using PG = PassGeo<LOGN, S0, R>;
  constexpr int RAD = 1 << R, NG = PG::NG;
  static_assert(NG * T * RAD == PG::N, "one set of groups per thread");
  const uint32_t q = lc.q, two_q = lc.two_q;
  int blk, base, pb;
  PG::of(tid, blk, base, pb);
  uint32_t v[RAD * NG];
#pragma unroll
  for (int k = 0; k < RAD; ++k) ld_n<NG, false>(s + pb + k * PG::PSTEP, v + k * NG);
#pragma unroll
  for (int d = R - 1; d >= 0; --d) {
    const int half = RAD >> (d + 1);
#pragma unroll
    for (int k = 0; k < RAD; ++k) {
      if (k & half) continue;
      if (LAST && SCALE && S0 + d == 0) {
#pragma unroll
        for (int j = 0; j < NG; ++j) {
          const uint32_t X = v[k * NG + j], Y = v[(k + half) * NG + j];
          v[k * NG + j] = shoup_mul(X + Y, lc.n_inv, lc.n_inv_sh, q);
          v[(k + half) * NG + j] = shoup_mul(X - Y + two_q, lc.last_w, lc.last_w_sh, q);
        }
      } else {
        const uint2 w = tw_at(tw, S0 + d, blk, d, k >> (R - d));
#pragma unroll
        for (int j = 0; j < NG; ++j) gs_bfly(v[k * NG + j], v[(k + half) * NG + j], w.x, w.y, q, two_q);
      }
    }
  }
  if (LAST) {
#pragma unroll
    for (int k = 0; k < RAD; ++k) epi_put<NG>(epi, v + k * NG, base + k * PG::TL);
  } else {
#pragma unroll
    for (int k = 0; k < RAD; ++k) st_n<NG>(s + pb + k * PG::PSTEP, v + k * NG);
  }
}

// The radix-32 pass on the contiguous group blk (32 coefficients), forward
// (stages S0..S0+4 ascending) or inverse (descending), with the thread-major
// twiddles of that pass: tg[p * T + blk] holds the twiddles of consumption
// order 2p and 2p+1.  Stage S0+d touches the pairs (k, k + 2^(4-d)) and uses
// twiddle m = k >> (5-d) of that stage.
template <bool INV>
__device__ __forceinline__ void pass32(uint32_t* v, const uint4* __restrict__ tg, int T, int blk,
                                       uint32_t q, uint32_t two_q) {
  int slot = 0;
#pragma unroll
  for (int dd = 0; dd < 5; ++dd) {
    const int d = INV ? 4 - dd : dd;
    const int half = 32 >> (d + 1);
#pragma unroll
    for (int m = 0; m < (1 << d); ++m) {
      const int sl = slot + m;
      const uint4 t4 = __ldg(tg + (sl >> 1) * T + blk);
      const uint32_t w = (sl & 1) ? t4.z : t4.x, ws = (sl & 1) ? t4.w : t4.y;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if ((k & half) || (k >> (5 - d)) != m) continue;
        if (INV) gs_bfly(v[k], v[k + half], w, ws, q, two_q);
        else ct_bfly(v[k], v[k + half], w, ws, q, two_q);
      }
    }
    slot += 1 << d;
  }
}

// Full forward NTT of one polynomial by T = N/32 threads: global `src` ->
// shared `s`, result in shared memory reduced to [0, q).  Caller syncs
// before reading `s`.  tw_l: the limb's tables (TwLayout words).
template <int LOGN, int R1 = Plan<LOGN>::R1>
__device__ __forceinline__ void ntt_forward_to_smem(uint32_t* s, const uint32_t* __restrict__ src,
                                                    const uint32_t* __restrict__ tw_l,
                                                    const LimbConst& lc, int tid) {
  constexpr int N = 1 << LOGN, T = N / 32, R2 = LOGN - 5 - R1;
  static_assert(plan_ok(LOGN, R1), "pass plan");
  const uint2* f = reinterpret_cast<const uint2*>(tw_l) + TW_FWD * N;
  const uint4* tg = reinterpret_cast<const uint4*>(tw_l + TwLayout<LOGN>::PAIRS_WORDS) + TW_FWD * 16 * T;
  fwd_pass<LOGN, T, 0, R1, true>(s, src, f, lc.q, lc.two_q, tid);
  __syncthreads();
  fwd_pass<LOGN, T, R1, R2, false>(s, nullptr, f, lc.q, lc.two_q, tid);
  __syncthreads();
  {
    uint32_t v[32];
    uint32_t* p = s + tid * ROW;
    lds_row(p, v);
    pass32<false>(v, tg, T, tid, lc.q, lc.two_q);
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = csub(csub(v[k], lc.two_q), lc.q);  // [0, 4q) -> [0, q)
    sts_row(p, v);
  }
}

// Full inverse NTT by T = N/32 threads of the polynomial in shared memory
// `s` (values in [0, 2q)); every output coefficient goes through
// `epi(value_in_[0,2q), u)`.  `bar()` synchronises every thread that takes
// part (several polynomials may be transformed side by side by disjoint
// thread groups sharing one barrier).
// gsrc: when not null, the first pass reads the thread's 32 coefficients
// straight from global memory instead of from `s`: the row's coefficients
// 8k .. 8k + 7 (natural order) are the 8 words at gsrc + k * gchunk (gchunk
// = 8 for a contiguous row).  Every such read happens before the first
// barrier, so the epilogue may write the result over gsrc in place.
template <int LOGN, class Epi, class Bar, bool SCALE = true, int R1 = Plan<LOGN>::R1>
__device__ __forceinline__ void intt_from_smem_bar(uint32_t* s, const uint32_t* __restrict__ tw_l,
                                                   const LimbConst& lc, int tid, Epi epi, Bar bar,
                                                   const uint32_t* gsrc = nullptr, size_t gchunk = 8) {
  constexpr int N = 1 << LOGN, T = N / 32, R2 = LOGN - 5 - R1;
  static_assert(plan_ok(LOGN, R1), "pass plan");
  const uint2* f = reinterpret_cast<const uint2*>(tw_l) + TW_INV * N;
  const uint4* tg = reinterpret_cast<const uint4*>(tw_l + TwLayout<LOGN>::PAIRS_WORDS) + TW_INV * 16 * T;
  {
    uint32_t v[32];
    uint32_t* p = s + tid * ROW;
    if (gsrc) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint4* src = reinterpret_cast<const uint4*>(gsrc + (size_t)(4 * tid + k) * gchunk);
        const uint4 x0 = src[0], x1 = src[1];
        v[8 * k] = x0.x, v[8 * k + 1] = x0.y, v[8 * k + 2] = x0.z, v[8 * k + 3] = x0.w;
        v[8 * k + 4] = x1.x, v[8 * k + 5] = x1.y, v[8 * k + 6] = x1.z, v[8 * k + 7] = x1.w;
      }
    } else {
      lds_row(p, v);
    }
    pass32<true>(v, tg, T, tid, lc.q, lc.two_q);
    sts_row(p, v);
  }
  bar();
  inv_pass<LOGN, T, R1, R2, false, Epi, SCALE>(s, f, lc, tid, epi);
  bar();
  inv_pass<LOGN, T, 0, R1, true, Epi, SCALE>(s, f, lc, tid, epi);
}

// As above with block-wide barriers.
template <int LOGN, class Epi>
__device__ __forceinline__ void intt_from_smem(uint32_t* s, const uint32_t* __restrict__ tw_l,
                                               const LimbConst& lc, int tid, Epi epi) {
  intt_from_smem_bar<LOGN>(s, tw_l, lc, tid, epi, [] { __syncthreads(); });
}

// N times the inverse transform, for inputs that already carry N^-1.
template <int LOGN, class Epi, int R1 = Plan<LOGN>::R1>
__device__ __forceinline__ void intt_from_smem_unscaled(uint32_t* s, const uint32_t* __restrict__ tw_l,
                                                        const LimbConst& lc, int tid, Epi epi,
                                                        const uint32_t* gsrc = nullptr, size_t gchunk = 8) {
  auto bar = [] { __syncthreads(); };
  intt_from_smem_bar<LOGN, Epi, decltype(bar), false, R1>(s, tw_l, lc, tid, epi, bar, gsrc, gchunk);
}

}  // namespace fl
