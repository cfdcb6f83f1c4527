// Persistent, warp-specialised homomorphic convolution over a stack of
// layers (rows a4-a6 for many layers and images in one launch).
//
// One CTA per SM pulls work items from a queue shared by every layer of the
// stack.  An item is one output ciphertext limb: (layer, image/band,
// output channel, limb), both components.  Two thread teams share the CTA:
//
//   producer team (PT threads): per-slot contraction mod q_l of the item's
//     weights with its NTT-domain inputs, 64-bit lazy accumulation.  Its
//     loads stream through a private cp.async ring, DEPTH stages deep per
//     thread, so that enough bytes are in flight to cover L2/HBM latency.  It
//     writes the reduced NTT-domain result straight into the item's place in
//     the output ciphertext (the lines stay in L2).
//   consumer team (PAR * N/32 threads): loads that result back into shared
//     memory, runs the inverse NTT of both components, adds the mask and
//     overwrites the output with the final coefficient-domain limb.
//
// The producer runs up to QD items ahead of the consumer, so the HBM- and
// L2-bound contraction overlaps the ALU-bound transform.  Hand-off uses
// shared-memory mbarriers (release/acquire at CTA scope, which orders the
// producer's global writes before the consumer's reads); every wait is
// bounded by a wall-clock limit after which the team sets an error word and
// leaves the loop (both teams then drain out: no thread is ever left in a
// hardware barrier).  Team-internal synchronisation uses named barriers whose
// thread counts are fixed, and each team's leader alone waits on an mbarrier
// and broadcasts the outcome, so all threads of a team take the same path.
#include <cuda_runtime.h>

#include "fl_device.cuh"
#include "fl_launch.h"

namespace fl {

namespace {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s
enum { BAR_CONSUMER = 1, BAR_PRODUCER = 2 };

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n}" ::"r"(a)
               : "memory");
}

// Wait for the phase with the given parity to complete; false on timeout
// (kWaitLimitNs of wall clock, or kWaitMaxPolls polls, whichever comes first).
constexpr unsigned kWaitMaxPolls = 1u << 26;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  const unsigned long long t0 = globaltimer();
  for (unsigned polls = 0; polls < kWaitMaxPolls; ++polls) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer() - t0 > kWaitLimitNs) return false;
  }
  return false;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

}  // namespace

// PAR = 2: the consumer team has 2 * N/32 threads and transforms both
// components side by side; PAR = 1: N/32 threads, one component after the
// other (N = 16384, where twice as many threads would leave too few
// registers).  MINB: resident CTAs per SM.
constexpr int QD = 4;  // items the producer may run ahead of the consumer

// Shared memory: consumer polys [2][SW] | mbarriers full[QD], empty[QD] |
// item ids [QD] | producer broadcast | two abort flags | producer ring.
template <int LOGN>
__host__ __device__ constexpr int ring_word_offset() {  // same for every GS
  return 2 * Geo<LOGN>::SMEM_WORDS + ((2 * QD * 8 + QD * 8 + 8 + 8 + 15) / 16) * 4;
}

// PAR = 2: the consumer team has 2 * N/32 threads and transforms both
// components side by side; PAR = 1: N/32 threads, one component after the
// other (N = 16384, where twice as many threads would leave too few
// registers).  DEPTH: producer stages in flight per thread, GS weight rows
// each.  MINB: resident CTAs per SM.
template <int LOGN, int PT, int PAR, int DEPTH, int GS, int MINB>
__global__ void __launch_bounds__(PT + PAR * ((1 << LOGN) / 32), MINB)
    k_stack(StackArgs a, unsigned long long* __restrict__ ctl, const uint32_t* __restrict__ tw, CtxConst cc) {
  constexpr int N = 1 << LOGN, T = N / 32, CTN = PAR * T, SW = Geo<LOGN>::SMEM_WORDS;
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* polys = sm;  // [2][SW]
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + 2 * SW);
  uint64_t* empty = full + QD;
  volatile long long* slot_item = reinterpret_cast<volatile long long*>(empty + QD);  // [QD]
  volatile long long* bcast = slot_item + QD;
  volatile int* abort_p = reinterpret_cast<volatile int*>(bcast + 1);
  volatile int* abort_c = abort_p + 1;
  unsigned long long* counter = ctl;
  unsigned long long* err = ctl + 1;

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int b = 0; b < QD; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], 1);
    }
    *abort_p = 0;
    *abort_c = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int L = cc.L;
  const size_t ct_words = (size_t)2 * L * N;

  if (tid < PT) {
    // ---------------- producer: contraction ----------------
    // Thread pt owns slot quad pt of every range of CS = 4*PT slots.  Each
    // item is a stream of stages (slot range r, rows g0..g0+GS); the thread
    // copies exactly the 16-byte pieces it will use (weight row, both input
    // components) into its own ring slot with cp.async, DEPTH stages ahead,
    // continuing into the next item, and accumulates from shared memory.
    const int pt = tid;
    constexpr int CS = 4 * PT;
    uint4* ring = reinterpret_cast<uint4*>(sm + ring_word_offset<LOGN>());  // [DEPTH][3][GS][PT]

    long long cur, nxt;
    if (pt == 0) *bcast = (long long)atomicAdd(counter, 1ull);
    named_sync(BAR_PRODUCER, PT);
    cur = *bcast;
    named_sync(BAR_PRODUCER, PT);

    // Stage stream cursor for issuing copies: item iss.it, slot range
    // iss_r, row chunk iss_g.  It runs at most DEPTH stages ahead of
    // consumption, and every item has at least N/CS >= 8 stages, so it never
    // passes the item after `cur`.  Counters advance incrementally (no
    // division) to keep the per-stage instruction count low.
    constexpr int NR = N / CS;
    struct Src {
      const uint32_t* W;  // weight rows of the item (row g at W + g*N)
      const uint32_t* C;  // component-0 input row g at C + g*ct_words, component 1 at + L*N
      uint32_t* out;      // component-0 output limb (component 1 at + L*N)
      int G, ngc;         // rows, row chunks
      long long it;
      bool live;
    };
    auto src_of = [&](long long it, Src& o) {
      o.it = it;
      o.live = it >= 0 && it < a.n_items;
      if (!o.live) return;
      const Item x = decode(a, it);
      const StackLayer& y = a.layer[x.li];
      const int bimg = x.bb / y.bands, band = x.bb % y.bands;
      o.W = y.w_hat + ((size_t)x.l * y.Cout + x.i) * y.G * N;
      o.C = y.c_hat + ((size_t)bimg * y.n_in + (size_t)band * y.G) * ct_words + (size_t)x.l * N;
      o.out = y.out + ((size_t)bimg * y.n_out + (size_t)x.i * y.bands + band) * ct_words + (size_t)x.l * N;
      o.G = y.G;
      o.ngc = (y.G + GS - 1) / GS;
    };
    Src iss, cons;
    src_of(cur, iss);
    cons = iss;
    int iss_r = 0, iss_g = 0, iss_slot = 0, inflight = 0;
    bool nxt_known = false;
    nxt = -1;
    const uint32_t ln = (uint32_t)L * N;

    auto issue = [&]() {
      const int u = iss_r * CS + 4 * pt;
      const int g0 = iss_g * GS;
      uint4* dst = ring + (iss_slot * 3 * GS) * PT + pt;
      const uint32_t* wsrc = iss.W + (size_t)g0 * N + u;
      const uint32_t* csrc = iss.C + (size_t)g0 * ct_words + u;
#pragma unroll
      for (int gs = 0; gs < GS; ++gs) {
        if (g0 + gs < iss.G) {
          cp_async16(dst + (0 * GS + gs) * PT, wsrc + (size_t)gs * N);
          cp_async16(dst + (1 * GS + gs) * PT, csrc + (size_t)gs * ct_words);
          cp_async16(dst + (2 * GS + gs) * PT, csrc + (size_t)gs * ct_words + ln);
        }
      }
      cp_async_commit();
      ++inflight;
      iss_slot = iss_slot + 1 == DEPTH ? 0 : iss_slot + 1;
      if (++iss_g == iss.ngc) {
        iss_g = 0;
        if (++iss_r == NR) {
          iss_r = 0;
          Src n;
          src_of(nxt_known ? nxt : -1, n);
          iss = n;
        }
      }
    };
    auto can_issue = [&]() { return iss.live && (nxt_known || iss.it == cur); };
    int cons_slot = 0;

    for (int j = 0;; ++j) {
      const int b = j % QD;
      if (pt == 0) {
        bool ok = true;
        if (cur < a.n_items) {
          *bcast = (long long)atomicAdd(counter, 1ull);
          if (j >= QD) ok = mbar_wait(&empty[b], (unsigned)((j / QD - 1) & 1));
        } else {
          *bcast = a.n_items;
        }
        if (!ok) {
          atomicOr(err, 1ull);
          *abort_p = 1;
        }
      }
      named_sync(BAR_PRODUCER, PT);
      if (*abort_p) break;
      nxt = *bcast;
      nxt_known = true;
      named_sync(BAR_PRODUCER, PT);  // everyone has read bcast
      if (cur >= a.n_items) {
        if (pt == 0) {
          slot_item[b] = -1;
          mbar_arrive(&full[b]);
        }
        break;
      }
      while (inflight < DEPTH && can_issue()) issue();

      const Item x = decode(a, cur);
      const LimbConst lc = cc.limb[x.l];
#pragma unroll 1
      for (int r = 0; r < NR; ++r) {
        uint64_t a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0};
        int folded = 0;
#pragma unroll 1
        for (int gc = 0; gc < cons.ngc; ++gc) {
          // wait for this thread's copies of the oldest stage in flight
          if (inflight >= 3) cp_async_wait<2>();
          else if (inflight == 2) cp_async_wait<1>();
          else cp_async_wait<0>();
          const uint4* src = ring + (cons_slot * 3 * GS) * PT + pt;
          const int rows = min(GS, cons.G - gc * GS);
#pragma unroll
          for (int gs = 0; gs < GS; ++gs) {
            if (gs < rows) {
              const uint4 w = src[(0 * GS + gs) * PT];
              const uint4 x0 = src[(1 * GS + gs) * PT];
              const uint4 x1 = src[(2 * GS + gs) * PT];
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
          folded += rows;
          if (folded > 16 - GS && gc + 1 < cons.ngc) {  // the next chunk could pass 16 products: fold
            folded = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              a0[q] = barrett64(a0[q], lc.q, lc.mu);
              a1[q] = barrett64(a1[q], lc.q, lc.mu);
            }
          }
          // The refill below overwrites the slot just read: make the
          // accumulations (which consume the shared-memory loads) complete
          // in program order before the copy is issued.
          asm volatile("" ::"l"(a0[0]), "l"(a0[1]), "l"(a0[2]), "l"(a0[3]), "l"(a1[0]), "l"(a1[1]), "l"(a1[2]),
                       "l"(a1[3]));
          --inflight;
          cons_slot = cons_slot + 1 == DEPTH ? 0 : cons_slot + 1;
          if (can_issue()) issue();
        }
        // slot range r complete: its NTT-domain result goes to the output
        const int u = r * CS + 4 * pt;
        uint4 y0, y1;
        y0.x = barrett64(a0[0], lc.q, lc.mu);
        y0.y = barrett64(a0[1], lc.q, lc.mu);
        y0.z = barrett64(a0[2], lc.q, lc.mu);
        y0.w = barrett64(a0[3], lc.q, lc.mu);
        y1.x = barrett64(a1[0], lc.q, lc.mu);
        y1.y = barrett64(a1[1], lc.q, lc.mu);
        y1.z = barrett64(a1[2], lc.q, lc.mu);
        y1.w = barrett64(a1[3], lc.q, lc.mu);
        *reinterpret_cast<uint4*>(cons.out + u) = y0;
        *reinterpret_cast<uint4*>(cons.out + ln + u) = y1;
      }
      named_sync(BAR_PRODUCER, PT);  // every result word of the item is written
      if (pt == 0) {
        slot_item[b] = cur;
        mbar_arrive(&full[b]);  // release at CTA scope: the writes above precede the consumer's reads
      }
      cur = nxt;
      Src nc;
      src_of(cur, nc);
      cons = nc;
    }
    cp_async_wait<0>();  // no copy of this thread is left in flight
  } else {
    // ---------------- consumer: inverse NTTs + mask ----------------
    const int ct = tid - PT;
    for (int k = 0;; ++k) {
      const int b = k % QD;
      if (ct == 0) {
        if (!mbar_wait(&full[b], (unsigned)((k / QD) & 1))) {
          atomicOr(err, 2ull);
          *abort_c = 1;
        }
      }
      named_sync(BAR_CONSUMER, CTN);
      if (*abort_c) break;
      const long long it = slot_item[b];
      if (it < 0) break;
      const Item x = decode(a, it);
      const StackLayer& s = a.layer[x.li];
      const LimbConst lc = cc.limb[x.l];
      const int bimg = x.bb / s.bands, band = x.bb % s.bands;
      const size_t oct = (size_t)bimg * s.n_out + (size_t)x.i * s.bands + band;
      uint32_t* o0 = s.out + oct * ct_words + (size_t)x.l * N;
      // the NTT-domain result of both components into shared memory
      for (int v = ct; v < N / 2; v += CTN) {
        const int h = v >= N / 4, vq = v - h * (N / 4);
        const uint4 y = __ldcg(reinterpret_cast<const uint4*>(o0 + (size_t)h * L * N) + vq);
        *reinterpret_cast<uint4*>(polys + (size_t)h * SW + pad(4 * vq)) = y;
      }
      named_sync(BAR_CONSUMER, CTN);
      const uint32_t* twl = tw + (size_t)x.l * TwLayout<LOGN>::LIMB_WORDS;
#pragma unroll 1
      for (int hs = 0; hs < 3 - PAR; ++hs) {
        const int h = PAR == 2 ? (ct >= T) : hs;
        const int lt = PAR == 2 ? ct - h * T : ct;
        uint32_t* op = o0 + (size_t)h * L * N;
        const uint32_t* rr = (s.r && h == 0) ? s.r + oct * N : nullptr;
        uint32_t* sp = polys + (size_t)h * SW;
        if (hs) named_sync(BAR_CONSUMER, CTN);
        // the encoded weights carry N^-1, so the transform skips that scaling
        MaskStore epi{op, rr, lc};
        auto bar = [] { named_sync(BAR_CONSUMER, CTN); };
        intt_from_smem_bar<LOGN, decltype(epi), decltype(bar), false>(sp, twl, lc, lt, epi, bar);
      }
      named_sync(BAR_CONSUMER, CTN);  // every consumer thread is done with the item
      if (ct == 0) mbar_arrive(&empty[b]);
    }
  }
}

template <int LOGN> struct StackCfg {
  static constexpr int PT = LOGN == 11 ? 64 : LOGN == 12 ? 128 : 256;
  static constexpr int PAR = LOGN <= 13 ? 2 : 1;
  static constexpr int DEPTH = 3;
  static constexpr int GS = LOGN <= 13 ? 4 : 2;
  static constexpr int MINB = LOGN == 11 ? 4 : LOGN == 12 ? 2 : 1;
  static constexpr int THREADS = PT + PAR * ((1 << LOGN) / 32);
};

template <int LOGN>
static size_t stack_smem() {
  using C = StackCfg<LOGN>;
  return (size_t)ring_word_offset<LOGN>() * 4 + (size_t)C::DEPTH * 3 * C::GS * C::PT * 16;
}

int stack_ctas_per_sm(int logn) {
  switch (logn) {
    case 11: return StackCfg<11>::MINB;
    case 12: return StackCfg<12>::MINB;
    case 13: return StackCfg<13>::MINB;
    case 14: return StackCfg<14>::MINB;
  }
  return 1;
}

template <int LOGN>
static cudaError_t stack_setup() {
  using C = StackCfg<LOGN>;
  return cudaFuncSetAttribute(k_stack<LOGN, C::PT, C::PAR, C::DEPTH, C::GS, C::MINB>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stack_smem<LOGN>());
}

cudaError_t launch_stack_setup(int logn) {
  switch (logn) {
    case 11: return stack_setup<11>();
    case 12: return stack_setup<12>();
    case 13: return stack_setup<13>();
    case 14: return stack_setup<14>();
  }
  return cudaErrorInvalidValue;
}

template <int LOGN>
static cudaError_t stack_launch(const StackArgs& a, unsigned long long* ctl, const uint32_t* tw, const CtxConst& cc,
                                int grid, cudaStream_t st) {
  using C = StackCfg<LOGN>;
  k_stack<LOGN, C::PT, C::PAR, C::DEPTH, C::GS, C::MINB><<<grid, C::THREADS, stack_smem<LOGN>(), st>>>(a, ctl, tw, cc);
  return cudaGetLastError();
}

// Self-test of the bounded wait: an mbarrier that expects one arrival which
// never comes.  The wait must give up, set bit 2 of the error word and
// return, leaving the context usable.
__global__ void k_wait_timeout_probe(unsigned long long* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0)) atomicOr(err, 4ull);
}

cudaError_t launch_wait_timeout_probe(unsigned long long* err, cudaStream_t st) {
  k_wait_timeout_probe<<<1, 32, 0, st>>>(err);
  return cudaGetLastError();
}

cudaError_t launch_stack(int logn, const StackArgs& a, unsigned long long* ctl, const uint32_t* tw,
                         const CtxConst& cc, int sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ctl, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (a.n_items == 0) return cudaSuccess;
  const long long slots = (long long)sms * stack_ctas_per_sm(logn);
  const int grid = (int)(a.n_items < slots ? a.n_items : slots);
  switch (logn) {
    case 11: return stack_launch<11>(a, ctl, tw, cc, grid, st);
    case 12: return stack_launch<12>(a, ctl, tw, cc, grid, st);
    case 13: return stack_launch<13>(a, ctl, tw, cc, grid, st);
    case 14: return stack_launch<14>(a, ctl, tw, cc, grid, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Forward NTT of many row segments in one launch (the inputs of every layer
// of a stack).  Segment s covers rows [row_begin[s], row_begin[s+1]) of the
// grid, reading contiguous rows [..][L][N] from src[s] into dst[s].
// ---------------------------------------------------------------------------
template <int LOGN, int R1 = Plan<LOGN>::R1>
__global__ void __launch_bounds__((1 << LOGN) / 32, 1024 >> (LOGN - 5))
    k_ntt_fwd_multi(NttSegs segs, const uint32_t* __restrict__ tw, CtxConst cc) {
  constexpr int N = 1 << LOGN, T = N / 32;
  extern __shared__ uint32_t sm[];
  const int r = blockIdx.x, tid = threadIdx.x;
  pdl_trigger();  // the stack's conv grid may be scheduled once every CTA is running
  int s = 0;
  while (s + 1 < segs.n && r >= segs.row_begin[s + 1]) ++s;
  const int lr = r - segs.row_begin[s];
  const int l = lr % cc.L;
  const LimbConst lc = cc.limb[l];
  const uint32_t* x = segs.src[s] + (size_t)lr * N;
  uint32_t* y = segs.dst[s] + (size_t)lr * N;
  ntt_forward_to_smem<LOGN, R1>(sm, x, tw + (size_t)l * TwLayout<LOGN>::LIMB_WORDS, lc, tid);
  __syncthreads();
  for (int v = tid; v < N / 4; v += T) {
    const uint4 o = *reinterpret_cast<const uint4*>(sm + pad(4 * v));  // 4 slots of one row
    reinterpret_cast<uint4*>(y)[v] = o;
  }
}

template <int LOGN>
static cudaError_t multi_setup() {
  cudaError_t e = cudaSuccess;
  for (int r1 = 3; r1 <= 5; ++r1) {  // every instantiated pass plan
    if (!plan_available(LOGN, r1)) continue;
    FL_PLAN_DISPATCH(LOGN, r1, (e = cudaFuncSetAttribute(k_ntt_fwd_multi<LG, R1>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         Geo<LG>::SMEM_WORDS * 4)));
    if (e) return e;
  }
  return e;
}

cudaError_t launch_ntt_multi_setup(int logn) {
  switch (logn) {
    case 11: return multi_setup<11>();
    case 12: return multi_setup<12>();
    case 13: return multi_setup<13>();
    case 14: return multi_setup<14>();
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_ntt_multi(int logn, const NttSegs& segs, const uint32_t* tw, const CtxConst& cc,
                             cudaStream_t st, int r1) {
  const int rows = segs.row_begin[segs.n];
  if (rows == 0) return cudaSuccess;
  const int N = 1 << logn;
  const size_t smem = (size_t)padded_words(N) * 4;
  FL_PLAN_DISPATCH(logn, r1, (k_ntt_fwd_multi<LG, R1><<<rows, N / 32, smem, st>>>(segs, tw, cc)));
  return cudaGetLastError();
}

}  // namespace fl
