// Persistent, warp-specialised homomorphic convolution over a stack of
// layers (rows a4-a6 for many layers and images in one launch).
//
// One CTA per SM pulls work items from a queue shared by every layer of the
// stack.  An item is one output ciphertext limb: (layer, image/band,
// output channel, limb), both components.  Two thread teams share the CTA:
//
//   producer team (PT threads): per-slot contraction mod q_l of the item's
//     weights with its NTT-domain inputs, 64-bit lazy accumulation, written
//     to one of BUFS shared-memory buffers (two polynomials each);
//   consumer team (2 * N/32 threads): inverse NTT of both components side by
//     side, mask epilogue, streaming stores of the output ciphertext limb.
//
// With two buffers the producer computes item k+1 while the consumer
// transforms item k, so the HBM-bound contraction overlaps the ALU-bound
// transform.  Hand-off uses shared-memory mbarriers; every wait is bounded
// by a wall-clock limit after which the team sets an error word and leaves
// the loop (both teams then drain out: no thread is ever left in a hardware
// barrier).  Team-internal synchronisation uses named barriers whose thread
// counts are fixed, and each team's leader alone waits on an mbarrier and
// broadcasts the outcome, so all threads of a team take the same path.
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

// Wait for the phase with the given parity to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  const unsigned long long t0 = globaltimer();
  while (true) {
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
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

// Item index -> layer (linear scan: stacks hold at most FL_STACK_MAX layers).
__device__ __forceinline__ int find_layer(const StackArgs& a, long long it) {
  int li = 0;
  while (li + 1 < a.n_layers && it >= a.layer[li + 1].item_begin) ++li;
  return li;
}

struct Item {
  int li, bb, i, l;
};

__device__ __forceinline__ Item decode(const StackArgs& a, long long it) {
  Item x;
  x.li = find_layer(a, it);
  const StackLayer& s = a.layer[x.li];
  long long r = it - s.item_begin;
  x.bb = (int)(r % s.BB);
  r /= s.BB;
  x.i = (int)(r % s.Cout);
  x.l = (int)(r / s.Cout);
  return x;
}

}  // namespace

// PAR = 2: the consumer team has 2 * N/32 threads and transforms both
// components side by side; PAR = 1: N/32 threads, one component after the
// other (N = 16384, where twice as many threads would leave too few
// registers).  MINB: resident CTAs per SM.
constexpr int DEPTH = 3;  // stages in flight per producer thread
constexpr int GS = 2;     // weight rows per stage

template <int LOGN, int BUFS>
__host__ __device__ constexpr int ring_word_offset() {
  // polys, then 2*BUFS mbarriers, BUFS+1 item words and two flags (rounded to 16 bytes)
  return BUFS * 2 * Geo<LOGN>::SMEM_WORDS + ((2 * BUFS * 8 + (BUFS + 1) * 8 + 8 + 15) / 16) * 4;
}

template <int LOGN, int BUFS, int PT, int PAR, int MINB>
__global__ void __launch_bounds__(PT + PAR * ((1 << LOGN) / 32), MINB)
    k_stack(StackArgs a, unsigned long long* __restrict__ ctl, const uint32_t* __restrict__ tw, CtxConst cc) {
  constexpr int N = 1 << LOGN, T = N / 32, CTN = PAR * T, SW = Geo<LOGN>::SMEM_WORDS;
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* polys = sm;  // [BUFS][2][SW]
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + BUFS * 2 * SW);
  uint64_t* empty = full + BUFS;
  volatile long long* slot_item = reinterpret_cast<volatile long long*>(empty + BUFS);  // [BUFS]
  volatile long long* bcast = slot_item + BUFS;                                         // producer broadcast
  volatile int* abort_p = reinterpret_cast<volatile int*>(bcast + 1);
  volatile int* abort_c = abort_p + 1;
  unsigned long long* counter = ctl;
  unsigned long long* err = ctl + 1;

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int b = 0; b < BUFS; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], 1);
    }
    *abort_p = 0;
    *abort_c = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (tid < PT) {
    // ---------------- producer: contraction ----------------
    // Thread pt owns slot quad pt of every range of CS = 4*PT slots.  Each
    // item is a stream of stages (slot range r, rows g0..g0+GS); the thread
    // copies exactly the 16-byte pieces it will use (weight row, both input
    // components) into its own ring slot with cp.async, DEPTH stages ahead,
    // continuing into the next item, and accumulates from shared memory.
    const int pt = tid;
    constexpr int CS = 4 * PT;
    uint4* ring = reinterpret_cast<uint4*>(sm + ring_word_offset<LOGN, BUFS>());  // [DEPTH][3][GS][PT]
    const int L = cc.L;
    const size_t ct_words = (size_t)2 * L * N;

    // current / next item (the leader fetches one item ahead)
    long long cur, nxt;
    if (pt == 0) *bcast = (long long)atomicAdd(counter, 1ull);
    named_sync(BAR_PRODUCER, PT);
    cur = *bcast;
    named_sync(BAR_PRODUCER, PT);

    // Stage stream cursor for issuing copies: item iss.it, stage iss_s.  It
    // runs at most DEPTH stages ahead of consumption, and every item has at
    // least 8 stages, so it never passes the item after `cur`.
    struct Src {
      const uint32_t* W;  // weight rows of the item (row g at W + g*N)
      const uint32_t* C;  // component-0 input row g at C + g*ct_words, component 1 at + L*N
      int G, ngc, ns;     // rows, row chunks, stages
      long long it;
    };
    auto src_of = [&](long long it, Src& o) {
      o.it = it;
      if (it < 0 || it >= a.n_items) {
        o.ns = 0;
        return;
      }
      const Item x = decode(a, it);
      const StackLayer& y = a.layer[x.li];
      const int bimg = x.bb / y.bands, band = x.bb % y.bands;
      o.W = y.w_hat + ((size_t)x.l * y.Cout + x.i) * y.G * N;
      o.C = y.c_hat + ((size_t)bimg * y.n_in + (size_t)band * y.G) * ct_words + (size_t)x.l * N;
      o.G = y.G;
      o.ngc = (y.G + GS - 1) / GS;
      o.ns = (N / CS) * o.ngc;
    };
    Src iss, cons;
    src_of(cur, iss);
    cons = iss;
    int iss_s = 0;     // next stage of `iss` to issue
    long long issued = 0, consumed = 0;
    bool nxt_known = false;
    nxt = -1;

    // issue the copies of one stage into ring slot (issued % DEPTH)
    auto issue = [&]() {
      const int slot = (int)(issued % DEPTH);
      const int r = iss_s / iss.ngc, g0 = (iss_s % iss.ngc) * GS;
      const int u = r * CS + 4 * pt;
#pragma unroll
      for (int gs = 0; gs < GS; ++gs) {
        const int g = g0 + gs;
        if (g < iss.G) {
          const uint32_t* wsrc = iss.W + (size_t)g * N + u;
          const uint32_t* c0 = iss.C + (size_t)g * ct_words + u;
          cp_async16(ring + ((slot * 3 + 0) * GS + gs) * PT + pt, wsrc);
          cp_async16(ring + ((slot * 3 + 1) * GS + gs) * PT + pt, c0);
          cp_async16(ring + ((slot * 3 + 2) * GS + gs) * PT + pt, c0 + (size_t)L * N);
        }
      }
      cp_async_commit();
      ++issued;
      if (++iss_s == iss.ns) {  // move the issue cursor to the next item
        iss_s = 0;
        Src n;
        src_of(nxt_known ? nxt : -1, n);
        iss = n;
      }
    };
    auto can_issue = [&]() { return iss.ns > 0 && (nxt_known || iss.it == cur); };

    for (int j = 0;; ++j) {
      const int b = j % BUFS;
      // leader: fetch the item after `cur`, and wait until buffer b is free
      if (pt == 0) {
        bool ok = true;
        if (cur < a.n_items) {
          *bcast = (long long)atomicAdd(counter, 1ull);
          if (j >= BUFS) ok = mbar_wait(&empty[b], (unsigned)((j / BUFS - 1) & 1));
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
      // keep DEPTH stages in flight
      while (issued - consumed < DEPTH && can_issue()) issue();

      const Item x = decode(a, cur);
      const LimbConst lc = cc.limb[x.l];
      uint32_t* s0 = polys + (size_t)(2 * b) * SW;
      uint32_t* s1 = s0 + SW;
      uint64_t a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0};
      int folded = 0;
#pragma unroll 1
      for (int st = 0; st < cons.ns; ++st) {
        // stage `consumed` is the oldest in flight: wait for this thread's copies
        const long long ahead = issued - consumed - 1;
        if (ahead >= 2) cp_async_wait<2>();
        else if (ahead == 1) cp_async_wait<1>();
        else cp_async_wait<0>();
        const int slot = (int)(consumed % DEPTH);
        const int r = st / cons.ngc, g0 = (st % cons.ngc) * GS;
#pragma unroll
        for (int gs = 0; gs < GS; ++gs) {
          if (g0 + gs < cons.G) {
            const uint4 w = ring[((slot * 3 + 0) * GS + gs) * PT + pt];
            const uint4 x0 = ring[((slot * 3 + 1) * GS + gs) * PT + pt];
            const uint4 x1 = ring[((slot * 3 + 2) * GS + gs) * PT + pt];
            a0[0] += (uint64_t)w.x * x0.x;
            a0[1] += (uint64_t)w.y * x0.y;
            a0[2] += (uint64_t)w.z * x0.z;
            a0[3] += (uint64_t)w.w * x0.w;
            a1[0] += (uint64_t)w.x * x1.x;
            a1[1] += (uint64_t)w.y * x1.y;
            a1[2] += (uint64_t)w.z * x1.z;
            a1[3] += (uint64_t)w.w * x1.w;
            if (++folded == 16) {  // 16 products < 2^64: fold before the next
              folded = 0;
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                a0[q] = barrett64(a0[q], lc.q, lc.mu);
                a1[q] = barrett64(a1[q], lc.q, lc.mu);
              }
            }
          }
        }
        // The refill below overwrites the slot just read: make the
        // accumulations (which consume the shared-memory loads) complete in
        // program order before the copy is issued.
        asm volatile("" ::"l"(a0[0]), "l"(a0[1]), "l"(a0[2]), "l"(a0[3]), "l"(a1[0]), "l"(a1[1]), "l"(a1[2]),
                     "l"(a1[3]));
        ++consumed;
        // refill the slot just freed (the ring slot is private to this thread)
        if (can_issue()) issue();
        if (st % cons.ngc == cons.ngc - 1) {  // slot range r complete
          const int pu = pad(r * CS + 4 * pt);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            s0[pu + q] = barrett64(a0[q], lc.q, lc.mu);
            s1[pu + q] = barrett64(a1[q], lc.q, lc.mu);
            a0[q] = 0;
            a1[q] = 0;
          }
          folded = 0;
        }
      }
      named_sync(BAR_PRODUCER, PT);  // all slots of the item written
      if (pt == 0) {
        slot_item[b] = cur;
        mbar_arrive(&full[b]);
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
      const int b = k % BUFS;
      if (ct == 0) {
        if (!mbar_wait(&full[b], (unsigned)((k / BUFS) & 1))) {
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
      const int L = cc.L;
      const LimbConst lc = cc.limb[x.l];
      const int bimg = x.bb / s.bands, band = x.bb % s.bands;
      const size_t ct_words = (size_t)2 * L * N;
      const size_t oct = (size_t)bimg * s.n_out + (size_t)x.i * s.bands + band;
      const uint32_t* twl = tw + (size_t)x.l * TwLayout<LOGN>::LIMB_WORDS;
#pragma unroll 1
      for (int hs = 0; hs < 3 - PAR; ++hs) {
        const int h = PAR == 2 ? (ct >= T) : hs;
        const int lt = PAR == 2 ? ct - h * T : ct;
        uint32_t* op = s.out + oct * ct_words + (size_t)h * L * N + (size_t)x.l * N;
        const uint32_t* rr = (s.r && h == 0) ? s.r + oct * N : nullptr;
        uint32_t* sp = polys + (size_t)(2 * b + h) * SW;
        if (hs) named_sync(BAR_CONSUMER, CTN);
        intt_from_smem_bar<LOGN>(sp, twl, lc, lt,
                                 [&](uint32_t v, int u) {
                                   uint32_t y = v;
                                   if (rr) y += shoup_mul(__ldg(rr + u), lc.delta, lc.delta_sh, lc.q);
                                   __stcs(op + u, csub(csub(y, lc.two_q), lc.q));
                                 },
                                 [] { named_sync(BAR_CONSUMER, CTN); });
      }
      named_sync(BAR_CONSUMER, CTN);  // every consumer thread is done with buffer b
      if (ct == 0) mbar_arrive(&empty[b]);
    }
  }
}

template <int LOGN, int BUFS, int PT>
static size_t stack_smem() {
  return (size_t)ring_word_offset<LOGN, BUFS>() * 4 + (size_t)DEPTH * 3 * GS * PT * 16;
}

// N <= 8192: two buffers (the producer runs one item ahead); N = 16384: the
// four padded polynomials of two buffers do not fit, so one buffer and a
// consumer team that transforms one component after the other.  Resident
// CTAs per SM follow from shared memory (about 135 KiB per SM).
template <int LOGN> struct StackCfg {
  static constexpr int BUFS = LOGN <= 13 ? 2 : 1;
  static constexpr int PT = LOGN == 11 ? 64 : LOGN == 12 ? 128 : 256;
  static constexpr int PAR = LOGN <= 13 ? 2 : 1;
  static constexpr int MINB = LOGN == 11 ? 4 : LOGN == 12 ? 2 : 1;
  static constexpr int THREADS = PT + PAR * ((1 << LOGN) / 32);
};

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
  return cudaFuncSetAttribute(k_stack<LOGN, C::BUFS, C::PT, C::PAR, C::MINB>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stack_smem<LOGN, C::BUFS, C::PT>());
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
  k_stack<LOGN, C::BUFS, C::PT, C::PAR, C::MINB>
      <<<grid, C::THREADS, stack_smem<LOGN, C::BUFS, C::PT>(), st>>>(a, ctl, tw, cc);
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
template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 32, 1024 >> (LOGN - 5))
    k_ntt_fwd_multi(NttSegs segs, const uint32_t* __restrict__ tw, CtxConst cc) {
  constexpr int N = 1 << LOGN, T = N / 32;
  extern __shared__ uint32_t sm[];
  const int r = blockIdx.x, tid = threadIdx.x;
  int s = 0;
  while (s + 1 < segs.n && r >= segs.row_begin[s + 1]) ++s;
  const int lr = r - segs.row_begin[s];
  const int l = lr % cc.L;
  const LimbConst lc = cc.limb[l];
  const uint32_t* x = segs.src[s] + (size_t)lr * N;
  uint32_t* y = segs.dst[s] + (size_t)lr * N;
  ntt_forward_to_smem<LOGN>(sm, x, tw + (size_t)l * TwLayout<LOGN>::LIMB_WORDS, lc, tid);
  __syncthreads();
  for (int v = tid; v < N / 4; v += T) {
    uint4 o;
    o.x = sm[pad(4 * v + 0)];
    o.y = sm[pad(4 * v + 1)];
    o.z = sm[pad(4 * v + 2)];
    o.w = sm[pad(4 * v + 3)];
    reinterpret_cast<uint4*>(y)[v] = o;
  }
}

template <int LOGN>
static cudaError_t multi_setup() {
  return cudaFuncSetAttribute(k_ntt_fwd_multi<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Geo<LOGN>::SMEM_WORDS * 4);
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
                             cudaStream_t st) {
  const int rows = segs.row_begin[segs.n];
  if (rows == 0) return cudaSuccess;
  const int N = 1 << logn;
  const size_t smem = (size_t)(N + N / 32) * 4;
  switch (logn) {
    case 11: k_ntt_fwd_multi<11><<<rows, N / 32, smem, st>>>(segs, tw, cc); break;
    case 12: k_ntt_fwd_multi<12><<<rows, N / 32, smem, st>>>(segs, tw, cc); break;
    case 13: k_ntt_fwd_multi<13><<<rows, N / 32, smem, st>>>(segs, tw, cc); break;
    case 14: k_ntt_fwd_multi<14><<<rows, N / 32, smem, st>>>(segs, tw, cc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fl
