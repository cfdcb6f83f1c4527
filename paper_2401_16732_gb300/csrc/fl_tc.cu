// Tensor-core form of the per-slot contraction (Algorithm 1's sum over input
// ciphertexts, evaluated in the NTT domain), beside the plain CUDA-core form
// of fl_kernels.cu.  It runs on the 5th-generation tensor cores (tcgen05.mma
// kind::f16, accumulators in tensor memory).  sm_103a has no integer kind of
// tcgen05, so the integers are carried exactly in fp16 with fp32
// accumulation.
//
// For limb l and slot u the contraction is a small matrix product mod q_l:
//   Y[i][col] = sum_g W[i][g] * X[g][col]   (mod q),  col = (image, band, component).
// Balanced base-256 digits.  A value v < 0x7F7F7F80 (so that v + 0x80808080
// does not wrap) is v = sum_a d_a(v) 256^a with d_a(v) = byte_a(v +
// 0x80808080) - 128 in [-128, 127]; every digit is exact in fp16.  The
// weights and inputs are residues below q < 2^30; X'_a = 256^a X mod q
// (a = 0..3) is a Shoup product of X < q, which lies below 1.25 q (the
// quotient estimate is one short only when the remainder is below X / 2^32
// of q), so every value split here is in range.
//   W X = sum_a d_a(W) 256^a X = sum_a d_a(W) X'_a  (mod q)
//       = sum_e 256^e P_e,   P_e = sum_(g, a) d_a(W[g]) d_e(X'_a[g]).
// So per slot one matrix product with K = (g, a) (4G) and N = (col, e) (4 per
// column) gives four partial sums P_e per output.  |P_e| <= 4G * 128^2 =
// G * 2^16 <= 2^22 for G <= 64, so every fp32 partial sum is an exact integer.
// Every accumulator starts at 3 * 2^22 (written into tensor memory before
// each group), which keeps every partial sum in [2^23, 2^24]: the fp32 bit
// pattern minus 0x4B400000 is then P_e itself.
// Recombination mod q on the CUDA cores: Y = sum_e 256^e P_e (|Y| < 2^46.1)
// is known exactly mod 2^32 from the bit patterns; its quotient k =
// round(Y / q) comes from an fp32 estimate of Y (error below 2^23.6, and
// every prime of a context lies above 2^29, so k is within 0.53 of Y / q),
// and Y - k q + q lies in [0, 2q), the input range of the inverse NTT,
// computed exactly in 32-bit arithmetic.
//
//   k_tc_weights   (offline) the encoded weights as fp16 digit tiles in the
//                  MMA's shared-memory layout, 16 KB per K step
//   k_tc_inputs    the NTT images of the inputs re-laid in slot groups of 4
//   k_conv_tc      one CTA per SM and (128 output channels, 16 columns, limb,
//                  run of 16 groups of 4 slots), warp-specialised: one warp
//                  bulk-copies each K step's weight tile into its operand
//                  stage (cp.async.bulk, completion on an mbarrier); 8
//                  producer warps split the inputs into fp16 digit tiles
//                  (4-byte cp.async ring -> canonical K-major layout); one
//                  MMA warp issues 4 MMAs M128 N64 K16 per K step, one per
//                  slot, into one of two tensor-memory accumulator buffers;
//                  8 epilogue warps load the accumulators, recombine, store
//                  the NTT-domain outputs in [0, 2q) into a scratch buffer
//                  in slot-tiled order and reset the buffer to the bias;
//                  every hand-off an mbarrier with a bounded wait
//   k_intt_mask_rows   inverse NTT of every output row, gathered from the
//                  scratch, + Delta*r on component 0, written to the output
//                  ciphertexts (the encoded weights carry N^-1, so the
//                  transform is the unscaled one)
//
// The scratch order, y_sc[l][u / 8][R][u % 8] with R = column * Cout + i for
// output channel i and column (image, band, component): a CTA's group pair
// (8 slots) of 128 channels x 16 columns lands as 16 runs of 4 KB.  Written
// straight into the output rows ([b][oct][c][l][u]) the same results are
// 32-byte pieces of 2048 rows 256-512 KB apart, and those scattered writes
// bounded the kernel at small G (no stores at all: 1.8x faster there).  The
// price is on the inverse NTT's side: each thread gathers its 32
// coefficients as four 32-byte pieces.
#include <cuda_runtime.h>

#include "fl_device.cuh"
#include "fl_launch.h"

namespace fl {

namespace {
constexpr int TC_M = 128;             // output channels per CTA (MMA M = tensor-memory lanes)
constexpr int TC_CW = 16;             // columns per CTA; MMA N = 4 * 16 = 64 (column, digit e)
constexpr int TC_NN = 4 * TC_CW;
constexpr int TC_U = 4;               // slots per group: one accumulator buffer of 4 x 64 columns
constexpr int TC_GS = 4;              // input ciphertexts per K step: 4 x 4 weight digits = K 16
constexpr int TC_PROD_WARPS = 8;      // input copies + digit conversion into the B tiles
constexpr int TC_EPI_WARPS = 8;       // recombination, two per tensor-memory lane quadrant
constexpr int TC_MMA_WARP = TC_PROD_WARPS + TC_EPI_WARPS;  // one warp issues the MMAs,
constexpr int TC_LOAD_WARP = TC_MMA_WARP + 1;              // one the bulk copies of the weight tiles
constexpr int TC_THREADS = 32 * (TC_LOAD_WARP + 1);        // 576
constexpr int TC_RING = 6;            // raw-input ring depth, in K steps
constexpr int TC_NS = 6;              // operand stages (weight tile + input tile)
// slot groups per CTA (the tile's length along the slots): 4, 8, 16, 32 or 64, a
// template parameter of k_conv_tc chosen per workload (even: the epilogue
// stores groups in pairs)
constexpr int TC_GPC_DEFAULT = 32;
constexpr int TC_TMEM_COLS = 2 * TC_U * TC_NN;  // 512: two accumulator buffers
// shared-memory layout (bytes)
constexpr int RAWB_STEP = TC_CW * TC_GS * 16;      // [image/band][g][component][4 slots]
constexpr int TILEA_SLOT = TC_M * 32;              // 128 rows x 16 halves
constexpr int TILEA_STEP = TC_U * TILEA_SLOT;      // one weight tile: 16 KB, one bulk copy
constexpr int TILEB_SLOT = TC_NN * 32 + 16;        // 64 rows x 16 halves, +16 B against bank conflicts
constexpr int STAGE_BYTES = TILEA_STEP + TC_U * TILEB_SLOT;
constexpr int OFF_TILE = 0;
constexpr int OFF_RAWB = OFF_TILE + TC_NS * STAGE_BYTES;
constexpr int OFF_HOLD = OFF_RAWB + TC_RING * RAWB_STEP;  // epilogue: even group's results [col][slot][thread]
constexpr int TC_SMEM = OFF_HOLD + (TC_CW / 2) * TC_U * 32 * TC_EPI_WARPS * 4;
static_assert(STAGE_BYTES % 16 == 0 && OFF_HOLD % 16 == 0, "bulk copies and vector accesses stay 16-byte aligned");
// more than half of the SM's shared memory: one CTA per SM, which then owns
// all of tensor memory
static_assert(TC_SMEM > 116 * 1024 && TC_SMEM <= 220 * 1024, "one CTA per SM with room for the static part");
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;  // 2 s bound on every wait
constexpr uint32_t FP_BIAS = 0x4B400000u;                 // bits of 3 * 2^22 in fp32

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor, no swizzle: start address,
// leading byte offset (between core matrices along K), stride byte offset
// (between 8-row groups along M or N), version bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: D f32 (bits 4-5 = 1), A and B f16
// (bits 7-9, 10-12 = 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on bar once every tcgen05 operation issued so far by this thread is done
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {  // one whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // the allocating warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes visible to the tensor core's (async-proxy) reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive tensor-memory columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
// the same 16 columns set to one value
__device__ __forceinline__ void tmem_st16_const(uint32_t taddr, uint32_t x) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(x)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n}" ::"r"(su32(bar))
               : "memory");
}
// Wait for the phase of the given parity; false after 2 s.  Each try_wait
// suspends the warp in hardware for up to 20 us unless the phase completes
// first, so waiting warps take no issue slots from the working ones.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  const unsigned long long t0 = gtimer();
  for (unsigned polls = 0; polls < (1u << 20); ++polls) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    if (done) return true;
    if (gtimer() - t0 > TC_WAIT_NS) return false;
  }
  return false;
}

// arrive on bar and announce `bytes` more bytes of transactions for its
// current phase (the bulk copy that follows completes them)
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes)
               : "memory");
}
// bulk copy (no tensor map) of `bytes` contiguous bytes global -> shared,
// completed on bar; both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(su32(bar)), "l"(pol)
      : "memory");
}
// 4-byte cp.async through L1 (the only form of that size), same policy operand
__device__ __forceinline__ void cp4_pol(uint32_t dst, const void* src, uint32_t src_bytes, uint64_t pol) {
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2, %3;" ::"r"(dst), "l"(src),
               "r"(src_bytes), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// fp16 pair (byte_lo - 128, byte_hi - 128) from two biased bytes placed in
// bytes 0 and 2 of t (bytes 1 and 3 are overwritten): 0x64xx is 1024 + xx
__device__ __forceinline__ uint32_t digits2(uint32_t t) {
  const uint32_t h = (t & 0x00FF00FFu) | 0x64006400u;
  uint32_t r;
  asm("sub.f16x2 %0, %1, %2;" : "=r"(r) : "r"(h), "r"(0x64806480u));  // - (1152, 1152)
  return r;
}
// the four balanced digits of v (< 2^31) as fp16, in K order a = 0..3
__device__ __forceinline__ uint2 digits4(uint32_t v) {
  const uint32_t y = v + 0x80808080u;
  // bytes (0, 1) into positions 0 and 2, then bytes (2, 3)
  return make_uint2(digits2(__byte_perm(y, 0, 0x0100)), digits2(__byte_perm(y, 0, 0x0302)));
}

// Y - k q + q in [0, 2q) for Y = sum_e 256^e P_e, from the accumulator bit
// patterns b[e] = bits(3 * 2^22 + P_e), b[e] in [2^23, 2^24].  The fp32
// estimate of Y leaves out 256^0 P_0 (|P_0| <= 2^22) and takes the biases of
// e = 1..3 out first: b[3] 2^24 - 3 * 2^22 (2^8 + 2^16 + 2^24) is exact (the
// constant has 18 significant bits, the difference is a multiple of 2^24
// below 2^46.1), and the two fmas that add b[2] 2^16 and b[1] 2^8 round by at
// most 2^22 each.  So the estimate is within 2^23.6 of Y, i.e. within
// 0.021 q for q > 2^29, and with the final rounding to an integer (0.5) and
// the rounding of 1/q (below 0.005 at |Y / q| < 2^16.1), k is within 0.53 of
// Y / q.
__device__ __forceinline__ uint32_t recombine(const uint32_t* b, float qinv, uint32_t nq, uint32_t c) {
  constexpr float kBias123 = (float)(12582912.0 * 16843008.0);  // exact
  const float y = fmaf(__uint_as_float(b[1]), 256.f,
                       fmaf(__uint_as_float(b[2]), 65536.f, fmaf(__uint_as_float(b[3]), 16777216.f, -kBias123)));
  const uint32_t kb = __float_as_uint(fmaf(y, qinv, 12582912.f));  // FP_BIAS + round(Y / q)
  const uint32_t lo = b[0] + (b[1] << 8) + (b[2] << 16) + (b[3] << 24);  // Y + FP_BIAS * 0x01010101 mod 2^32
  return kb * nq + lo + c;
}
}  // namespace

// Grid (mtiles * nchunks, N / (4 * GPC), L): blockIdx.x picks the 128
// output channels and 16 columns (fastest, so CTAs sharing input slots run
// together), blockIdx.y the run of GPC groups of 4 slots, blockIdx.z the
// limb.  Step t of the CTA is (group t / nch, K step t % nch) with nch =
// ceil(G / 4) K steps per group.
// Warp roles (every hand-off an mbarrier with a bounded wait):
//   load warp (1 thread) tile_empty -> bulk copy of the weight tile into stage
//                        t % TC_NS, completing a_full
//   producers (8 warps)  tile_empty -> raw input ring -> fp16 input tile of
//                        stage t % TC_NS, arrive tile_full
//   MMA warp (1 thread)  a_full + tile_full -> 4 MMAs into accumulator buffer
//                        grp % 2 -> commit to tile_empty (and to acc_full
//                        after a group)
//   epilogue (8 warps)   acc_full -> tensor-memory loads -> recombination ->
//                        stores of the NTT-domain outputs -> bias written
//                        back into the buffer -> arrive acc_empty
template <int GPC>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv_tc(const uint16_t* __restrict__ w_tc, const uint32_t* __restrict__ c_hat, uint32_t* __restrict__ y_sc,
              ConvDims cd, int B, int N, CtxConst cc, unsigned long long* err) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  __shared__ uint64_t a_full[TC_NS], tile_full[TC_NS], tile_empty[TC_NS], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  __shared__ long long colrow[TC_CW];  // scratch row R of each column at output channel 0; -1 outside
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cols = 2 * B * cd.bands, mtiles = (cd.Cout + TC_M - 1) / TC_M;
  const int mt = blockIdx.x % mtiles, i0 = mt * TC_M, col0 = (blockIdx.x / mtiles) * TC_CW;
  static_assert(GPC % 2 == 0, "the epilogue stores groups in pairs");
  const int l = blockIdx.z, grp0 = blockIdx.y * GPC, L = cc.L, G = cd.G;
  const LimbConst lc = cc.limb[l];
  const size_t R_total = (size_t)cols * cd.Cout;  // scratch rows
  const int nch = (G + TC_GS - 1) / TC_GS, T = GPC * nch;
  const uint32_t sb = su32(tsm);

  if (warp == 0) tmem_alloc(&tmem_base, TC_TMEM_COLS);
  if (tid == 0) {
    for (int k = 0; k < TC_NS; ++k) {
      mbar_init(&a_full[k], 1);                 // the weight tile's bulk copy
      mbar_init(&tile_full[k], TC_PROD_WARPS);  // the input tile: one arrival per producer warp
      mbar_init(&tile_empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&acc_full[k], 1);
      mbar_init(&acc_empty[k], TC_EPI_WARPS);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < TC_CW) {
    const int colg = col0 + tid;
    colrow[tid] = colg < cols ? (long long)colg * cd.Cout : -1;
  }
  pdl_wait();  // the inputs come from the preceding forward NTT
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_trigger();
  const uint32_t tbase = tmem_base;

  if (warp < TC_PROD_WARPS) {
    // ------------------------------------------------------------ producers
    const int pt = tid;  // 0..255
    // The input tiles.  Raw words of each K step go into ring slot
    // t % TC_RING by 4-byte cp.async (c_tc[l][u / 4][b][ct][c][4]): column
    // pt >> 4 (image/band (pt >> 5), component (pt >> 4) & 1), slot
    // (pt >> 2) & 3, ciphertext pt & 3, so a warp reads 128 contiguous bytes;
    // outside the layer the copies fill zeros.  Every producer thread
    // converts exactly the word it copied itself, so it waits only for its
    // own copy groups and the producers need no barrier among themselves.
    const int bc_col = pt >> 4, bc_s = (pt >> 2) & 3, bc_g = pt & 3;
    const uint32_t b_off = ((((bc_col >> 1) * TC_GS + bc_g) * 2 + (bc_col & 1)) * 4 + bc_s) * 4;  // bytes in a step
    bool b_ok;
    const uint32_t* b_src = c_hat;
    {
      const int colg = col0 + bc_col, bb = colg >> 1, b = bb / cd.bands, band = bb - b * cd.bands;
      b_ok = colg < cols;
      if (b_ok)
        b_src = c_hat + (((size_t)l * (N / 4) * B + b) * cd.n_in + (size_t)band * G + bc_g) * 8 + (colg & 1) * 4 + bc_s;
    }
    const size_t b_grp = (size_t)B * cd.n_in * 8;  // words of one 4-slot group of the inputs
    // the inputs are read once per output-channel tile, by CTAs that run
    // together (evict last)
    const uint64_t pol_x = policy_evict_last();
    int it = 0, ich = 0, igrp = grp0;  // the next step to copy: K step ich of group igrp
    auto issue = [&]() {
      if (it < T) {
        const int g0 = TC_GS * ich;
        const bool ok = b_ok && g0 + bc_g < G;
        cp4_pol(sb + OFF_RAWB + (it % TC_RING) * RAWB_STEP + b_off,
                ok ? b_src + igrp * b_grp + (size_t)g0 * 8 : c_hat, ok ? 4 : 0, pol_x);
        ++it;
        if (++ich == nch) {
          ich = 0;
          ++igrp;
        }
      }
      cp_commit();
    };
    const uint32_t q = lc.q;
    const uint32_t w1s = (uint32_t)((256ull << 32) / q), w2s = (uint32_t)((65536ull << 32) / q),
                   w3s = (uint32_t)((16777216ull << 32) / q);
    bool aborted = false;
#pragma unroll 1
    for (int t = 0; t < TC_RING - 1; ++t) issue();
#pragma unroll 1
    for (int t = 0; t < T; ++t) {
      const int st = t % TC_NS, r = t % TC_RING;
      // stage st was last read by the MMAs of step t - TC_NS; the decision
      // to stop is the warp's, so that no lane is left at __syncwarp
      if (__any_sync(0xffffffffu, !mbar_wait_bounded(&tile_empty[st], ((t / TC_NS) & 1) ^ 1))) {
        aborted = true;
        break;
      }
      cp_wait<TC_RING - 2>();  // this thread's copy of step t has landed
      issue();                 // step t + TC_RING - 1, into the ring slot this thread emptied at step t - 1
      // B: rows (col, e), K (g, a) of slot bc_s
      const uint32_t x = *reinterpret_cast<const uint32_t*>(tsm + OFF_RAWB + r * RAWB_STEP + b_off);
      // (the copies filled zeros beyond G, and the digits of 0 are zeros)
      const uint32_t y0 = x + 0x80808080u;
      const uint32_t y1 = shoup_mul(x, 256u, w1s, q) + 0x80808080u;  // X'_a < 1.25 q, congruent to 256^a X
      const uint32_t y2 = shoup_mul(x, 65536u, w2s, q) + 0x80808080u;
      const uint32_t y3 = shoup_mul(x, 16777216u, w3s, q) + 0x80808080u;
      uint2 dd[4];
#pragma unroll
      for (int e = 0; e < 4; ++e)
        dd[e] = make_uint2(digits2(__byte_perm(y0, y1, e | ((4 + e) << 8))),
                           digits2(__byte_perm(y2, y3, e | ((4 + e) << 8))));
      uint8_t* tb = tsm + OFF_TILE + st * STAGE_BYTES + TILEA_STEP + bc_s * TILEB_SLOT + (bc_g >> 1) * 128 +
                    (bc_g & 1) * 8;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = 4 * bc_col + e;
        *reinterpret_cast<uint2*>(tb + (row >> 3) * 256 + (row & 7) * 16) = dd[e];
      }
      // every lane's tile writes visible to the tensor core, then one
      // arrival per warp
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tile_full[st]);
    }
    cp_wait<0>();
    if (aborted) s_abort = 1;
  } else if (warp == TC_LOAD_WARP) {
    // ------------------------------------------------------------ weight tiles
    // k_tc_weights stored every (limb, output-channel tile, 4-slot group,
    // K step) as the 16 KB weight tile of one stage, in the MMA's shared-
    // memory layout, and a CTA's steps as consecutive tiles: one bulk copy
    // per step, read once (evict first).
    if (lane == 0) {
      const uint64_t pol_w = policy_evict_first();
      const uint8_t* src =
          reinterpret_cast<const uint8_t*>(w_tc) + (((size_t)l * mtiles + mt) * (N / 4) + grp0) * nch * TILEA_STEP;
      int t = 0;
#pragma unroll 1
      for (; t < T; ++t) {
        const int st = t % TC_NS;
        if (!mbar_wait_bounded(&tile_empty[st], ((t / TC_NS) & 1) ^ 1)) {
          s_abort = 1;
          break;
        }
        mbar_arrive_expect_tx(&a_full[st], TILEA_STEP);
        bulk_g2s(sb + OFF_TILE + st * STAGE_BYTES, src + (size_t)t * TILEA_STEP, TILEA_STEP, &a_full[st], pol_w);
      }
      // no copy may still be writing when the CTA exits: wait for the last
      // one into every stage (earlier ones completed before their stage was
      // reused)
#pragma unroll 1
      for (int k = t > TC_NS ? t - TC_NS : 0; k < t; ++k)
        if (!mbar_wait_bounded(&a_full[k % TC_NS], (k / TC_NS) & 1)) s_abort = 1;
    }
  } else if (warp == TC_MMA_WARP) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
#pragma unroll 1
      for (int t = 0; t < T; ++t) {
        const int st = t % TC_NS, ch = t % nch, grp = t / nch, ab = grp & 1;
        // use grp >> 1 of buffer ab needs the epilogue's arrival number
        // grp >> 1 (the first one: the bias written before any group)
        if (ch == 0 && !mbar_wait_bounded(&acc_empty[ab], (grp >> 1) & 1)) {
          s_abort = 1;
          break;
        }
        if (!mbar_wait_bounded(&a_full[st], (t / TC_NS) & 1) || !mbar_wait_bounded(&tile_full[st], (t / TC_NS) & 1)) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t ta = sb + OFF_TILE + st * STAGE_BYTES, tb = ta + TILEA_STEP;
#pragma unroll
        for (int s = 0; s < TC_U; ++s)
          mma_f16(tbase + (ab * TC_U + s) * TC_NN, smem_desc(ta + s * TILEA_SLOT, 128, 256),
                  smem_desc(tb + s * TILEB_SLOT, 128, 256), idesc_f16(TC_M, TC_NN), 1u);  // onto the bias
        mma_commit(&tile_empty[st]);
        if (ch == nch - 1) mma_commit(&acc_full[ab]);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int qd = warp & 3;                          // tensor-memory lane quadrant: the warp index mod 4
    const int hc = (warp - TC_PROD_WARPS) >> 2;       // columns 8 hc .. 8 hc + 7
    const int rrow = 32 * qd + lane;
    const bool row_ok = i0 + rrow < cd.Cout;
    const float qinv = 1.0f / (float)lc.q;
    const uint32_t nq = 0u - lc.q, cfix = FP_BIAS * lc.q + lc.q - FP_BIAS * 0x01010101u;
    const uint32_t ta = tbase + ((uint32_t)(32 * qd) << 16);
    // Groups come in pairs (8 slots, one 32-byte sector of every output row):
    // the even group's results wait in shared memory for the odd one's.
    constexpr int HS = 32 * TC_EPI_WARPS;  // hold[local column][epilogue thread], the 4 slots of a group
    uint4* hold = reinterpret_cast<uint4*>(tsm + OFF_HOLD) + (tid - 32 * TC_PROD_WARPS);
    // this lane's output channel; a group pair's 8 slots are 8 words of row R
    uint32_t* scr = y_sc + (size_t)l * (N / 8) * R_total * 8 + (size_t)(i0 + rrow) * 8;
    // Every accumulator of a buffer starts at 3 * 2^22: this warp writes the
    // bias into its lanes and columns (column chunk p of every slot) once it
    // has read them, and hands the buffer back to the MMA warp.
    auto bias = [&](int ab, int p) {
#pragma unroll
      for (int s = 0; s < TC_U; ++s) tmem_st16_const(ta + (ab * TC_U + s) * TC_NN + 4 * (8 * hc + 4 * p), FP_BIAS);
    };
    auto release = [&](int ab) {
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);  // one arrival per epilogue warp
    };
#pragma unroll
    for (int ab = 0; ab < 2; ++ab) {
#pragma unroll
      for (int p = 0; p < TC_CW / 8; ++p) bias(ab, p);
      release(ab);
    }
#pragma unroll 1
    for (int grp = 0; grp < GPC; ++grp) {
      const int ab = grp & 1;
      const size_t u8 = (size_t)(grp0 + grp) >> 1;  // the group pair's 8 slots
      // the decision to stop is the warp's: the tensor-memory loads below are
      // warp-collective
      if (__any_sync(0xffffffffu, !mbar_wait_bounded(&acc_full[ab], (grp >> 1) & 1))) {
        s_abort = 1;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int p = 0; p < TC_CW / 8; ++p) {  // columns 8 hc + 4p .. + 3
        uint32_t v[TC_U][16];
#pragma unroll
        for (int s = 0; s < TC_U; ++s) tmem_ld16(ta + (ab * TC_U + s) * TC_NN + 4 * (8 * hc + 4 * p), v[s]);
        tmem_wait_ld();
#pragma unroll
        for (int cc2 = 0; cc2 < 4; ++cc2) {
          const int cl = 4 * p + cc2, c = 8 * hc + cl;
          uint32_t o[TC_U];
#pragma unroll
          for (int s = 0; s < TC_U; ++s) o[s] = recombine(&v[s][4 * cc2], qinv, nq, cfix);
          if (ab == 0) {
            hold[cl * HS] = make_uint4(o[0], o[1], o[2], o[3]);
          } else {
            const long long cr = colrow[c];
            if (row_ok && cr >= 0) {
              uint4* dst = reinterpret_cast<uint4*>(scr + (u8 * R_total + (size_t)cr) * 8);
              __stcs(dst, hold[cl * HS]);
              __stcs(dst + 1, make_uint4(o[0], o[1], o[2], o[3]));
            }
          }
        }
        bias(ab, p);  // this chunk's accumulators have been read
      }
      release(ab);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (s_abort && tid == 0) atomicOr(err, 1ull);
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, TC_TMEM_COLS);
  }
}

// Scratch row R = column * Cout + i (column = (image, band, component)) of
// limb l = blockIdx.y, NTT domain with values in [0, 2q), in the order
// y_sc[l][u / 8][R][u % 8], becomes N times its inverse transform, + Delta_l
// * r[oct] when the component is 0 and r is set, in the output row
// (b, oct = i * bands + band, component, l) of y.  Grid (R_total, L): the
// CTAs that run together read neighbouring rows, so each 8-slot piece they
// gather is part of a contiguous run.
template <int LOGN, int R1>
__global__ void __launch_bounds__((1 << LOGN) / 32, minb_one_poly<LOGN>())
    k_intt_mask_rows(const uint32_t* __restrict__ y_sc, uint32_t* __restrict__ y, const uint32_t* __restrict__ r,
                     const uint32_t* __restrict__ tw, int Cout, int bands, int n_out, CtxConst cc) {
  constexpr int N = 1 << LOGN;
  extern __shared__ uint32_t sm[];
  const int L = cc.L, l = blockIdx.y;
  const size_t R = blockIdx.x, R_total = gridDim.x;
  const int colg = (int)(R / Cout), i = (int)(R - (size_t)colg * Cout);
  const int c = colg & 1, bb = colg >> 1, b = bb / bands, band = bb - b * bands;
  const size_t oct = (size_t)b * n_out + (size_t)i * bands + band;  // output ciphertext, image-major
  const LimbConst lc = cc.limb[l];
  uint32_t* p = y + ((oct * 2 + c) * L + l) * N;
  pdl_wait();
  // the first (radix-32) pass gathers its coefficients from the scratch
  intt_from_smem_unscaled<LOGN, MaskStore, R1>(sm, tw + (size_t)l * TwLayout<LOGN>::LIMB_WORDS, lc, threadIdx.x,
                                               MaskStore{p, (r && c == 0) ? r + oct * N : nullptr, lc},
                                               y_sc + ((size_t)l * (N / 8) * R_total + R) * 8, R_total * 8);
}

// The encoded weights as k_conv_tc's weight tiles: for every limb l,
// output-channel tile mt (128 rows), 4-slot group u4 and K step kc (input
// ciphertexts 4 kc .. 4 kc + 3), one 16 KB tile of fp16 digits in the MMA's
// shared-memory layout, tiles ordered [l][mt][u4][kc].  Within a tile, slot
// s = u % 4 takes 4 KB; row r, K index k = 4 (g % 4) + a (digit a of
// ciphertext g) sits in core matrix (r / 8, k / 8) at byte ((r / 8) * 2 +
// k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.  Rows beyond Cout and
// ciphertexts beyond G are zeros.  One thread per (tile, 16-byte chunk of a
// slot), for the 4 slots: it reads 4 consecutive slots of 2 ciphertexts.
__global__ void k_tc_weights(const uint32_t* __restrict__ w_hat, uint16_t* __restrict__ w_tc, int Cout, int G, int N,
                             int mtiles, int nch, long long total) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int c = (int)(e & 255);  // chunk (r / 8, kh, r % 8) of a slot
  long long rest = e >> 8;
  const int kc = (int)(rest % nch);
  rest /= nch;
  const int u4 = (int)(rest % (N / 4));
  rest /= N / 4;
  const int mt = (int)(rest % mtiles), l = (int)(rest / mtiles);
  const int kh = (c >> 3) & 1, i = mt * TC_M + (c >> 4) * 8 + (c & 7);
  uint2 d[2][TC_U];
#pragma unroll
  for (int gl = 0; gl < 2; ++gl) {
    const int g = TC_GS * kc + 2 * kh + gl;
    uint4 v = make_uint4(0, 0, 0, 0);  // the digits of 0 are zeros
    if (i < Cout && g < G) v = *reinterpret_cast<const uint4*>(w_hat + (((size_t)l * Cout + i) * G + g) * N + 4 * u4);
    d[gl][0] = digits4(v.x);
    d[gl][1] = digits4(v.y);
    d[gl][2] = digits4(v.z);
    d[gl][3] = digits4(v.w);
  }
  uint4* dst = reinterpret_cast<uint4*>(w_tc + ((((size_t)l * mtiles + mt) * (N / 4) + u4) * nch + kc) * (TILEA_STEP / 2));
#pragma unroll
  for (int s = 0; s < TC_U; ++s)
    dst[s * (TILEA_SLOT / 16) + c] = make_uint4(d[0][s].x, d[0][s].y, d[1][s].x, d[1][s].y);
}

size_t tc_scratch_words(int B, const ConvDims& cd, int L, int N) { return (size_t)2 * B * cd.bands * cd.Cout * L * N; }

size_t tc_weights_bytes(int L, int Cout, int G, int N) {
  return (size_t)L * ((Cout + TC_M - 1) / TC_M) * (N / 4) * ((G + TC_GS - 1) / TC_GS) * TILEA_STEP;
}

cudaError_t launch_tc_weights(const uint32_t* w_hat, uint16_t* w_tc, int L, int Cout, int G, int N, cudaStream_t st) {
  if (G < 1 || G > kTcMaxG) return cudaErrorInvalidValue;
  const int mtiles = (Cout + TC_M - 1) / TC_M, nch = (G + TC_GS - 1) / TC_GS;
  const long long total = (long long)L * mtiles * (N / 4) * nch * 256;
  if (total == 0) return cudaSuccess;
  const long long blocks = (total + 255) / 256;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  k_tc_weights<<<(unsigned)blocks, 256, 0, st>>>(w_hat, w_tc, Cout, G, N, mtiles, nch, total);
  return cudaGetLastError();
}

// Slot-tiled copy of the NTT-domain inputs for k_conv_tc: c_tc[l][u / 4][b][ct][c][j]
// = c_hat[b][ct][c][l][u] with u = 4 (u / 4) + j, so that one K step of one
// CTA reads its 4 ciphertexts x 2 components of an image as one 128-byte run.
// One thread per (l, b, ct, 4-slot group, c); neighbouring threads take the
// two components, so each writes half of one 32-byte sector.
__global__ void k_tc_inputs(const uint32_t* __restrict__ c_hat, uint32_t* __restrict__ c_tc, int n_in, int L, int N,
                            long long total) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int c = (int)(e & 1), ng = N / 4;
  const long long rest = e >> 1;
  const int grp = (int)(rest % ng);
  const long long bct = rest / ng;  // (b * L + l) * n_in + ct
  const long long lb = bct / n_in;
  const int ct = (int)(bct % n_in);
  const int l = (int)(lb % L);
  const long long b = lb / L;
  const uint4 v = reinterpret_cast<const uint4*>(c_hat + (((b * n_in + ct) * 2 + c) * L + l) * (long long)N)[grp];
  const long long B = total / ((long long)2 * ng * n_in * L);
  reinterpret_cast<uint4*>(c_tc)[(((l * (long long)ng + grp) * B + b) * n_in + ct) * 2 + c] = v;
}

cudaError_t launch_tc_inputs(const uint32_t* c_hat, uint32_t* c_tc, int B, int n_in, int L, int N, cudaStream_t st) {
  const long long total = (long long)B * n_in * L * 2 * (N / 4);
  if (total == 0) return cudaSuccess;
  const long long blocks = (total + 255) / 256;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  k_tc_inputs<<<(unsigned)blocks, 256, 0, st>>>(c_hat, c_tc, n_in, L, N, total);
  return cudaGetLastError();
}

size_t conv_tc_smem_bytes() { return TC_SMEM; }

static cudaLaunchConfig_t pdl_config(dim3 grid, dim3 block, size_t smem, cudaStream_t st, cudaLaunchAttribute* at,
                                     bool pdl) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cfg;
}

// pdl: the previous operation in `st` is the forward NTT of these inputs.
// gpc: slot groups per CTA (4, 8, 16, 32 or 64; 0 = the default).
cudaError_t launch_conv_tc(int B, const ConvDims& cd, const uint16_t* w_tc, const uint32_t* c_hat, uint32_t* y_sc,
                           int N, const CtxConst& cc, unsigned long long* err, cudaStream_t st, bool pdl, int gpc) {
  if (B == 0 || cd.Cout == 0) return cudaSuccess;
  if (cd.G < 1 || cd.G > kTcMaxG) return cudaErrorInvalidValue;
  if (gpc == 0) gpc = TC_GPC_DEFAULT;
  if (gpc != 4 && gpc != 8 && gpc != 16 && gpc != 32 && gpc != 64) return cudaErrorInvalidValue;
  const long long mtiles = (cd.Cout + TC_M - 1) / TC_M, nchunks = (2LL * B * cd.bands + TC_CW - 1) / TC_CW;
  if (mtiles * nchunks > 0x7fffffffLL || N % (4 * gpc) != 0) return cudaErrorInvalidConfiguration;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = pdl_config(dim3((unsigned)(mtiles * nchunks), N / (4 * gpc), cc.L), dim3(TC_THREADS),
                                      TC_SMEM, st, at, pdl);
  switch (gpc) {
    case 4: return cudaLaunchKernelEx(&cfg, k_conv_tc<4>, w_tc, c_hat, y_sc, cd, B, N, cc, err);
    case 8: return cudaLaunchKernelEx(&cfg, k_conv_tc<8>, w_tc, c_hat, y_sc, cd, B, N, cc, err);
    case 32: return cudaLaunchKernelEx(&cfg, k_conv_tc<32>, w_tc, c_hat, y_sc, cd, B, N, cc, err);
    case 64: return cudaLaunchKernelEx(&cfg, k_conv_tc<64>, w_tc, c_hat, y_sc, cd, B, N, cc, err);
    default: return cudaLaunchKernelEx(&cfg, k_conv_tc<16>, w_tc, c_hat, y_sc, cd, B, N, cc, err);
  }
}

template <int LOGN>
static cudaError_t intt_rows_setup() {
  cudaError_t e = cudaSuccess;
  for (int r1 = 3; r1 <= 5; ++r1) {  // every instantiated pass plan
    if (!plan_available(LOGN, r1)) continue;
    FL_PLAN_DISPATCH(LOGN, r1, (e = cudaFuncSetAttribute(k_intt_mask_rows<LG, R1>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         padded_words(1 << LG) * 4)));
    if (e) return e;
  }
  return e;
}

cudaError_t launch_tc_setup(int logn) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_conv_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM)) ||
      (e = cudaFuncSetAttribute(k_conv_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM)) ||
      (e = cudaFuncSetAttribute(k_conv_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM)) ||
      (e = cudaFuncSetAttribute(k_conv_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM)) ||
      (e = cudaFuncSetAttribute(k_conv_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM)))
    return e;
  switch (logn) {
    case 11: return intt_rows_setup<11>();
    case 12: return intt_rows_setup<12>();
    case 13: return intt_rows_setup<13>();
    case 14: return intt_rows_setup<14>();
  }
  return cudaErrorInvalidValue;
}

// pdl: the previous operation in `st` is the contraction that wrote y.
cudaError_t launch_intt_mask_rows(int logn, int B, const ConvDims& cd, const uint32_t* y_sc, uint32_t* y,
                                  const uint32_t* r, const uint32_t* tw, const CtxConst& cc, cudaStream_t st, bool pdl,
                                  int r1) {
  const long long rows = 2LL * B * cd.bands * cd.Cout;  // scratch rows per limb
  if (rows == 0) return cudaSuccess;
  if (rows > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  cudaLaunchAttribute at[1];
  cudaError_t e = cudaSuccess;
  FL_PLAN_DISPATCH(logn, r1, {
    cudaLaunchConfig_t cfg = pdl_config(dim3((unsigned)rows, cc.L), dim3((1 << LG) / 32),
                                        (size_t)padded_words(1 << LG) * 4, st, at, pdl);
    e = cudaLaunchKernelEx(&cfg, k_intt_mask_rows<LG, R1>, y_sc, y, r, tw, cd.Cout, cd.bands, cd.n_out, cc);
  });
  return e;
}

}  // namespace fl
