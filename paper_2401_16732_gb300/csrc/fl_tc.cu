// Byte-split tensor-core form of the per-slot contraction (Algorithm 1's
// sum over input ciphertexts, evaluated in the NTT domain), beside the plain
// CUDA-core form of fl_kernels.cu.  sm_103a has no integer kind of tcgen05,
// so the products run on the warp-level integer MMA
// (mma.sync m16n8k32, u8 x u8 -> s32), which is exact by construction.
//
// For limb l and slot u the contraction is a small integer matrix product
//   Y[i][col] = sum_g W[i][g] * X[g][col]  (mod q_l),   col = (image, band, component).
// Every residue (< 2^30) is split into its 4 bytes, W = sum_a W_a 2^(8a) and
// X = sum_d X_d 2^(8d).  The weight byte index goes into K and the digit
// shift s = a + d into N:
//   A[i][(g, a)]       = W_a[i][g]
//   B[(g, a)][(col, s)] = X_(s-a)[g][col]   (0 outside 0 <= s-a <= 3)
//   Y_s[i][col]        = sum_(g, a) A * B = sum_g sum_(a+d=s) W_a X_d
// and Y = sum_(s=0..6) 2^(8s) Y_s.  Every partial sum is at most
// 4 * G * 255^2 < 2^31, so the s32 accumulation is exact.  With K = (g, a)
// in the order of the residue's bytes, a thread's A fragment registers are
// the weight residues themselves, and a B fragment register is a
// byte-reversed, shifted window of an input residue.
//
//   k_conv_tc          one CTA per (8 slots, 16 output channels, limb,
//                      8 columns); one warp per slot; writes the NTT-domain
//                      outputs, reduced to [0, q)
//   k_intt_mask_rows   in-place inverse NTT of every output row, + Delta*r
//                      on component 0 (the encoded weights carry N^-1, so the
//                      transform is the unscaled one)
#include <cuda_runtime.h>

#include "fl_device.cuh"
#include "fl_launch.h"

namespace fl {

namespace {
constexpr int TC_SLOTS = 8;        // slots per CTA, one per warp
constexpr int TC_ROWS = 16;        // output channels per CTA (the MMA's M)
constexpr int TC_COLS = 8;         // (image/band, component) columns per CTA
constexpr int TC_GK = 8;           // input ciphertexts per K step: 8 x 4 weight bytes = 32
constexpr int TC_N = 7 * TC_COLS;  // (column, shift) pairs: 56, i.e. 7 n-tiles of 8
constexpr int TC_THREADS = 32 * TC_SLOTS;

// Bytes [x_s, x_(s-1), x_(s-2), x_(s-3)] of x (x_j its byte j; 0 outside 0..3):
// rows (g, a = 0..3) of B's column (col, s).
__device__ __forceinline__ uint32_t digit_window(uint32_t x, int s) {
  const uint32_t r = __byte_perm(x, 0, 0x0123);  // x_3 x_2 x_1 x_0
  return s <= 3 ? r >> (8 * (3 - s)) : r << (8 * (s - 3));
}

__device__ __forceinline__ void mma_u8(int (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
}  // namespace

// Grid (N / 8, ceil(Cout / 16), L * ceil(2 * B * bands / 8)).
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(const uint32_t* __restrict__ w_hat,
                                                         const uint32_t* __restrict__ c_hat,
                                                         uint32_t* __restrict__ y_hat, ConvDims cd, int B, int N,
                                                         CtxConst cc) {
  __shared__ uint32_t Wst[TC_ROWS][TC_GK][TC_SLOTS];
  __shared__ uint32_t Xst[TC_GK][TC_COLS][TC_SLOTS];
  __shared__ int Ys[TC_SLOTS][TC_ROWS][TC_N + 1];
  __shared__ uint32_t Ot[TC_ROWS][TC_COLS][TC_SLOTS];
  const int L = cc.L;
  const int u0 = blockIdx.x * TC_SLOTS, i0 = blockIdx.y * TC_ROWS;
  const int l = blockIdx.z % L, chunk = blockIdx.z / L;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, grp = lane >> 2, t = lane & 3;
  const int ncols = min(TC_COLS, 2 * B * cd.bands - chunk * TC_COLS);  // >= 1 by the grid
  const int ntiles = (7 * ncols + 7) / 8;
  const size_t ct_words = (size_t)2 * L * N;
  const LimbConst lc = cc.limb[l];

  int acc[7][4];
#pragma unroll
  for (int j = 0; j < 7; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0;

  for (int g0 = 0; g0 < cd.G; g0 += TC_GK) {
    __syncthreads();  // the previous K step's operands are no longer read
    for (int e = tid; e < TC_ROWS * TC_GK * TC_SLOTS; e += TC_THREADS) {
      const int uu = e % TC_SLOTS, gg = (e / TC_SLOTS) % TC_GK, ii = e / (TC_SLOTS * TC_GK);
      const int i = i0 + ii, g = g0 + gg;
      Wst[ii][gg][uu] =
          (i < cd.Cout && g < cd.G) ? __ldg(w_hat + (((size_t)l * cd.Cout + i) * cd.G + g) * N + u0 + uu) : 0u;
    }
    for (int e = tid; e < TC_GK * TC_COLS * TC_SLOTS; e += TC_THREADS) {
      const int uu = e % TC_SLOTS, cl = (e / TC_SLOTS) % TC_COLS, gg = e / (TC_SLOTS * TC_COLS);
      const int g = g0 + gg, col = chunk * TC_COLS + cl;
      uint32_t x = 0;
      if (g < cd.G && cl < ncols) {
        const int bb = col >> 1, c = col & 1, b = bb / cd.bands, band = bb % cd.bands;
        x = __ldg(c_hat + ((size_t)b * cd.n_in + (size_t)band * cd.G + g) * ct_words + (size_t)c * L * N +
                  (size_t)l * N + u0 + uu);
      }
      Xst[gg][cl][uu] = x;
    }
    __syncthreads();
    // A fragment: rows grp, grp+8; K columns 4t..4t+3 (g = t) and 16+4t.. (g = 4+t)
    const uint32_t a[4] = {Wst[grp][t][warp], Wst[grp + 8][t][warp], Wst[grp][4 + t][warp],
                           Wst[grp + 8][4 + t][warp]};
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      if (j < ntiles) {  // warp-uniform
        // B fragment: column n = 8j + grp of the tile, K rows as for A
        const int n = 8 * j + grp, cl = n / 7, s = n % 7;
        mma_u8(acc[j], a, digit_window(Xst[t][cl][warp], s), digit_window(Xst[4 + t][cl][warp], s));
      }
    }
  }

  // accumulators -> Ys[slot][row][n]: c0, c1 at row grp, c2, c3 at row grp + 8; n = 8j + 2t + {0, 1}
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    if (j < ntiles) {
      Ys[warp][grp][8 * j + 2 * t] = acc[j][0];
      Ys[warp][grp][8 * j + 2 * t + 1] = acc[j][1];
      Ys[warp][grp + 8][8 * j + 2 * t] = acc[j][2];
      Ys[warp][grp + 8][8 * j + 2 * t + 1] = acc[j][3];
    }
  }
  __syncwarp();
  // recombine Y = sum_s 2^(8s) Y_s mod q: Y_0..Y_4 by shifts below 2^64, then
  // (Y_5 + 2^8 Y_6) * (2^40 mod q)
  const uint32_t c40 = red64((uint64_t)lc.r32 << 8, lc);
  for (int p = lane; p < TC_ROWS * TC_COLS; p += 32) {
    const int ii = p / TC_COLS, cl = p % TC_COLS;
    uint32_t y = 0;
    if (cl < ncols) {
      const int* ys = &Ys[warp][ii][7 * cl];
      uint64_t lo = 0;
#pragma unroll
      for (int s = 0; s < 5; ++s) lo += (uint64_t)(uint32_t)ys[s] << (8 * s);
      const uint64_t hi = (uint64_t)(uint32_t)ys[5] + ((uint64_t)(uint32_t)ys[6] << 8);
      y = csub(red64(lo, lc) + red64((uint64_t)red64(hi, lc) * c40, lc), lc.q);
    }
    Ot[ii][cl][warp] = y;
  }
  __syncthreads();
  for (int e = tid; e < TC_ROWS * TC_COLS * TC_SLOTS; e += TC_THREADS) {
    const int uu = e % TC_SLOTS, cl = (e / TC_SLOTS) % TC_COLS, ii = e / (TC_SLOTS * TC_COLS);
    const int i = i0 + ii, col = chunk * TC_COLS + cl;
    if (i < cd.Cout && cl < ncols) {
      const int bb = col >> 1, c = col & 1, b = bb / cd.bands, band = bb % cd.bands;
      const size_t oct = (size_t)b * cd.n_out + (size_t)i * cd.bands + band;
      y_hat[(oct * 2 + c) * L * N + (size_t)l * N + u0 + uu] = Ot[ii][cl][uu];
    }
  }
}

// Row r = (oct * 2 + c) * L + l of y (NTT domain, values in [0, q)) becomes
// N times its inverse transform, + Delta_l * r[oct] when c == 0 and r is set.
template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 32, minb_one_poly<LOGN>())
    k_intt_mask_rows(uint32_t* __restrict__ y, const uint32_t* __restrict__ r, const uint32_t* __restrict__ tw,
                     CtxConst cc) {
  constexpr int N = 1 << LOGN, T = N / 32;
  extern __shared__ uint32_t sm[];
  const int L = cc.L;
  const size_t row = blockIdx.x;
  const int l = (int)(row % L), c = (int)((row / L) % 2);
  const size_t oct = row / (2 * (size_t)L);
  const LimbConst lc = cc.limb[l];
  uint32_t* p = y + row * N;
  for (int v = threadIdx.x; v < N / 4; v += T)
    *reinterpret_cast<uint4*>(sm + pad(4 * v)) = reinterpret_cast<const uint4*>(p)[v];
  __syncthreads();  // the whole row is in shared memory before any of it is overwritten
  intt_from_smem_unscaled<LOGN>(sm, tw + (size_t)l * TwLayout<LOGN>::LIMB_WORDS, lc, threadIdx.x,
                                MaskStore{p, (r && c == 0) ? r + oct * N : nullptr, lc});
}

cudaError_t launch_conv_tc(int B, const ConvDims& cd, const uint32_t* w_hat, const uint32_t* c_hat, uint32_t* y_hat,
                           int N, const CtxConst& cc, cudaStream_t st) {
  const long long cols = 2LL * B * cd.bands;
  if (cols == 0 || cd.Cout == 0) return cudaSuccess;
  const long long chunks = (cols + TC_COLS - 1) / TC_COLS;
  const dim3 grid(N / TC_SLOTS, (cd.Cout + TC_ROWS - 1) / TC_ROWS, (unsigned)(cc.L * chunks));
  if (grid.y > 65535 || cc.L * chunks > 65535) return cudaErrorInvalidConfiguration;
  k_conv_tc<<<grid, TC_THREADS, 0, st>>>(w_hat, c_hat, y_hat, cd, B, N, cc);
  return cudaGetLastError();
}

template <int LOGN>
static cudaError_t intt_rows_setup() {
  return cudaFuncSetAttribute(k_intt_mask_rows<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              padded_words(1 << LOGN) * 4);
}

cudaError_t launch_tc_setup(int logn) {
  switch (logn) {
    case 11: return intt_rows_setup<11>();
    case 12: return intt_rows_setup<12>();
    case 13: return intt_rows_setup<13>();
    case 14: return intt_rows_setup<14>();
  }
  return cudaErrorInvalidValue;
}

template <int LOGN>
static cudaError_t intt_rows(long long rows, uint32_t* y, const uint32_t* r, const uint32_t* tw, const CtxConst& cc,
                             cudaStream_t st) {
  constexpr int N = 1 << LOGN;
  k_intt_mask_rows<LOGN><<<(unsigned)rows, N / 32, (size_t)padded_words(N) * 4, st>>>(y, r, tw, cc);
  return cudaGetLastError();
}

cudaError_t launch_intt_mask_rows(int logn, long long rows, uint32_t* y, const uint32_t* r, const uint32_t* tw,
                                  const CtxConst& cc, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  switch (logn) {
    case 11: return intt_rows<11>(rows, y, r, tw, cc, st);
    case 12: return intt_rows<12>(rows, y, r, tw, cc, st);
    case 13: return intt_rows<13>(rows, y, r, tw, cc, st);
    case 14: return intt_rows<14>(rows, y, r, tw, cc, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fl
