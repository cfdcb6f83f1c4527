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
//   k_conv_tc          one CTA per (8-32 slots, 16 output channels, limb):
//                      weights staged once, then every group of 8 columns;
//                      each warp takes its slots in turn over all K steps;
//                      writes the NTT-domain outputs, reduced to [0, q)
//   k_intt_mask_rows   in-place inverse NTT of every output row, + Delta*r
//                      on component 0 (the encoded weights carry N^-1, so the
//                      transform is the unscaled one)
#include <cuda_runtime.h>

#include "fl_device.cuh"
#include "fl_launch.h"

namespace fl {

namespace {
constexpr int TC_ROWS = 16;        // output channels per CTA (the MMA's M)
constexpr int TC_COLS = 8;         // (image/band, component) columns per column group
constexpr int TC_GK = 8;           // input ciphertexts per K step: 8 x 4 weight bytes = 32
constexpr int TC_N = 7 * TC_COLS;  // (column, shift) pairs: 56, i.e. 7 n-tiles of 8
constexpr int TC_WARPS = 8;
constexpr int TC_THREADS = 32 * TC_WARPS;
constexpr int TC_WROW = 24;        // row stride of a staged weight: 16 rows + 8 words of padding
constexpr int TC_MAX_DYN_SMEM = 226 * 1024;  // dynamic shared memory limit, 1 KB below the CTA maximum

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

// Dynamic shared memory of k_conv_tc<SPW> for Gp = G rounded up to 8, in words:
//   Wst [U][Gp][24]    weights of the CTA's 16 output channels (rows 16..23 padding)
//   Xst [U][Gp][8]     inputs of one column group
//   Ys  [8][16][57]    one slot's seven shift sums per warp
//   Ot  [16][8][U + 4] reduced NTT-domain outputs of the column group
// with U = 8 * SPW slots.  The weight layout puts the 32 lanes' A-fragment
// words (g = 8k + t, row = grp or grp + 8) in 32 different banks.
__host__ __device__ constexpr size_t tc_smem_words(int spw, int gp) {
  return (size_t)8 * spw * gp * TC_WROW + (size_t)8 * spw * gp * TC_COLS + (size_t)TC_WARPS * TC_ROWS * (TC_N + 1) +
         (size_t)TC_ROWS * TC_COLS * (8 * spw + 4);
}
}  // namespace

// Grid (N / U, ceil(Cout / 16), L), U = 8 * SPW slots per CTA; every CTA
// loops over the column groups of 8 (image/band, component) columns, with
// its weights staged once.  Warp w takes slots w*SPW .. w*SPW + SPW - 1 in
// turn, each over all K steps.
template <int SPW>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(const uint32_t* __restrict__ w_hat,
                                                         const uint32_t* __restrict__ c_hat,
                                                         uint32_t* __restrict__ y_hat, ConvDims cd, int B, int N,
                                                         CtxConst cc) {
  constexpr int U = 8 * SPW, U4 = U / 4, UP = U + 4;  // UP: padded row of Ot
  extern __shared__ __align__(16) uint32_t tsm[];
  const int Gp = (cd.G + TC_GK - 1) / TC_GK * TC_GK;
  uint32_t* Wst = tsm;                                            // [U][Gp][24]
  uint32_t* Xst = Wst + (size_t)U * Gp * TC_WROW;                 // [U][Gp][8]
  int* Ys = reinterpret_cast<int*>(Xst + (size_t)U * Gp * TC_COLS);  // [8][16][57]
  uint32_t* Ot = reinterpret_cast<uint32_t*>(Ys + TC_WARPS * TC_ROWS * (TC_N + 1));  // [16][8][UP]
  const int L = cc.L;
  const int u0 = blockIdx.x * U, i0 = blockIdx.y * TC_ROWS, l = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, grp = lane >> 2, t = lane & 3;
  const size_t ct_words = (size_t)2 * L * N;
  const LimbConst lc = cc.limb[l];
  const uint32_t c40 = red64((uint64_t)lc.r32 << 8, lc);  // 2^40 mod q
  const int cols = 2 * B * cd.bands;

  // weights: Wst[uu][g][ii] = W[l][i0 + ii][g][u0 + uu], zero outside the
  // layer.  Each thread owns one (row, 4-slot group) and walks g; no index
  // division by a runtime value.
  {
    constexpr int WP = TC_ROWS * U4, WS = TC_THREADS / WP;
    const int ii = tid % TC_ROWS, q4 = (tid / TC_ROWS) % U4, gs = tid / WP;
    const int i = i0 + ii;
    const uint4* src = reinterpret_cast<const uint4*>(w_hat + ((size_t)l * cd.Cout + (i < cd.Cout ? i : 0)) * cd.G * N + u0) + q4;
    uint32_t* d = Wst + (size_t)(4 * q4) * Gp * TC_WROW + ii;
    for (int g = gs; g < Gp; g += WS) {
      uint4 w = make_uint4(0, 0, 0, 0);
      if (i < cd.Cout && g < cd.G) w = __ldg(src + (size_t)g * (N / 4));
      d[g * TC_WROW] = w.x;
      d[(Gp + g) * TC_WROW] = w.y;
      d[(2 * Gp + g) * TC_WROW] = w.z;
      d[(3 * Gp + g) * TC_WROW] = w.w;
    }
  }
  __shared__ long long colbase[TC_COLS];  // output offset of each column of the group, row i0 excluded
  const size_t rowstride = (size_t)cd.bands * 2 * L * N;  // between output channels i and i + 1

  for (int chunk = 0; chunk * TC_COLS < cols; ++chunk) {
    const int ncols = min(TC_COLS, cols - chunk * TC_COLS);
    const int ntiles = (7 * ncols + 7) / 8;
    const unsigned rc = (65536u + ncols - 1) / ncols;  // (p * rc) >> 16 == p / ncols for p < 128
    __syncthreads();  // the weights are staged; the previous group's Xst and Ot are no longer read
    // inputs: Xst[uu][g][cl] = X[g][column chunk*8 + cl][u0 + uu], zero
    // outside; each thread owns one (column, 4-slot group) and walks g
    {
      constexpr int XP = TC_COLS * U4, XS = TC_THREADS / XP;
      const int cl = tid % TC_COLS, q4 = (tid / TC_COLS) % U4, gs = tid / XP;
      const int col = chunk * TC_COLS + cl, bb = col >> 1, c = col & 1;
      const int b = bb / cd.bands, band = bb - b * cd.bands;  // one division per thread and group
      const bool ok = cl < ncols;
      const uint4* src = reinterpret_cast<const uint4*>(
          c_hat + (ok ? ((size_t)b * cd.n_in + (size_t)band * cd.G) * ct_words + (size_t)c * L * N : 0) +
          (size_t)l * N + u0) + q4;
      uint32_t* d = Xst + (size_t)(4 * q4) * Gp * TC_COLS + cl;
      for (int g = gs; g < Gp; g += XS) {
        uint4 x = make_uint4(0, 0, 0, 0);
        if (ok && g < cd.G) x = __ldg(src + (size_t)g * (ct_words / 4));
        d[g * TC_COLS] = x.x;
        d[(Gp + g) * TC_COLS] = x.y;
        d[(2 * Gp + g) * TC_COLS] = x.z;
        d[(3 * Gp + g) * TC_COLS] = x.w;
      }
      if (tid < TC_COLS)
        colbase[cl] = ok ? (long long)(((size_t)b * cd.n_out + band) * 2 * L * N + (size_t)c * L * N + (size_t)l * N +
                                       u0 + (size_t)i0 * rowstride)
                         : 0;
    }
    __syncthreads();
    int* ys = Ys + warp * TC_ROWS * (TC_N + 1);
#pragma unroll 1
    for (int sl = 0; sl < SPW; ++sl) {
      const int uu = warp * SPW + sl;
      const uint32_t* ws = Wst + (size_t)uu * Gp * TC_WROW;
      const uint32_t* xs = Xst + (size_t)uu * Gp * TC_COLS;
      int acc[7][4];
#pragma unroll
      for (int j = 0; j < 7; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0;
#pragma unroll 1
      for (int g0 = 0; g0 < Gp; g0 += TC_GK) {
        // A fragment: rows grp, grp+8; K columns 4t..4t+3 (g = g0+t) and 16+4t.. (g = g0+4+t)
        const uint32_t* w0 = ws + (g0 + t) * TC_WROW;
        const uint32_t* w1 = ws + (g0 + 4 + t) * TC_WROW;
        const uint32_t a[4] = {w0[grp], w0[grp + 8], w1[grp], w1[grp + 8]};
        const uint32_t* x0 = xs + (g0 + t) * TC_COLS;
        const uint32_t* x1 = xs + (g0 + 4 + t) * TC_COLS;
#pragma unroll
        for (int j = 0; j < 7; ++j) {
          if (j < ntiles) {  // warp-uniform
            // B fragment: column n = 8j + grp of the tile, K rows as for A
            const int n = 8 * j + grp, cl = n / 7, s = n % 7;
            mma_u8(acc[j], a, digit_window(x0[cl], s), digit_window(x1[cl], s));
          }
        }
      }
      // accumulators -> ys[row][n]: c0, c1 at row grp, c2, c3 at row grp + 8; n = 8j + 2t + {0, 1}
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        if (j < ntiles) {
          ys[grp * (TC_N + 1) + 8 * j + 2 * t] = acc[j][0];
          ys[grp * (TC_N + 1) + 8 * j + 2 * t + 1] = acc[j][1];
          ys[(grp + 8) * (TC_N + 1) + 8 * j + 2 * t] = acc[j][2];
          ys[(grp + 8) * (TC_N + 1) + 8 * j + 2 * t + 1] = acc[j][3];
        }
      }
      __syncwarp();
      // Y = sum_s 2^(8s) Y_s mod q for the 16 x ncols outputs (lanes on valid
      // pairs only): Y_0..Y_4 by shifts, plus ((Y_5 + 2^8 Y_6) mod q) *
      // (2^40 mod q), one reduction.  With Y_s < 4 * 192 * 255^2 < 2^26 (G at
      // most 192, the shared-memory limit) the first part stays below 2^59
      // and the second below 2^60.
      for (int p = lane; p < TC_ROWS * ncols; p += 32) {
        const int ii = (int)(((unsigned)p * rc) >> 16), cl = p - ii * ncols;  // p / ncols, p < 128
        const int* v = ys + ii * (TC_N + 1) + 7 * cl;
        uint64_t lo = 0;
#pragma unroll
        for (int s = 0; s < 5; ++s) lo += (uint64_t)(uint32_t)v[s] << (8 * s);
        const uint64_t hi = (uint64_t)(uint32_t)v[5] + ((uint64_t)(uint32_t)v[6] << 8);
        Ot[(ii * TC_COLS + cl) * UP + uu] = red64(lo + (uint64_t)red64(hi, lc) * c40, lc);
      }
      __syncwarp();  // ys is rewritten by the next slot
    }
    __syncthreads();
    // rows (i, column) of the group: U consecutive slots each, as 16-byte stores
    for (int e = tid; e < TC_ROWS * TC_COLS * U4; e += TC_THREADS) {
      const int q4 = e % U4, cl = (e / U4) % TC_COLS, ii = e / (U4 * TC_COLS);
      if (i0 + ii < cd.Cout && cl < ncols)
        reinterpret_cast<uint4*>(y_hat + colbase[cl] + (size_t)ii * rowstride)[q4] =
            reinterpret_cast<const uint4*>(Ot + (ii * TC_COLS + cl) * UP)[q4];
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

// Slots per warp for a layer: the most (4, 2) that still lets two CTAs share
// an SM (113 KB of shared memory each), else 1.
static int tc_spw(int G) {
  const int gp = (G + TC_GK - 1) / TC_GK * TC_GK;
  for (int spw = 4; spw > 1; spw /= 2)
    if (tc_smem_words(spw, gp) * 4 <= 113 * 1024) return spw;
  return 1;
}

size_t conv_tc_smem_bytes(int G) {
  const int gp = (G + TC_GK - 1) / TC_GK * TC_GK;
  return tc_smem_words(tc_spw(G), gp) * 4;
}

template <int SPW>
static cudaError_t conv_tc(int B, const ConvDims& cd, const uint32_t* w_hat, const uint32_t* c_hat, uint32_t* y_hat,
                           int N, const CtxConst& cc, cudaStream_t st) {
  const int gp = (cd.G + TC_GK - 1) / TC_GK * TC_GK;
  const size_t smem = tc_smem_words(SPW, gp) * 4;
  const dim3 grid(N / (8 * SPW), (cd.Cout + TC_ROWS - 1) / TC_ROWS, cc.L);
  k_conv_tc<SPW><<<grid, TC_THREADS, smem, st>>>(w_hat, c_hat, y_hat, cd, B, N, cc);
  return cudaGetLastError();
}

cudaError_t launch_conv_tc(int B, const ConvDims& cd, const uint32_t* w_hat, const uint32_t* c_hat, uint32_t* y_hat,
                           int N, const CtxConst& cc, cudaStream_t st) {
  if (B == 0 || cd.Cout == 0) return cudaSuccess;
  if ((cd.Cout + TC_ROWS - 1) / TC_ROWS > 65535 || conv_tc_smem_bytes(cd.G) > TC_MAX_DYN_SMEM)
    return cudaErrorInvalidConfiguration;
  switch (tc_spw(cd.G)) {
    case 4: return conv_tc<4>(B, cd, w_hat, c_hat, y_hat, N, cc, st);
    case 2: return conv_tc<2>(B, cd, w_hat, c_hat, y_hat, N, cc, st);
    default: return conv_tc<1>(B, cd, w_hat, c_hat, y_hat, N, cc, st);
  }
}

template <int LOGN>
static cudaError_t intt_rows_setup() {
  return cudaFuncSetAttribute(k_intt_mask_rows<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              padded_words(1 << LOGN) * 4);
}

cudaError_t launch_tc_setup(int logn) {
  // the contraction kernels may use up to the per-CTA maximum of shared
  // memory less 1 KB kept for their static part (the column offsets)
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_conv_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_MAX_DYN_SMEM)) ||
      (e = cudaFuncSetAttribute(k_conv_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_MAX_DYN_SMEM)) ||
      (e = cudaFuncSetAttribute(k_conv_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_MAX_DYN_SMEM)))
    return e;
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
