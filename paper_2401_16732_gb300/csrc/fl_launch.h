// Host-side launchers of the kernels in fl_kernels.cu (internal interface
// between the C-ABI layer and the kernels; not part of the public header).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "fl_device.cuh"

namespace fl {

struct ConvDims {  // per-launch shape of the fused contraction + INTT
  int Cout, G, n_in, n_out, bands;
};

struct GeomDims {  // geometry fields the packing / extraction kernels read
  int Cin, Cout, H, W, k, s, pad, Hp, Wp, Ho, Wo, Rin, Rout, bands, P, c_n, G, n_in, n_out;
};

struct DecConst {  // exact RNS scale-and-round constants
  uint32_t q[FL_MAX_L];
  uint32_t inv[FL_MAX_L];  // (q / q_l)^-1 mod q_l
  uint64_t Qhi[FL_MAX_L], Qlo[FL_MAX_L];  // q / q_l as 128-bit
  uint64_t qhi, qlo;  // q as 128-bit
  uint32_t t;
  int L;
};

struct ModSwitchConst {  // modulus switching from L to L_out limbs
  uint32_t q[FL_MAX_L];
  uint32_t inv[FL_MAX_L][FL_MAX_L], inv_sh[FL_MAX_L][FL_MAX_L];  // q_d^-1 mod q_i (i < d), Shoup companion
  int L, L_out;
};

#define FL_STACK_MAX 64

struct StackLayer {  // one layer of a persistent stack launch
  const uint32_t* w_hat;  // [L][Cout][G][N] NTT-domain weights
  const uint32_t* c_hat;  // [B][n_in][2][L][N] NTT-domain inputs
  uint32_t* out;          // [B][n_out][2][L][N]
  const uint32_t* r;      // [B][n_out][N] masks or nullptr
  int Cout, G, n_in, n_out, bands, BB;  // BB = B * bands
  long long item_begin;   // first item of this layer in the queue
};

struct StackArgs {
  StackLayer layer[FL_STACK_MAX];
  int n_layers;
  long long n_items;
};

#ifdef __CUDACC__
// Item index of a stack queue -> (layer, image*bands + band, output channel,
// limb).  Items of a layer run limb-major, then output channel, then
// image/band, so neighbouring items share weights (over images) or inputs
// (over output channels).  Linear scan: a stack holds at most FL_STACK_MAX
// layers.
struct Item {
  int li, bb, i, l;
};

__device__ __forceinline__ int find_layer(const StackArgs& a, long long it) {
  int li = 0;
  while (li + 1 < a.n_layers && it >= a.layer[li + 1].item_begin) ++li;
  return li;
}

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
#endif

struct NttSegs {  // forward NTT of several contiguous row ranges in one launch
  const uint32_t* src[FL_STACK_MAX];
  uint32_t* dst[FL_STACK_MAX];
  int row_begin[FL_STACK_MAX + 1];
  int n;
};

#ifdef __CUDACC__
// Dispatch over the instantiated (ring degree, pass plan) pairs: CALL sees
// constexpr LG (log2 N) and R1 (first row pass radix 2^R1).  r1 = 0 picks
// the default plan; an invalid pair returns cudaErrorInvalidValue.
#define FL_PLAN_DISPATCH(logn, r1, CALL)                                              \
  do {                                                                                \
    const int r1_ = (r1) ? (r1) : default_plan_r1(logn);                              \
    switch ((logn) * 8 + r1_) {                                                       \
      case 11 * 8 + 3: { constexpr int LG = 11, R1 = 3; CALL; break; }              \
      case 12 * 8 + 3: { constexpr int LG = 12, R1 = 3; CALL; break; }              \
      case 12 * 8 + 4: { constexpr int LG = 12, R1 = 4; CALL; break; }              \
      case 13 * 8 + 3: { constexpr int LG = 13, R1 = 3; CALL; break; }              \
      case 13 * 8 + 4: { constexpr int LG = 13, R1 = 4; CALL; break; }              \
      case 13 * 8 + 5: { constexpr int LG = 13, R1 = 5; CALL; break; }              \
      case 14 * 8 + 4: { constexpr int LG = 14, R1 = 4; CALL; break; }              \
      case 14 * 8 + 5: { constexpr int LG = 14, R1 = 5; CALL; break; }              \
      default: return cudaErrorInvalidValue;                                          \
    }                                                                                 \
  } while (0)
#endif
// the default first-pass radix of each ring degree, and whether (logn, r1)
// is an instantiated plan
inline int default_plan_r1(int logn) { return logn == 11 ? 3 : logn == 14 ? 5 : 4; }
inline bool plan_available(int logn, int r1) {
  return r1 == 0 || (logn == 11 && r1 == 3) || (logn == 12 && (r1 == 3 || r1 == 4)) ||
         (logn == 13 && r1 >= 3 && r1 <= 5) || (logn == 14 && (r1 == 4 || r1 == 5));
}

cudaError_t launch_setup(int logn);
cudaError_t launch_stack_setup(int logn);
cudaError_t launch_wait_timeout_probe(unsigned long long* err, cudaStream_t st);
cudaError_t launch_ntt_multi_setup(int logn);
int stack_ctas_per_sm(int logn);
cudaError_t launch_stack(int logn, const StackArgs& a, unsigned long long* ctl, const uint32_t* tw,
                         const CtxConst& cc, int sms, cudaStream_t st);
cudaError_t launch_ntt_multi(int logn, const NttSegs& segs, const uint32_t* tw, const CtxConst& cc,
                             cudaStream_t st, int r1 = 0);
size_t twiddle_limb_words(int logn);
cudaError_t launch_ntt_fwd(int logn, int rows, const uint32_t* src, int src_per, int src_stride,
                           uint32_t* dst, int dst_per, int dst_stride, int limb_div,
                           const uint32_t* tw, const CtxConst& cc, cudaStream_t st, int r1 = 0);
cudaError_t launch_ntt_inv(int logn, int rows, uint32_t* data, const uint32_t* tw, const CtxConst& cc,
                           cudaStream_t st);
cudaError_t launch_conv_queue(int logn, const StackArgs& a, unsigned long long* ctl, const uint32_t* tw,
                              const CtxConst& cc, int sms, cudaStream_t st);
cudaError_t launch_conv_intt(int logn, int B, const ConvDims& cd, const uint32_t* w_hat,
                             const uint32_t* c_hat, uint32_t* out, const uint32_t* r,
                             const uint32_t* tw, const CtxConst& cc, cudaStream_t st, bool pdl = false);
cudaError_t launch_pmul_intt(int logn, int mode, int n, uint32_t* ws, uint32_t* ct, const uint32_t* sk,
                             const int32_t* x, const int32_t* e, const GeomDims& gd,
                             const uint32_t* tw, const CtxConst& cc, cudaStream_t st);
cudaError_t launch_dec_round(const uint32_t* ws, uint32_t* m, int n, int N, const DecConst& dc,
                             cudaStream_t st);
cudaError_t launch_noise(const uint32_t* ws, const uint32_t* m, int n, int N, const DecConst& dc, const CtxConst& cc,
                         unsigned long long* out, cudaStream_t st);
cudaError_t launch_extract(const uint32_t* m, int32_t* y, const GeomDims& g, int B, int N,
                           cudaStream_t st);
cudaError_t launch_mask(uint32_t* ct, const uint32_t* r, int n, int N, const CtxConst& cc,
                        cudaStream_t st);
cudaError_t launch_enc_online(const uint32_t* enc0, uint32_t* ct, const int32_t* x, const GeomDims& gd,
                              int n, int N, const CtxConst& cc, cudaStream_t st);
cudaError_t launch_w_scatter(const int8_t* w, uint32_t* w_hat, const GeomDims& g, int N,
                             const CtxConst& cc, cudaStream_t st);
cudaError_t launch_sk_expand(const int8_t* s, uint32_t* out, int N, const CtxConst& cc,
                             cudaStream_t st);

// modulus switching (fl_modswitch.cu)
cudaError_t launch_mod_switch(const uint32_t* in, uint32_t* out, long long rows, int N, const ModSwitchConst& mc,
                              cudaStream_t st);

// on-the-fly weights (fl_otf.cu)
cudaError_t launch_otf_setup(int logn);
cudaError_t launch_conv_otf(int logn, int B, const GeomDims& gd, const int8_t* w, const uint32_t* c_hat,
                            uint32_t* out, const uint32_t* r, const uint32_t* tw, const CtxConst& cc,
                            cudaStream_t st);

// tensor-core contraction (fl_tc.cu): NTT-domain outputs in [0, 2q), then the
// in-place inverse NTT of every output row with the mask.  kTcMaxG: the most
// input ciphertexts per band whose digit products stay exact in fp32.
constexpr int kTcMaxG = 64;
cudaError_t launch_tc_setup(int logn);
size_t conv_tc_smem_bytes();
// bytes of the tensor-core weight tiles of one layer (k_tc_weights)
size_t tc_weights_bytes(int L, int Cout, int G, int N);
cudaError_t launch_tc_weights(const uint32_t* w_hat, uint16_t* w_tc, int L, int Cout, int G, int N, cudaStream_t st);
cudaError_t launch_tc_inputs(const uint32_t* c_hat, uint32_t* c_tc, int B, int n_in, int L, int N, cudaStream_t st);
// the contraction into the scratch y_sc[l][u / 8][column * Cout + i][u % 8]
// (tc_scratch_words words), then the inverse NTT + mask of every scratch row
// into the output ciphertexts y
size_t tc_scratch_words(int B, const ConvDims& cd, int L, int N);
cudaError_t launch_conv_tc(int B, const ConvDims& cd, const uint16_t* w_tc, const uint32_t* c_hat, uint32_t* y_sc,
                           int N, const CtxConst& cc, unsigned long long* err, cudaStream_t st, bool pdl, int gpc = 0);
cudaError_t launch_intt_mask_rows(int logn, int B, const ConvDims& cd, const uint32_t* y_sc, uint32_t* y,
                                  const uint32_t* r, const uint32_t* tw, const CtxConst& cc, cudaStream_t st, bool pdl,
                                  int r1 = 0);
// direct form (fl_direct.cu)
cudaError_t launch_direct_setup(int logn);
cudaError_t launch_direct(int logn, int B, const GeomDims& g, const int8_t* w, const uint32_t* ct, uint32_t* out,
                          const uint32_t* r, const CtxConst& cc, cudaStream_t st);

// x^2 + x protocol and batch encoding (fl_act.cu)
cudaError_t launch_act_setup(int logn);
cudaError_t launch_batch_decode(int logn, int n, const uint32_t* m, uint32_t* slots, const uint32_t* tw_t,
                                const LimbConst& tc, cudaStream_t st);
cudaError_t launch_batch_encode(int logn, int n, const uint32_t* slots, uint32_t scale, uint32_t* dst,
                                long long dst_stride, int lift_L, const uint32_t* tw_t, const LimbConst& tc,
                                const CtxConst& cc, cudaStream_t st);
cudaError_t launch_x2x_const(const uint32_t* r, const uint32_t* v, uint32_t* dst, long long dst_stride, int n, int N,
                             const LimbConst& tc, cudaStream_t st);
cudaError_t launch_x2x_round1(int logn, int n, const uint32_t* prep, const uint32_t* ct, uint32_t* out,
                              const uint32_t* tw, const CtxConst& cc, cudaStream_t st);
cudaError_t launch_x2x_round2(const uint32_t* prep, const uint32_t* X, const uint32_t* Y, uint32_t* out, int n,
                              int N, const CtxConst& cc, cudaStream_t st);
cudaError_t launch_repack(const uint32_t* src, uint32_t* dst, const GeomDims& pv, const GeomDims& nx, int B, int N,
                          cudaStream_t st);

}  // namespace fl
