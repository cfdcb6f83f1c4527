/*
 * flashgpu: GB300 (sm_103a) library for the server-side hot path of the Flash
 * hybrid private-inference protocol (arXiv 2401.16732): homomorphic
 * convolution of BFV/RLWE ciphertexts holding direct-encoded activations by
 * plaintext integer CNN filters, followed by the random-mask addition that
 * turns each output ciphertext into additive secret shares.
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Ring R_q = Z_q[x]/(x^N + 1), N in {2048, 4096, 8192, 16384}; q is held as
 *   L <= 4 RNS primes q_0 > ... > q_{L-1}, the largest primes below 2^30 with
 *   q_l = 1 mod 2N (Sec. 2.2, Table 1 use a single q; the RNS split is this
 *   library's representation of it).  Plaintext modulus t (65537 in the
 *   workloads), Delta = floor(q / t) (Table 1).
 * - A ciphertext array is uint32 [n][2][L][N]: ciphertext, component c0/c1,
 *   limb, coefficient; canonical residues in [0, q_l); coefficient domain.
 * - Pointers named *_dev are CUDA device pointers on the device that was
 *   current when the context was created; the caller owns and allocates them.
 *   Host pointers are named *_host.  `stream` is a cudaStream_t (NULL = the
 *   legacy default stream); work is enqueued asynchronously on it and the
 *   call returns before it completes.
 * - Return value: 0 on success, a negative FL_ERR_* code otherwise; no device
 *   work is enqueued when an argument check fails.  fl_last_error() gives a
 *   thread-local message for the last failure on the calling thread.
 * - Nothing here falls back to the CPU: without a CUDA device every compute
 *   call fails with FL_ERR_CUDA.
 *
 * Layout of one convolution layer (fl_conv_geom) follows Sec. 3.3 and
 * Algorithm 1: the client zero-pads each H x W channel to Hp x Wp
 * (Hp = H + 2 pad), direct-encodes it (Eq. 1) and packs c_n = floor(N / P)
 * padded planes of P = Rin * Wp coefficients per ciphertext, channel j in
 * ciphertext j / c_n at offset (j mod c_n) * P.  A plane larger than N is cut
 * into `bands` row bands of Rin padded rows (Rout output rows each); each band
 * is its own set of G = ceil(Cin / c_n) input ciphertexts (index band*G + g).
 * The output is one ciphertext per output channel and band (index
 * i*bands + band, Sec. 3.3: no output packing); output pixel (oy, ox) of band
 * b sits at coefficient (s * (oy - b*Rout)) * Wp + s * ox.
 */
#ifndef FLASHGPU_H
#define FLASHGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FL_OK 0
#define FL_ERR_ARG (-1)   /* null pointer, size out of range, short workspace */
#define FL_ERR_SHAPE (-2) /* geometry that the packing cannot represent */
#define FL_ERR_CUDA (-3)  /* a CUDA runtime call failed (message has the reason) */
#define FL_ERR_OOM (-4)   /* the context's own tables could not be allocated */
#define FL_ERR_TIMEOUT (-5) /* a bounded device-side wait gave up (kernel returned early) */
#define FL_MAX_LIMBS 4

typedef struct fl_ctx fl_ctx; /* opaque: parameters + device twiddle tables */

typedef struct fl_conv_geom {
  int32_t N, Cin, Cout, H, W, k, stride, pad;
  int32_t Hp, Wp, Ho, Wo;   /* padded input and output sizes */
  int32_t Rin, Rout, bands; /* padded rows per ct, output rows per band */
  int32_t P, c_n, G;        /* plane size, channels per ct, cts per band */
  int32_t n_in, n_out;      /* input cts per image (bands*G), output cts (Cout*bands) */
} fl_conv_geom;

/* Thread-local message describing the last failing call on this thread. */
const char *fl_last_error(void);

/* Fill *out with the ciphertext layout of a k x k convolution (stride, pad)
 * from Cin to Cout channels on an H x W input at ring degree N (Sec. 3.3,
 * Algorithm 1; readings: tap step ky*Wp + kx, channel offset (j mod c_n)*P,
 * c_n = floor(N/P), row bands when Hp*Wp > N).  Pure host code.
 * FL_ERR_SHAPE if a padded row band of k rows does not fit in N. */
int fl_conv_geom_make(int N, int Cin, int Cout, int H, int W, int k, int stride, int pad,
                      fl_conv_geom *out);

/* Create a context on the current CUDA device: find the L primes, a
 * primitive 2N-th root of unity per prime, the NTT twiddle tables (allocated
 * on the device and owned by the context) and the per-limb constants
 * (Delta mod q_l, N^-1, CRT constants for decryption).  When t is prime with
 * t = 1 mod 2N it also builds the tables of t for batch encoding.  1 <= L <=
 * 4, 3 <= t < 2^20 odd.  N and L outside the supported set: FL_ERR_ARG. */
int fl_ctx_create(int N, int L, uint32_t t, fl_ctx **out);
/* Free the context and its device tables (the caller has synchronised). */
void fl_ctx_destroy(fl_ctx *ctx);
/* Copy out the primes [L], Delta mod q_l [L] and psi_l [L] (the primitive
 * 2N-th roots the NTT uses); any output pointer may be NULL. */
int fl_ctx_params(const fl_ctx *ctx, uint32_t *primes_host, uint32_t *delta_host,
                  uint32_t *psi_host);

/* ---- Row a1: client side (key, packing, private-key encryption) ---- */

/* Secret key: s_dev int8 [N] ternary (Table 2's s(x)); writes its NTT image
 * sk_dev uint32 [L][N] (the form every other key argument takes). */
int fl_keygen(fl_ctx *ctx, const int8_t *s_dev, uint32_t *sk_dev, void *stream);

/* Pack and encrypt B images (Sec. 3.3 packing, Eq. 1, Table 2 private-key
 * encryption): c0 = [-(a*s + e) + Delta*m]_q, c1 = a, where m is the
 * direct-encoded zero-padded input.  x_dev int32 [B][Cin][H][W] with values
 * in [0, t); a_dev uint32 [B][n_in][L][N] uniform residues; e_dev int32
 * [B][n_in][N] noise (|e| < 2^20); ct_dev uint32 [B][n_in][2][L][N] output. */
int fl_encrypt(fl_ctx *ctx, const uint32_t *sk_dev, const fl_conv_geom *geom, int B,
               const int32_t *x_dev, const uint32_t *a_dev, const int32_t *e_dev,
               uint32_t *ct_dev, void *stream);

/* Algorithm 2 (online encryption): ct = Enc(0) + Delta*m.  enc0_dev holds
 * pre-computed encryptions of zero [B][n_in][2][L][N]; x_dev as in
 * fl_encrypt; ct_dev may alias enc0_dev. */
int fl_encrypt_online(fl_ctx *ctx, const fl_conv_geom *geom, int B, const int32_t *x_dev,
                      const uint32_t *enc0_dev, uint32_t *ct_dev, void *stream);

/* Decrypt n ciphertexts (Appendix A: Delta*m + v = [c1*s + c0]_q, m =
 * round(t/q * [c1*s + c0]_q) mod t, exact RNS scale-and-round): ct_dev
 * [n][2][L][N] -> m_dev uint32 [n][N] in [0, t).  workspace: at least
 * fl_decrypt_workspace_bytes(ctx, n) device bytes. */
size_t fl_decrypt_workspace_bytes(const fl_ctx *ctx, int n);
int fl_decrypt(fl_ctx *ctx, const uint32_t *sk_dev, int n, const uint32_t *ct_dev,
               uint32_t *m_dev, void *workspace_dev, size_t workspace_bytes, void *stream);

/* Test hook on the noise of decryption (Appendix A: c0 + c1*s = Delta*m + v
 * mod q, decryption correct while the noise v stays small): for n
 * ciphertexts ct_dev [n][2][L][N] under the key sk_dev and their expected
 * messages m_dev uint32 [n][N] in [0, t), *max_noise_host receives the
 * largest |v| over every coefficient, v taken centred in (-q/2, q/2] (a
 * double: exact below 2^53).  workspace: fl_noise_workspace_bytes(ctx, n)
 * device bytes.  Synchronises `stream`. */
size_t fl_noise_workspace_bytes(const fl_ctx *ctx, int n);
int fl_noise_inf(fl_ctx *ctx, const uint32_t *sk_dev, int n, const uint32_t *ct_dev, const uint32_t *m_dev,
                 void *workspace_dev, size_t workspace_bytes, void *stream, double *max_noise_host);

/* Ciphertext words between the caller's host buffer and device memory of
 * the context's device (`words` 32-bit words, e.g. n*2*L*N for n
 * ciphertexts): the client's side of the exchange (Sec. 5.2: the client
 * sends encrypted inputs, the server returns masked ciphertexts).  Enqueued
 * on `stream`; asynchronous when the host buffer is pinned.  FL_ERR_ARG
 * when dev is not device memory of the context's device, or host is. */
int fl_copy_to_device(fl_ctx *ctx, const uint32_t *host, uint32_t *dev, size_t words, void *stream);
int fl_copy_to_host(fl_ctx *ctx, const uint32_t *dev, uint32_t *host, size_t words, void *stream);

/* Read the convolution outputs out of decrypted output polynomials:
 * m_dev uint32 [B][n_out][N] -> y_dev int32 [B][Cout][Ho][Wo]. */
int fl_extract_outputs(const fl_conv_geom *geom, int B, const uint32_t *m_dev,
                       int32_t *y_dev, void *stream);

/* ---- Row a2: server-side weight encoding (offline) ---- */

/* Size in bytes of the encoded weights of one layer: L*Cout*G*N*4. */
size_t fl_weights_bytes(const fl_ctx *ctx, const fl_conv_geom *geom);

/* Encode filters w_dev int8 [Cout][Cin][k][k] as the NTT images of the
 * weight polynomials W_{i,g}(x) = sum_{j in g} sum_{ky,kx} w[i][j][ky][kx] *
 * x^-(ky*Wp + kx + (j mod c_n)*P) -- Algorithm 1's DRot/CMult sequence for
 * output channel i folded into one plaintext (Eq. 2: DRot(c, e) = c*x^-e).
 * Each image is multiplied by N^-1 mod q_l, which the convolution's inverse
 * NTT then leaves out.  w_hat_dev uint32 [L][Cout][G][N] (fl_weights_bytes
 * bytes). */
int fl_encode_weights(fl_ctx *ctx, const fl_conv_geom *geom, const int8_t *w_dev,
                      uint32_t *w_hat_dev, void *stream);

/* ---- Rows a3-a6: the hot path ---- */

/* Workspace of fl_he_conv2d / fl_he_conv2d_mask: the NTT images of the input
 * ciphertexts, B*n_in*2*L*N*4 bytes. */
size_t fl_he_conv2d_workspace_bytes(const fl_ctx *ctx, const fl_conv_geom *geom, int B);

/* Homomorphic convolution (Algorithm 1, evaluated as y_{i,band} =
 * sum_g W_{i,g} * ct_{band*G+g} in R_q): forward NTT of the inputs into the
 * workspace (a3), per-slot contraction mod q_l with lazy 64-bit accumulation
 * (a4, Sec. 6.1) fused with the inverse NTT of each output (a5; the factor
 * N^-1 comes with the encoded weights).  The fused kernel is launched as a
 * programmatic dependent of the input NTT.
 * ct_in_dev [B][n_in][2][L][N]; ct_out_dev [B][n_out][2][L][N].  The result
 * equals Algorithm 1 coefficient for coefficient. */
int fl_he_conv2d(fl_ctx *ctx, const fl_conv_geom *geom, int B, const uint32_t *w_hat_dev,
                 const uint32_t *ct_in_dev, uint32_t *ct_out_dev, void *workspace_dev,
                 size_t workspace_bytes, void *stream);

/* Mask addition (Sec. 5.2: the server adds its random r to the encrypted
 * result, HAdd(<a>, <r>); here the plaintext add c0 <- c0 + Delta*r, since
 * the server holds no key).  ct_dev [n][2][L][N] updated in place; r_dev
 * uint32 [n][N] with values in [0, t) (pre-generated offline, Sec. 6.3).
 * The client then decrypts a + r; the server's share is (t - r) mod t
 * (Sec. 2.3). */
int fl_mask_to_share(fl_ctx *ctx, int n, uint32_t *ct_dev, const uint32_t *r_dev, void *stream);

/* fl_he_conv2d followed by fl_mask_to_share on its outputs, with the mask
 * fused into the inverse-NTT epilogue (one pass over the outputs).
 * r_dev uint32 [B][n_out][N]. */
int fl_he_conv2d_mask(fl_ctx *ctx, const fl_conv_geom *geom, int B, const uint32_t *w_hat_dev,
                      const uint32_t *ct_in_dev, const uint32_t *r_dev, uint32_t *ct_out_dev,
                      void *workspace_dev, size_t workspace_bytes, void *stream);

/* The two stages of fl_he_conv2d_mask as separate calls (same results):
 * fl_he_conv2d_ntt_inputs: row a3 only, the forward NTT of ct_in_dev into
 * the workspace (fl_he_conv2d_workspace_bytes bytes).
 * fl_he_conv2d_from_ntt: rows a4-a6, contraction + inverse NTT (+ mask when
 * r_dev is not NULL) from a workspace filled by the first stage. */
int fl_he_conv2d_ntt_inputs(fl_ctx *ctx, const fl_conv_geom *geom, int B, const uint32_t *ct_in_dev,
                            void *workspace_dev, size_t workspace_bytes, void *stream);
int fl_he_conv2d_from_ntt(fl_ctx *ctx, const fl_conv_geom *geom, int B, const uint32_t *w_hat_dev,
                          const void *workspace_dev, size_t workspace_bytes, const uint32_t *r_dev,
                          uint32_t *ct_out_dev, void *stream);

/* The same convolution with on-the-fly weights.  It takes the int8 filters
 * w_dev [Cout][Cin][k][k] in place of fl_encode_weights' output.  Every CTA
 * rebuilds the weight polynomials W_{i,g} it needs in shared memory from
 * their c_n*k^2 taps (Algorithm 1's DRot offsets, x^-e = -x^(N-e)).  It
 * forward-transforms them there and uses them at once, so no NTT-domain
 * weights are stored.  That removes the footprint of Table 3's PMult
 * comparison: Cout*G*L*N*4 bytes per layer, 56.7 GiB for ResNet-50 at
 * N = 16384.  The cost is one forward NTT per (image, output channel, limb,
 * input ciphertext).  The workspace, its size and the result (bit-identical,
 * plus the mask when r_dev is not NULL) are those of fl_he_conv2d_mask. */
int fl_he_conv2d_otf(fl_ctx *ctx, const fl_conv_geom *geom, int B, const int8_t *w_dev,
                     const uint32_t *ct_in_dev, const uint32_t *r_dev, uint32_t *ct_out_dev,
                     void *workspace_dev, size_t workspace_bytes, void *stream);

/* Direct form of the same convolution: Algorithm 1's DRot + CMult, where
 * DRot by e is multiplication by x^-e (Eq. 2).  It runs on the GPU with no
 * NTT, from the int8 filters w_dev [Cout][Cin][k][k] as they are (no encoded
 * weights).  Products are accumulated exactly in signed 64 bits and reduced
 * once per coefficient (lazy reduction, Sec. 6.1).  The result is
 * bit-identical to fl_he_conv2d, plus the mask when r_dev is not NULL.  It
 * costs Cin*k^2 multiply-adds per output coefficient, against about G for the
 * NTT route plus the transforms.  So it only pays for layers with few taps,
 * such as a 3-channel stem, or a single small layer.  Needs
 * Cin*k^2 <= FL_DIRECT_MAX_TAPS (FL_ERR_SHAPE otherwise).  ct_in_dev,
 * ct_out_dev and r_dev are 16-byte aligned.  The output must not overlap the
 * input. */
#define FL_DIRECT_MAX_TAPS 16384
int fl_he_conv2d_direct(fl_ctx *ctx, const fl_conv_geom *geom, int B, const int8_t *w_dev,
                        const uint32_t *ct_in_dev, const uint32_t *r_dev, uint32_t *ct_out_dev, void *stream);

/* Tensor-core form of the same convolution: the per-slot contraction of
 * Algorithm 1's sum over input ciphertexts (evaluated in the NTT domain) on
 * the 5th-generation tensor cores (tcgen05.mma kind::f16, accumulators in
 * tensor memory).  It takes the same inputs and masks as fl_he_conv2d_mask,
 * the encoded weights in the layout of fl_tc_weights and a workspace of
 * fl_he_conv2d_tc_workspace_bytes, and gives a bit-identical result.
 * - Exactness: every residue is split into four balanced base-256 digits in
 *   [-128, 127], exact in fp16.  The inputs are first multiplied by 256^a mod
 *   q_l (a = 0..3), so the product sum_g W X becomes four digit products
 *   P_e (e = 0..3) per output, each an integer of magnitude at most
 *   G * 2^16 accumulated in fp32; for G <= FL_TC_MAX_G every partial sum is
 *   an exact integer.  The CUDA cores rebuild sum_e 256^e P_e mod q_l.
 * - Tiling: a CTA holds 128 output channels x 16 (image/band, component)
 *   columns x 8 slots of one limb in tensor memory; the K dimension runs
 *   over (input ciphertext, weight digit) in steps of 16.
 * - Weights: w_tc_dev holds the weight tiles of fl_tc_weights (fp16 digits
 *   in the MMA's shared-memory layout), which the kernel bulk-copies into
 *   shared memory as they are; only the inputs are split into digits on
 *   the fly.
 * - Unlike the plain form it is not fused with the inverse NTT: a tile spans
 *   128 output channels of 8 slots, while the inverse NTT needs every slot of
 *   one output.  So the NTT-domain outputs go through the workspace, in an
 *   order where each tile's results are contiguous runs, and a second kernel
 *   gathers every output row from there, transforms it, adds the mask and
 *   writes ct_out_dev.
 * - Every internal wait is bounded (2 s); a wait that runs out sets the
 *   context's tensor-core error word (fl_tc_error).
 * G > FL_TC_MAX_G: FL_ERR_SHAPE. */
#define FL_TC_MAX_G 64
/* Workspace of fl_he_conv2d_tc: the NTT images of the inputs (as for
 * fl_he_conv2d), then their copy in slot groups of 4 ([L][N/4][B][n_in][2][4])
 * that the contraction reads, then the NTT-domain outputs in slot-tiled
 * order ([L][N/8][R][8], R = column * Cout + output channel, column =
 * (image, band, component)) that the inverse NTT gathers:
 * 2 * B*n_in*2*L*N*4 + B*n_out*2*L*N*4 bytes.  The output ciphertexts must
 * not overlap it. */
size_t fl_he_conv2d_tc_workspace_bytes(const fl_ctx *ctx, const fl_conv_geom *geom, int B);
/* Bytes of the tensor-core weight tiles of one layer (fl_tc_weights):
 * L * ceil(Cout/128) * (N/4) * ceil(G/4) * 16384; 0 when G > FL_TC_MAX_G
 * or an argument is NULL. */
size_t fl_tc_weights_bytes(const fl_ctx *ctx, const fl_conv_geom *geom);
/* The encoded weights w_hat_dev [L][Cout][G][N] (fl_encode_weights) as the
 * weight tiles of fl_he_conv2d_tc, w_tc_dev (fl_tc_weights_bytes bytes of
 * fp16 bit patterns, 16-byte aligned, not overlapping w_hat_dev).  For every
 * limb l, tile of 128 output channels mt, 4-slot group u4 = u / 4 and K step
 * kc (input ciphertexts 4 kc .. 4 kc + 3), one 16 KB tile, ordered
 * [l][mt][u4][kc]: slot u % 4 takes 4 KB, in which row r (output channel
 * i = 128 mt + r) and K index k = 4 (g % 4) + a hold the balanced base-256
 * digit a of w_hat[l][i][g][u], d_a(v) = byte_a(v + 0x80808080) - 128, at
 * byte ((r / 8) * 2 + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2 (8 x 16-byte
 * core matrices, K-major).  Rows beyond Cout and ciphertexts beyond G are
 * zeros.  About 2 to 3 times the bytes of w_hat: two bytes per digit, K
 * padded to a multiple of 4 ciphertexts, rows to a multiple of 128.
 * Offline, like the encoding itself.  G > FL_TC_MAX_G: FL_ERR_SHAPE. */
int fl_tc_weights(fl_ctx *ctx, const fl_conv_geom *geom, const uint32_t *w_hat_dev, uint16_t *w_tc_dev,
                  void *stream);
int fl_he_conv2d_tc(fl_ctx *ctx, const fl_conv_geom *geom, int B, const uint16_t *w_tc_dev,
                    const uint32_t *ct_in_dev, const uint32_t *r_dev, uint32_t *ct_out_dev,
                    void *workspace_dev, size_t workspace_bytes, void *stream);

/* The stages of fl_he_conv2d_tc after the input NTT, as separate calls
 * (same results).  fl_he_conv2d_tc_from_ntt: the tensor-core contraction
 * from a workspace (fl_he_conv2d_tc_workspace_bytes) whose first part
 * fl_he_conv2d_ntt_inputs filled; it writes the slot-tiled copy of the
 * inputs into the second part and the NTT-domain outputs (values in
 * [0, 2 q_l), slot-tiled) into the third.  fl_intt_mask_outputs: the inverse
 * NTT of those B * n_out output ciphertexts (whose weights carried N^-1),
 * gathered from the workspace, plus Delta * r on c0 when r_dev is not NULL,
 * into ct_out_dev (not overlapping the workspace); the result is
 * fl_he_conv2d_mask's. */
int fl_he_conv2d_tc_from_ntt(fl_ctx *ctx, const fl_conv_geom *geom, int B, const uint16_t *w_tc_dev,
                             void *workspace_dev, size_t workspace_bytes, void *stream);
int fl_intt_mask_outputs(fl_ctx *ctx, const fl_conv_geom *geom, int B, const void *workspace_dev,
                         size_t workspace_bytes, const uint32_t *r_dev, uint32_t *ct_out_dev, void *stream);

/* Synchronise `stream`, read the tensor-core form's error word into
 * *error_host and clear it.  FL_OK when it is 0; FL_ERR_TIMEOUT when a
 * bounded wait inside fl_he_conv2d_tc ran out (bit 0): that call's outputs
 * are incomplete, and the context stays usable. */
int fl_tc_error(fl_ctx *ctx, void *stream, uint64_t *error_host);

/* ---- Many layers in one launch ---- */

/* One layer of a stack: its geometry (host pointer), batch size, encoded
 * weights, input ciphertexts [B][n_in][2][L][N], masks [B][n_out][N] (NULL:
 * no mask) and output ciphertexts [B][n_out][2][L][N]. */
typedef struct fl_stack_layer {
  const fl_conv_geom *geom;
  int32_t B;
  const uint32_t *w_hat_dev;
  const uint32_t *ct_in_dev;
  const uint32_t *r_dev;
  uint32_t *ct_out_dev;
} fl_stack_layer;

#define FL_STACK_MAX_LAYERS 64

/* Workspace of fl_he_conv2d_stack: 256 control bytes plus the NTT images of
 * every layer's inputs. */
size_t fl_stack_workspace_bytes(const fl_ctx *ctx, const fl_stack_layer *layers, int n_layers);

/* fl_he_conv2d (or fl_he_conv2d_mask where r_dev is set) of up to 64
 * independent layers: one forward NTT launch over every layer's inputs (a3),
 * then the contraction + inverse NTT + mask (a4-a6) by the context's stack
 * kernel (fl_ctx_set_stack_kernel): per-layer launches, one queue-driven
 * launch, or one persistent warp-specialised launch.  Each output equals
 * the single-layer call's bit for bit.  The persistent kernel bounds every
 * internal wait (2 s); if one runs out it stops and records the failure in
 * the workspace's error word (fl_stack_error).  The layer array holds device
 * pointers only: every buffer it names must stay allocated until the
 * enqueued work completes. */
int fl_he_conv2d_stack(fl_ctx *ctx, const fl_stack_layer *layers, int n_layers, void *workspace_dev,
                       size_t workspace_bytes, void *stream);

/* The two stages of fl_he_conv2d_stack as separate calls (same arguments,
 * same results): the forward NTT of every layer's inputs into the workspace
 * (a3), then the contraction + inverse NTT + mask kernel(s) (a4-a6).  In
 * one fl_he_conv2d_stack call the queue kernel follows the NTT as a
 * programmatic dependent launch; split calls lose only that overlap. */
int fl_he_conv2d_stack_ntt(fl_ctx *ctx, const fl_stack_layer *layers, int n_layers, void *workspace_dev,
                           size_t workspace_bytes, void *stream);
int fl_he_conv2d_stack_run(fl_ctx *ctx, const fl_stack_layer *layers, int n_layers, void *workspace_dev,
                           size_t workspace_bytes, void *stream);

/* Kernel used by the second stage of a stack:
 * FL_STACK_PER_LAYER: one fused contraction + inverse NTT + mask launch per
 *   layer (two CTAs of 2*N/32 threads per SM, both components side by side),
 *   the layers spread over three streams of the context that fork from and
 *   join back into `stream` (so one context should not run two stacks at
 *   once from different host threads);
 * FL_STACK_PERSISTENT: one persistent warp-specialised launch over all
 *   layers (a cp.async-fed contraction team and an inverse-NTT team per SM
 *   handing items over through shared-memory mbarriers);
 * FL_STACK_QUEUE: one launch of resident CTAs that pull the fused items
 *   (image/band, output channel, limb) of every layer from a queue in the
 *   workspace, each running the contraction + inverse NTT + mask of
 *   FL_STACK_PER_LAYER; no per-layer wave tails or launch gaps.
 * All give identical outputs; which is faster depends on the stack's shapes
 * (the Python package's autotuner times them and picks).  Default:
 * FL_STACK_PER_LAYER. */
#define FL_STACK_PER_LAYER 0
#define FL_STACK_PERSISTENT 1
#define FL_STACK_QUEUE 2
int fl_ctx_set_stack_kernel(fl_ctx *ctx, int kernel);
int fl_ctx_get_stack_kernel(const fl_ctx *ctx);

/* Tuning choices of a context (the Python package's autotuner times them
 * per workload); every choice gives bit-identical results.
 * - NTT pass plan: the forward NTT of the inputs (single layers, stacks and
 *   the tensor-core form; also fl_ntt_forward) and the inverse-NTT-rows kernel of the
 *   tensor-core form run log2 N stages as two row-strided passes of radix
 *   2^r1 and 2^(log2 N - 5 - r1), then one radix-32 pass.  Available r1:
 *   3 at N = 2048; 3, 4 at 4096; 3, 4, 5 at 8192; 4, 5 at 16384; 0 selects
 *   the default (3, 4, 4, 5 for the four ring degrees).  FL_ERR_ARG for any
 *   other value.  The getter returns the r1 in use.
 * - Tensor-core tile: slot groups of 4 per CTA of fl_he_conv2d_tc (4, 8, 16,
 *   32 or 64; 0 selects the default 32).  FL_ERR_ARG otherwise.  Each call
 *   reads the setting when it launches, so a caller may set it before every
 *   layer's call (the autotuner picks it per layer).
 * The settings are plain fields of the context: set them from one host
 * thread, between calls. */
int fl_ctx_set_ntt_plan(fl_ctx *ctx, int r1);
int fl_ctx_get_ntt_plan(const fl_ctx *ctx);
int fl_ctx_set_tc_tile(fl_ctx *ctx, int groups);
int fl_ctx_get_tc_tile(const fl_ctx *ctx);

/* Synchronise `stream` and read the error word of a workspace last used by
 * fl_he_conv2d_stack into *error_host.  Returns FL_OK when the word is 0 and
 * FL_ERR_TIMEOUT when an internal wait ran out: bit 0 means the contraction
 * team gave up, bit 1 the inverse-NTT team.  The kernel then returned early,
 * its outputs are incomplete and the context stays usable. */
int fl_stack_error(const void *workspace_dev, void *stream, uint64_t *error_host);

/* Self-test of the device-side wait bound (failure detection without a
 * fault).  It launches one CTA that waits, through the persistent kernel's
 * bounded mbarrier wait, on a barrier that nothing completes.  The wait gives
 * up after its 2 s limit, sets bit 2 of an error word and returns, and the
 * call reads the word into *error_host.  The expected result is
 * FL_ERR_TIMEOUT with bit 2 set; FL_OK would mean the bound does not work.
 * It allocates 8 bytes of device memory and synchronises `stream`. */
int fl_selftest_wait_timeout(void *stream, uint64_t *error_host);

/* ---- Output volume ---- */

/* BFV modulus switching: n ciphertexts ct_in_dev [n][2][L][N] ->
 * ct_out_dev [n][2][L_out][N], dropping the last L - L_out primes one at a
 * time with rounding (Fan and Vercauteren's scale-and-round by q'/q; each
 * coefficient becomes the nearest integer to x / p mod q' for every dropped
 * prime p).  The result decrypts under a context of the first L_out primes
 * (fl_ctx_create(N, L_out, t) picks exactly those) to the same plaintext.
 * The noise is scaled by q'/q, plus at most (1 + ||s||_1)/2 per dropped
 * prime.  The paper keeps one modulus; this only shrinks what leaves the
 * device (output volume, one factor L / L_out).  Decryption needs q' well
 * above t^2, so with t = 65537 and 30-bit primes keep L_out >= 2.
 * 1 <= L_out <= L (FL_ERR_ARG otherwise).  The buffers must not overlap
 * (FL_ERR_ARG). */
int fl_mod_switch(fl_ctx *ctx, int n, const uint32_t *ct_in_dev, int L_out, uint32_t *ct_out_dev, void *stream);

/* ---- For callers that may not allocate device memory ---- */

/* fl_he_conv2d_mask_noalloc: the same computation and arguments as
 * fl_he_conv2d_mask, minus the workspace.  It is meant for callers that are
 * not allowed to allocate device memory -- e.g. a plugin whose host
 * framework owns all device memory and only passes it input and output
 * buffers, or a latency-critical request loop that must not allocate (an
 * allocation can synchronise the device) on the request path.  It has no
 * counterpart in the paper; it only changes where the scratch lives.
 *
 * - Scratch: a fixed array of FL_NOALLOC_SCRATCH_BYTES inside the library,
 *   one per device, held by every device that loads the library until the
 *   process exits.  The call needs B*n_in*2*L*N*4 bytes of it
 *   (fl_he_conv2d_workspace_bytes); a larger call is rejected with
 *   FL_ERR_ARG and a message, before any work is queued.
 * - Every call looks up the array's device address (cudaGetSymbolAddress)
 *   with the context's device current, so the address stays right after a
 *   device reset.  The first call on a device may load the library's device
 *   code for that lookup; make that first call before any stream capture
 *   begins.
 * - Calls share the array: two calls whose work overlaps on the GPU (other
 *   streams, or other threads) race on it and give undefined results;
 *   order them (one stream, or events).  The array keeps the last call's
 *   contents; no part of it has to start at zero, because the first stage
 *   overwrites every word the second stage reads.
 * - Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
#define FL_NOALLOC_SCRATCH_BYTES (16u << 20)
int fl_he_conv2d_mask_noalloc(fl_ctx *ctx, const fl_conv_geom *geom, int B, const uint32_t *w_hat_dev,
                              const uint32_t *ct_in_dev, const uint32_t *r_dev, uint32_t *ct_out_dev,
                              void *stream);

/* ---- The x^2 + x activation protocol, server side (Sec. 5.2) ---- */

/* After a convolution and its mask r (fl_he_conv2d_mask), the client holds
 * z = a + r.  It returns <X> with X = z^2 + z under direct encoding and <z>
 * under batch encoding.  Server round 1 computes <Y> = <2rz + v> (batch
 * encoded) with a fresh mask v.  The client decrypts and decodes Y and
 * returns it under direct encoding.  Server round 2 computes
 * <a^2 + a> = <X> - <Y> + (r^2 - r + v), the next convolution's input.
 *
 * Every call here works on n ciphertexts [n][2][L][N] whose plaintexts are
 * vectors of N values mod t.  One value sits at each coefficient (direct) or
 * slot (batch).  r and v are vectors [n][N] in that same layout:
 * fl_repack_outputs brings a convolution's mask into the next layer's input
 * layout.  All of it needs t prime with t = 1 mod 2N (t = 65537 serves every
 * supported N).  With another t each call returns FL_ERR_ARG.  Pointers are
 * device pointers, 16-byte aligned.  Work is queued on `stream` and nothing
 * is allocated. */

/* Batch (SIMD) encoding over Z_t[x]/(x^N+1) (Sec. 2.2).  Slot k of a
 * plaintext m holds m(psi_t^(2k+1)) mod t.  psi_t is the first
 * g^((t-1)/2N), g = 2, 3, ..., of multiplicative order 2N.  encode:
 * slots_dev [n][N] (each reduced mod t) -> m_dev [n][N] in [0, t).
 * decode: m_dev [n][N] with values in [0, t) -> slots_dev [n][N]. */
int fl_batch_encode(fl_ctx *ctx, int n, const uint32_t *slots_dev, uint32_t *m_dev, void *stream);
int fl_batch_decode(fl_ctx *ctx, int n, const uint32_t *m_dev, uint32_t *slots_dev, void *stream);

/* Offline step: r_dev, v_dev [n][N] (reduced mod t) -> prep_dev, which
 * holds fl_x2x_prep_bytes(ctx, n) bytes laid out [n][L+2][N].  Rows
 * [0, L) hold NTT_l of the batch encoding of 2r, lifted to (-t/2, t/2] mod
 * q_l and multiplied by N^-1 (round 1's inverse NTT leaves that factor out).  Row L holds the batch encoding of v in [0, t).  Row L+1 holds
 * r^2 - r + v mod t (direct encoding).  Sec. 6.3 pre-generates r, v and
 * r^2. */
size_t fl_x2x_prep_bytes(const fl_ctx *ctx, int n);
int fl_x2x_prepare(fl_ctx *ctx, int n, const uint32_t *r_dev, const uint32_t *v_dev, uint32_t *prep_dev,
                   void *stream);

/* Round 1: ct_out = PMult(ct_z, encode(2r)) + encode(v), both batch
 * encoded.  PMult is defined in Sec. 2.2.  ct_z_dev is the client's <z>
 * [n][2][L][N].  ct_out_dev may equal ct_z_dev (in place) and must not
 * overlap prep_dev. */
int fl_x2x_round1(fl_ctx *ctx, int n, const uint32_t *prep_dev, const uint32_t *ct_z_dev, uint32_t *ct_out_dev,
                  void *stream);

/* Round 2: ct_out = ct_x - ct_y + Delta*(r^2 - r + v) in R_q.  These are the
 * direct-encoded <X> and <Y> [n][2][L][N].  ct_out_dev may equal either
 * input and must not overlap prep_dev. */
int fl_x2x_round2(fl_ctx *ctx, int n, const uint32_t *prep_dev, const uint32_t *ct_x_dev, const uint32_t *ct_y_dev,
                  uint32_t *ct_out_dev, void *stream);

/* Plain-vector re-layout (server side, for its own masks).  src_dev
 * [B][prev->n_out][N] is laid out as prev's outputs: output (j, y, x) of
 * image b sits at coefficient (s*(y % Rout))*Wp + s*x of polynomial
 * j*bands + y/Rout.  dst_dev [B][next->n_in][N] gets the same values as
 * next's zero-padded packed inputs (fl_encrypt's packing), with 0 at padding
 * and unused coefficients.  prev->Cout, Ho, Wo and N must equal next->Cin,
 * H, W and N (FL_ERR_SHAPE otherwise).  The buffers must not overlap. */
int fl_repack_outputs(const fl_conv_geom *prev, const fl_conv_geom *next, int B, const uint32_t *src_dev,
                      uint32_t *dst_dev, void *stream);

/* ---- Building blocks, exposed for tests ---- */

/* In-place negacyclic NTT / inverse NTT of n RNS polynomials data_dev
 * [n][L][N].  Forward output slot k holds a(psi^(2*brev(k)+1)) with brev the
 * log2(N)-bit reversal; inverse undoes it (values canonical in [0, q_l)). */
int fl_ntt_forward(fl_ctx *ctx, int n, uint32_t *data_dev, void *stream);
int fl_ntt_inverse(fl_ctx *ctx, int n, uint32_t *data_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FLASHGPU_H */
