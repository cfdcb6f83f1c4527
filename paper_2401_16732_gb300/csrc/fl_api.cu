// C-ABI of flashgpu (declarations and contracts in include/flashgpu.h).
//
// Host side of the library: parameter set-up (primes, roots of unity,
// twiddle tables, per-limb and CRT constants), argument validation and the
// sequencing of kernel launches.  All arithmetic on ciphertexts runs in the
// kernels of fl_kernels.cu; nothing here computes on ciphertext data.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/flashgpu.h"
#include "fl_launch.h"

using fl::CtxConst;
using fl::DecConst;
using fl::GeomDims;
typedef unsigned __int128 u128;

constexpr int kAuxStreams = 3;

struct fl_ctx {
  int N, logN, L, device, sms;
  int stack_kernel;  // FL_STACK_PER_LAYER, FL_STACK_PERSISTENT or FL_STACK_QUEUE
  int ntt_plan;      // first row-pass radix exponent of the input NTT and inverse-NTT-rows kernels (0: default)
  int tc_tile;       // slot groups of 4 per tensor-core CTA (0: default)
  // per-layer stack launches fan out over these (fork/join through events)
  cudaStream_t aux[kAuxStreams];
  cudaEvent_t fork_ev, join_ev[kAuxStreams];
  uint32_t t;
  uint32_t psi[FL_MAX_L];
  CtxConst cc;
  DecConst dc;
  uint32_t* tw;  // device twiddle tables, twiddle_limb_words(logN) words per limb
  // error word of the tensor-core contraction's bounded waits (in the same
  // allocation as the tables, after them)
  unsigned long long* tc_err;
  // batch encoding over Z_t[x]/(x^N+1), present when t is prime and t = 1 mod 2N:
  // the tables of t follow the L limbs' tables in `tw`
  int batch;
  uint32_t psi_t;
  fl::LimbConst tc;
};

static_assert(FL_TC_MAX_G == fl::kTcMaxG, "header and kernel agree on the G bound");

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(FL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }

uint64_t powmod(uint64_t b, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  b %= m;
  while (e) {
    if (e & 1) r = mulmod(r, b, m);
    b = mulmod(b, b, m);
    e >>= 1;
  }
  return r;
}

// Deterministic Miller-Rabin for n < 4,759,123,141 with bases 2, 7, 61
// (Jaeschke, 1993).
bool is_prime32(uint32_t n) {
  if (n < 2) return false;
  for (uint32_t p : {2u, 3u, 5u, 7u, 11u, 13u, 61u})
    if (n % p == 0) return n == p;
  uint32_t d = n - 1;
  int s = 0;
  while (!(d & 1)) d >>= 1, ++s;
  for (uint32_t a : {2u, 7u, 61u}) {
    uint64_t x = powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; ++r) {
      x = mulmod(x, x, n);
      if (x == n - 1) { comp = false; break; }
    }
    if (comp) return false;
  }
  return true;
}

uint32_t brev(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; ++i) r = (r << 1) | ((x >> i) & 1);
  return r;
}

uint32_t shoup(uint32_t w, uint32_t q) { return (uint32_t)(((uint64_t)w << 32) / q); }

// Twiddle tables (fl::TwLayout) and constants of one NTT modulus q, prime
// with q = 1 mod 2N: an RNS limb of the ciphertext modulus, or the plaintext
// modulus t for batch encoding.  Delta fields are left to the caller.
void build_tables(uint32_t q, int N, int logN, uint32_t* Tw, fl::LimbConst& lc, uint32_t* psi_out) {
  const uint64_t step = 2ull * N;
  // psi: first g^((q-1)/2N), g = 2, 3, ..., with psi^N = -1 (order 2N)
  uint32_t psi = 0;
  for (uint64_t g = 2; g < q && !psi; ++g) {
    uint64_t cand = powmod(g, (q - 1) / step, q);
    if (powmod(cand, N, q) == q - 1) psi = (uint32_t)cand;
  }
  const uint32_t psi_inv = (uint32_t)powmod(psi, q - 2, q);
  *psi_out = psi;
  uint2* pairs = reinterpret_cast<uint2*>(Tw);
  std::vector<uint32_t> fw(N), iv(N);
  for (int i = 0; i < N; ++i) {
    fw[i] = (uint32_t)powmod(psi, brev(i, logN), q);
    iv[i] = (uint32_t)powmod(psi_inv, brev(i, logN), q);
    pairs[fl::TW_FWD * N + i] = make_uint2(fw[i], shoup(fw[i], q));
    pairs[fl::TW_INV * N + i] = make_uint2(iv[i], shoup(iv[i], q));
  }
  // thread-major twiddles of the radix-32 pass over stages [logN-5, logN):
  // thread blk consumes, for stage S0+d (ascending forward, descending
  // inverse), twiddles (1 << (S0+d)) + blk*2^d + m for m < 2^d.
  const int Tn = N / 32, S0 = logN - 5;
  uint32_t* grouped = Tw + 4 * N;
  for (int dir = 0; dir < 2; ++dir) {
    const std::vector<uint32_t>& tab = dir == fl::TW_FWD ? fw : iv;
    for (int blk = 0; blk < Tn; ++blk) {
      int slot = 0;
      for (int dd = 0; dd < 5; ++dd) {
        const int d = dir == fl::TW_INV ? 4 - dd : dd;
        for (int m = 0; m < (1 << d); ++m, ++slot) {
          const uint32_t w = tab[(1 << (S0 + d)) + (blk << d) + m];
          uint32_t* e = grouped + (((size_t)dir * 16 + slot / 2) * Tn + blk) * 4 + (slot & 1) * 2;
          e[0] = w;
          e[1] = shoup(w, q);
        }
      }
    }
  }
  memset(&lc, 0, sizeof lc);
  lc.q = q;
  lc.two_q = 2 * q;
  lc.n_inv = (uint32_t)powmod(N, q - 2, q);
  lc.n_inv_sh = shoup(lc.n_inv, q);
  lc.last_w = (uint32_t)mulmod(iv[1], lc.n_inv, q);
  lc.last_w_sh = shoup(lc.last_w, q);
  lc.mu = ~0ull / q;
  lc.r32 = (uint32_t)((1ull << 32) % q);
  lc.r32_sh = shoup(lc.r32, q);
}

GeomDims dims_of(const fl_conv_geom& g) {
  GeomDims d;
  d.Cin = g.Cin; d.Cout = g.Cout; d.H = g.H; d.W = g.W; d.k = g.k; d.s = g.stride; d.pad = g.pad;
  d.Hp = g.Hp; d.Wp = g.Wp; d.Ho = g.Ho; d.Wo = g.Wo; d.Rin = g.Rin; d.Rout = g.Rout;
  d.bands = g.bands; d.P = g.P; d.c_n = g.c_n; d.G = g.G; d.n_in = g.n_in; d.n_out = g.n_out;
  return d;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

int check_ctx(const fl_ctx* ctx) {
  if (!ctx) return fail(FL_ERR_ARG, "null context");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != ctx->device)
    return fail(FL_ERR_ARG, "current device %d is not the context's device %d", dev, ctx->device);
  return FL_OK;
}

int check_geom(const fl_ctx* ctx, const fl_conv_geom* g) {
  if (!g) return fail(FL_ERR_ARG, "null geometry");
  fl_conv_geom ref;
  int rc = fl_conv_geom_make(g->N, g->Cin, g->Cout, g->H, g->W, g->k, g->stride, g->pad, &ref);
  if (rc) return rc;
  if (memcmp(&ref, g, sizeof ref) != 0)
    return fail(FL_ERR_SHAPE, "geometry fields are inconsistent (build it with fl_conv_geom_make)");
  if (g->N != ctx->N) return fail(FL_ERR_SHAPE, "geometry N=%d but context N=%d", g->N, ctx->N);
  if (g->Cout > 65535) return fail(FL_ERR_SHAPE, "Cout=%d above 65535", g->Cout);
  return FL_OK;
}

int check_ptrs(std::initializer_list<const void*> ps) {
  for (const void* p : ps) {
    if (!p) return fail(FL_ERR_ARG, "null device pointer");
    if (!aligned16(p)) return fail(FL_ERR_ARG, "device pointer %p is not 16-byte aligned", p);
  }
  return FL_OK;
}

int launched(cudaError_t e, const char* what) { return e == cudaSuccess ? FL_OK : cuda_fail(e, what); }

// Row and CTA counts are passed to launchers as int: reject larger jobs.
int rows_ok(long long rows, const char* what) {
  return rows <= 0x7fffffffLL ? FL_OK : fail(FL_ERR_ARG, "%s: %lld rows exceed one launch", what, rows);
}

}  // namespace

namespace fl {
int ctx_internals(const fl_ctx* ctx, int* logN, int* L, int* device, const uint32_t** tw, const CtxConst** cc) {
  if (!ctx) return fail(FL_ERR_ARG, "null context");
  *logN = ctx->logN;
  *L = ctx->L;
  *device = ctx->device;
  *tw = ctx->tw;
  *cc = &ctx->cc;
  return FL_OK;
}

int fail_msg(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
}  // namespace fl

extern "C" {

const char* fl_last_error(void) { return g_err.c_str(); }

int fl_conv_geom_make(int N, int Cin, int Cout, int H, int W, int k, int stride, int pad,
                      fl_conv_geom* out) {
  if (!out) return fail(FL_ERR_ARG, "null output");
  if (N < 2 || (N & (N - 1)) || N > (1 << 20)) return fail(FL_ERR_SHAPE, "N=%d is not a power of two", N);
  if (Cin < 1 || Cout < 1 || H < 1 || W < 1 || k < 1 || stride < 1 || pad < 0)
    return fail(FL_ERR_SHAPE, "non-positive convolution size");
  if ((long long)Cin * Cout * k * k > (1ll << 31) || H > (1 << 16) || W > (1 << 16) || pad > (1 << 16))
    return fail(FL_ERR_SHAPE, "convolution too large");
  fl_conv_geom g;
  memset(&g, 0, sizeof g);
  g.N = N; g.Cin = Cin; g.Cout = Cout; g.H = H; g.W = W; g.k = k; g.stride = stride; g.pad = pad;
  g.Hp = H + 2 * pad;
  g.Wp = W + 2 * pad;
  if (k > g.Hp || k > g.Wp) return fail(FL_ERR_SHAPE, "kernel %d larger than padded input", k);
  g.Ho = (g.Hp - k) / stride + 1;
  g.Wo = (g.Wp - k) / stride + 1;
  if ((long long)g.Hp * g.Wp <= N) {
    g.Rin = g.Hp;
    g.Rout = g.Ho;
    g.bands = 1;
  } else {
    g.Rin = N / g.Wp;
    if (g.Rin < k) return fail(FL_ERR_SHAPE, "a band of %d padded rows of width %d exceeds N=%d", k, g.Wp, N);
    g.Rout = (g.Rin - k) / stride + 1;
    g.bands = (g.Ho + g.Rout - 1) / g.Rout;
  }
  g.P = g.Rin * g.Wp;
  g.c_n = N / g.P;
  g.G = (Cin + g.c_n - 1) / g.c_n;
  g.n_in = g.bands * g.G;
  g.n_out = Cout * g.bands;
  *out = g;
  return FL_OK;
}

int fl_ctx_create(int N, int L, uint32_t t, fl_ctx** out) {
  if (!out) return fail(FL_ERR_ARG, "null output");
  *out = nullptr;
  int logN = 0;
  while ((1 << logN) < N) ++logN;
  if ((1 << logN) != N || logN < 11 || logN > 14)
    return fail(FL_ERR_ARG, "N=%d: supported ring degrees are 2048, 4096, 8192, 16384", N);
  if (L < 1 || L > FL_MAX_L) return fail(FL_ERR_ARG, "L=%d outside [1, %d]", L, FL_MAX_L);
  if (t < 3 || t >= (1u << 20) || !(t & 1)) return fail(FL_ERR_ARG, "t=%u must be odd in [3, 2^20)", t);
  fl_ctx* c = new fl_ctx();
  c->N = N; c->logN = logN; c->L = L; c->t = t;
  c->stack_kernel = FL_STACK_PER_LAYER;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaGetDevice"); }

  // primes: largest below 2^30 with q = 1 mod 2N, descending
  std::vector<uint32_t> qs;
  const uint64_t step = 2ull * N;
  for (uint64_t cand = ((1ull << 30) - 2) / step * step + 1; cand > step && (int)qs.size() < L; cand -= step)
    if (is_prime32((uint32_t)cand)) qs.push_back((uint32_t)cand);
  if ((int)qs.size() < L) { delete c; return fail(FL_ERR_ARG, "not enough NTT-friendly primes"); }

  u128 Q = 1;
  for (uint32_t q : qs) Q *= q;
  const u128 Delta = Q / t;
  const size_t limb_words = fl::twiddle_limb_words(logN);
  const bool batch = is_prime32(t) && (t - 1) % (2ull * N) == 0;
  std::vector<uint32_t> host((size_t)(L + (batch ? 1 : 0)) * limb_words);
  memset(&c->cc, 0, sizeof c->cc);
  memset(&c->dc, 0, sizeof c->dc);
  c->cc.L = L; c->cc.t = t;
  c->dc.L = L; c->dc.t = t;
  c->dc.qhi = (uint64_t)(Q >> 64); c->dc.qlo = (uint64_t)Q;
  for (int l = 0; l < L; ++l) {
    const uint32_t q = qs[l];
    build_tables(q, N, logN, host.data() + (size_t)l * limb_words, c->cc.limb[l], &c->psi[l]);
    fl::LimbConst& lc = c->cc.limb[l];
    lc.delta = (uint32_t)(Delta % q);
    lc.delta_sh = shoup(lc.delta, q);
    const u128 Ql = Q / q;
    c->dc.q[l] = q;
    c->dc.inv[l] = (uint32_t)powmod((uint64_t)(Ql % q), q - 2, q);
    c->dc.Qhi[l] = (uint64_t)(Ql >> 64);
    c->dc.Qlo[l] = (uint64_t)Ql;
  }
  if (batch) {
    build_tables(t, N, logN, host.data() + (size_t)L * limb_words, c->tc, &c->psi_t);
    c->batch = 1;
  }
  if ((e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess) {
    delete c;
    return cuda_fail(e, "SM count");
  }
  if ((e = fl::launch_setup(logN)) != cudaSuccess || (e = fl::launch_stack_setup(logN)) != cudaSuccess ||
      (e = fl::launch_ntt_multi_setup(logN)) != cudaSuccess || (e = fl::launch_act_setup(logN)) != cudaSuccess ||
      (e = fl::launch_direct_setup(logN)) != cudaSuccess || (e = fl::launch_otf_setup(logN)) != cudaSuccess ||
      (e = fl::launch_tc_setup(logN)) != cudaSuccess) {
    delete c;
    return cuda_fail(e, "kernel set-up");
  }
  bool ok = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < kAuxStreams && ok; ++k)
    ok = cudaStreamCreateWithFlags(&c->aux[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->join_ev[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    delete c;
    return fail(FL_ERR_OOM, "auxiliary streams / events");
  }
  const size_t tw_words = (host.size() + 3) / 4 * 4;  // the error word follows, 16-byte aligned
  if ((e = cudaMalloc(&c->tw, (tw_words + 4) * sizeof(uint32_t))) != cudaSuccess) {
    delete c;
    return fail(FL_ERR_OOM, "twiddle tables: %s", cudaGetErrorString(e));
  }
  c->tc_err = reinterpret_cast<unsigned long long*>(c->tw + tw_words);
  if ((e = cudaMemcpy(c->tw, host.data(), host.size() * sizeof(uint32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(c->tc_err, 0, 16)) != cudaSuccess) {
    cudaFree(c->tw);
    delete c;
    return cuda_fail(e, "twiddle upload");
  }
  *out = c;
  return FL_OK;
}

void fl_ctx_destroy(fl_ctx* ctx) {
  if (!ctx) return;
  for (int k = 0; k < kAuxStreams; ++k) {
    if (ctx->aux[k]) cudaStreamDestroy(ctx->aux[k]);
    if (ctx->join_ev[k]) cudaEventDestroy(ctx->join_ev[k]);
  }
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->tw) cudaFree(ctx->tw);
  delete ctx;
}

int fl_ctx_params(const fl_ctx* ctx, uint32_t* primes_host, uint32_t* delta_host, uint32_t* psi_host) {
  if (!ctx) return fail(FL_ERR_ARG, "null context");
  for (int l = 0; l < ctx->L; ++l) {
    if (primes_host) primes_host[l] = ctx->cc.limb[l].q;
    if (delta_host) delta_host[l] = ctx->cc.limb[l].delta;
    if (psi_host) psi_host[l] = ctx->psi[l];
  }
  return FL_OK;
}

int fl_keygen(fl_ctx* ctx, const int8_t* s_dev, uint32_t* sk_dev, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx))) return rc;
  if (!s_dev) return fail(FL_ERR_ARG, "null secret");
  if ((rc = check_ptrs({sk_dev}))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = launched(fl::launch_sk_expand(s_dev, sk_dev, ctx->N, ctx->cc, st), "sk expand"))) return rc;
  return launched(fl::launch_ntt_fwd(ctx->logN, ctx->L, sk_dev, ctx->L, ctx->L, sk_dev, ctx->L, ctx->L, 1,
                                     ctx->tw, ctx->cc, st),
                  "sk ntt");
}

int fl_encrypt(fl_ctx* ctx, const uint32_t* sk_dev, const fl_conv_geom* geom, int B, const int32_t* x_dev,
               const uint32_t* a_dev, const int32_t* e_dev, uint32_t* ct_dev, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx)) || (rc = check_geom(ctx, geom))) return rc;
  if (B < 0) return fail(FL_ERR_ARG, "B=%d", B);
  if (B == 0) return FL_OK;
  if ((rc = check_ptrs({sk_dev, a_dev, ct_dev})) || !x_dev || !e_dev)
    return rc ? rc : fail(FL_ERR_ARG, "null input");
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = rows_ok((long long)B * geom->n_in * 2 * ctx->L, "encrypt"))) return rc;
  const int n = B * geom->n_in, L = ctx->L, N = ctx->N;
  // c1 = a
  cudaError_t e = cudaMemcpy2DAsync(ct_dev + (size_t)L * N, (size_t)2 * L * N * 4, a_dev, (size_t)L * N * 4,
                                    (size_t)L * N * 4, n, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "c1 copy");
  // c0 slot <- NTT(a)
  if ((rc = launched(fl::launch_ntt_fwd(ctx->logN, n * L, a_dev, n * L, 0, ct_dev, L, 2 * L, 1, ctx->tw,
                                        ctx->cc, st),
                     "encrypt ntt")))
    return rc;
  // c0 <- Delta*m - INTT(NTT(a) * NTT(s)) - e
  return launched(fl::launch_pmul_intt(ctx->logN, 1, n, nullptr, ct_dev, sk_dev, x_dev, e_dev, dims_of(*geom),
                                       ctx->tw, ctx->cc, st),
                  "encrypt");
}

int fl_encrypt_online(fl_ctx* ctx, const fl_conv_geom* geom, int B, const int32_t* x_dev,
                      const uint32_t* enc0_dev, uint32_t* ct_dev, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx)) || (rc = check_geom(ctx, geom))) return rc;
  if (B < 0) return fail(FL_ERR_ARG, "B=%d", B);
  if (B == 0) return FL_OK;
  if ((rc = check_ptrs({enc0_dev, ct_dev})) || !x_dev) return rc ? rc : fail(FL_ERR_ARG, "null input");
  if ((rc = rows_ok((long long)B * geom->n_in * 2 * ctx->L, "online encryption"))) return rc;
  return launched(fl::launch_enc_online(enc0_dev, ct_dev, x_dev, dims_of(*geom), B * geom->n_in, ctx->N,
                                        ctx->cc, (cudaStream_t)stream),
                  "online encrypt");
}

size_t fl_decrypt_workspace_bytes(const fl_ctx* ctx, int n) {
  return ctx && n > 0 ? (size_t)n * ctx->L * ctx->N * 4 : 0;
}

int fl_decrypt(fl_ctx* ctx, const uint32_t* sk_dev, int n, const uint32_t* ct_dev, uint32_t* m_dev,
               void* workspace_dev, size_t workspace_bytes, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx))) return rc;
  if (n < 0) return fail(FL_ERR_ARG, "n=%d", n);
  if (n == 0) return FL_OK;
  if ((rc = check_ptrs({sk_dev, ct_dev, m_dev, workspace_dev})) || (rc = rows_ok((long long)n * 2 * ctx->L, "decrypt")))
    return rc;
  if (workspace_bytes < fl_decrypt_workspace_bytes(ctx, n))
    return fail(FL_ERR_ARG, "workspace %zu bytes, need %zu", workspace_bytes, fl_decrypt_workspace_bytes(ctx, n));
  cudaStream_t st = (cudaStream_t)stream;
  const int L = ctx->L;
  uint32_t* ws = (uint32_t*)workspace_dev;
  // ws <- NTT(c1): source row r is ciphertext r/L, limb r%L of component 1
  if ((rc = launched(fl::launch_ntt_fwd(ctx->logN, n * L, ct_dev + (size_t)L * ctx->N, L, 2 * L, ws, n * L, 0, 1,
                                        ctx->tw, ctx->cc, st),
                     "decrypt ntt")))
    return rc;
  GeomDims none;
  memset(&none, 0, sizeof none);
  if ((rc = launched(fl::launch_pmul_intt(ctx->logN, 0, n, ws, const_cast<uint32_t*>(ct_dev), sk_dev, nullptr,
                                          nullptr, none, ctx->tw, ctx->cc, st),
                     "decrypt phase")))
    return rc;
  return launched(fl::launch_dec_round(ws, m_dev, n, ctx->N, ctx->dc, st), "decrypt round");
}

size_t fl_noise_workspace_bytes(const fl_ctx* ctx, int n) { return fl_decrypt_workspace_bytes(ctx, n) + 256; }

int fl_noise_inf(fl_ctx* ctx, const uint32_t* sk_dev, int n, const uint32_t* ct_dev, const uint32_t* m_dev,
                 void* workspace_dev, size_t workspace_bytes, void* stream, double* max_noise_host) {
  int rc;
  if ((rc = check_ctx(ctx))) return rc;
  if (n < 0 || !max_noise_host) return fail(FL_ERR_ARG, "n=%d or null result pointer", n);
  if (n == 0) {
    *max_noise_host = 0.0;
    return FL_OK;
  }
  if ((rc = check_ptrs({sk_dev, ct_dev, m_dev, workspace_dev})) || (rc = rows_ok((long long)n * 2 * ctx->L, "noise")))
    return rc;
  if (workspace_bytes < fl_noise_workspace_bytes(ctx, n))
    return fail(FL_ERR_ARG, "workspace %zu bytes, need %zu", workspace_bytes, fl_noise_workspace_bytes(ctx, n));
  cudaStream_t st = (cudaStream_t)stream;
  const int L = ctx->L;
  uint32_t* ws = (uint32_t*)workspace_dev;
  unsigned long long* word = (unsigned long long*)((char*)workspace_dev + fl_decrypt_workspace_bytes(ctx, n));
  cudaError_t e = cudaMemsetAsync(word, 0, sizeof *word, st);
  if (e != cudaSuccess) return cuda_fail(e, "noise word");
  // the phase [c0 + c1 s]_{q_l} per limb, as in fl_decrypt
  if ((rc = launched(fl::launch_ntt_fwd(ctx->logN, n * L, ct_dev + (size_t)L * ctx->N, L, 2 * L, ws, n * L, 0, 1,
                                        ctx->tw, ctx->cc, st),
                     "noise ntt")))
    return rc;
  GeomDims none;
  memset(&none, 0, sizeof none);
  if ((rc = launched(fl::launch_pmul_intt(ctx->logN, 0, n, ws, const_cast<uint32_t*>(ct_dev), sk_dev, nullptr,
                                          nullptr, none, ctx->tw, ctx->cc, st),
                     "noise phase")))
    return rc;
  if ((rc = launched(fl::launch_noise(ws, m_dev, n, ctx->N, ctx->dc, ctx->cc, word, st), "noise")))
    return rc;
  unsigned long long bits = 0;
  if ((e = cudaMemcpyAsync(&bits, word, sizeof bits, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(e, "noise read");
  memcpy(max_noise_host, &bits, sizeof bits);
  return FL_OK;
}

// Host <-> device copies of ciphertext words through the library (the
// caller's buffers; pinned host memory makes them asynchronous).
static int copy_checks(fl_ctx* ctx, const void* host, const void* dev, size_t words) {
  int rc;
  if ((rc = check_ctx(ctx))) return rc;
  if (words == 0) return FL_OK;
  if (!host || !dev) return fail(FL_ERR_ARG, "null buffer");
  cudaPointerAttributes ha{}, da{};
  if (cudaPointerGetAttributes(&da, dev) != cudaSuccess || da.type != cudaMemoryTypeDevice || da.device != ctx->device)
    return fail(FL_ERR_ARG, "the device buffer is not device memory of the context's device");
  if (cudaPointerGetAttributes(&ha, host) == cudaSuccess && ha.type == cudaMemoryTypeDevice)
    return fail(FL_ERR_ARG, "the host buffer is device memory");
  cudaGetLastError();  // clear a lookup error left by pageable host memory
  return FL_OK;
}

int fl_copy_to_device(fl_ctx* ctx, const uint32_t* host, uint32_t* dev, size_t words, void* stream) {
  int rc;
  if ((rc = copy_checks(ctx, host, dev, words)) || words == 0) return rc;
  const cudaError_t e = cudaMemcpyAsync(dev, host, words * 4, cudaMemcpyHostToDevice, (cudaStream_t)stream);
  return e == cudaSuccess ? FL_OK : cuda_fail(e, "copy to device");
}

int fl_copy_to_host(fl_ctx* ctx, const uint32_t* dev, uint32_t* host, size_t words, void* stream) {
  int rc;
  if ((rc = copy_checks(ctx, host, dev, words)) || words == 0) return rc;
  const cudaError_t e = cudaMemcpyAsync(host, dev, words * 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  return e == cudaSuccess ? FL_OK : cuda_fail(e, "copy to host");
}

int fl_extract_outputs(const fl_conv_geom* geom, int B, const uint32_t* m_dev, int32_t* y_dev, void* stream) {
  if (!geom) return fail(FL_ERR_ARG, "null geometry");
  fl_conv_geom ref;
  int rc = fl_conv_geom_make(geom->N, geom->Cin, geom->Cout, geom->H, geom->W, geom->k, geom->stride, geom->pad,
                             &ref);
  if (rc) return rc;
  if (memcmp(&ref, geom, sizeof ref)) return fail(FL_ERR_SHAPE, "geometry fields are inconsistent");
  if (B < 0) return fail(FL_ERR_ARG, "B=%d", B);
  if (B == 0) return FL_OK;
  if (!m_dev || !y_dev) return fail(FL_ERR_ARG, "null pointer");
  return launched(fl::launch_extract(m_dev, y_dev, dims_of(*geom), B, geom->N, (cudaStream_t)stream), "extract");
}

size_t fl_weights_bytes(const fl_ctx* ctx, const fl_conv_geom* geom) {
  return ctx && geom ? (size_t)ctx->L * geom->Cout * geom->G * ctx->N * 4 : 0;
}

int fl_encode_weights(fl_ctx* ctx, const fl_conv_geom* geom, const int8_t* w_dev, uint32_t* w_hat_dev,
                      void* stream) {
  int rc;
  if ((rc = check_ctx(ctx)) || (rc = check_geom(ctx, geom))) return rc;
  if ((rc = check_ptrs({w_hat_dev})) || !w_dev) return rc ? rc : fail(FL_ERR_ARG, "null filters");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(w_hat_dev, 0, fl_weights_bytes(ctx, geom), st);
  if (e != cudaSuccess) return cuda_fail(e, "weights memset");
  if ((rc = launched(fl::launch_w_scatter(w_dev, w_hat_dev, dims_of(*geom), ctx->N, ctx->cc, st), "w scatter")))
    return rc;
  if ((rc = rows_ok((long long)ctx->L * geom->Cout * geom->G, "weight rows"))) return rc;
  const int rows = ctx->L * geom->Cout * geom->G;
  return launched(fl::launch_ntt_fwd(ctx->logN, rows, w_hat_dev, rows, 0, w_hat_dev, rows, 0, geom->Cout * geom->G,
                                     ctx->tw, ctx->cc, st),
                  "weights ntt");
}

size_t fl_he_conv2d_workspace_bytes(const fl_ctx* ctx, const fl_conv_geom* geom, int B) {
  return ctx && geom && B > 0 ? (size_t)B * geom->n_in * 2 * ctx->L * ctx->N * 4 : 0;
}

static int conv_checks(fl_ctx* ctx, const fl_conv_geom* geom, int B, size_t workspace_bytes) {
  int rc;
  if ((rc = check_ctx(ctx)) || (rc = check_geom(ctx, geom))) return rc;
  if (B < 0) return fail(FL_ERR_ARG, "B=%d", B);
  const size_t need = fl_he_conv2d_workspace_bytes(ctx, geom, B);
  if (workspace_bytes < need) return fail(FL_ERR_ARG, "workspace %zu bytes, need %zu", workspace_bytes, need);
  if ((long long)B * geom->bands > 0x7fffffff) return fail(FL_ERR_ARG, "batch too large");
  if ((rc = rows_ok((long long)B * geom->n_in * 2 * ctx->L, "input rows"))) return rc;
  return rows_ok((long long)B * geom->n_out * 2 * ctx->L, "output rows");
}

static int stage_ntt(fl_ctx* ctx, const fl_conv_geom* geom, int B, const uint32_t* ct_in_dev, void* ws,
                     cudaStream_t st) {
  const int rows = B * geom->n_in * 2 * ctx->L;
  return launched(fl::launch_ntt_fwd(ctx->logN, rows, ct_in_dev, rows, 0, (uint32_t*)ws, rows, 0, 1, ctx->tw,
                                     ctx->cc, st, ctx->ntt_plan),
                  "input ntt");
}

static int stage_conv(fl_ctx* ctx, const fl_conv_geom* geom, int B, const uint32_t* w_hat_dev, const void* ws,
                      const uint32_t* r_dev, uint32_t* ct_out_dev, cudaStream_t st) {
  fl::ConvDims cd{geom->Cout, geom->G, geom->n_in, geom->n_out, geom->bands};
  // launched as a programmatic dependent of the previous grid in `st` (the
  // input NTT when called from he_conv2d_impl); the kernel waits for it
  return launched(fl::launch_conv_intt(ctx->logN, B, cd, w_hat_dev, (const uint32_t*)ws, ct_out_dev, r_dev, ctx->tw,
                                       ctx->cc, st, true),
                  "contraction + intt");
}

static int he_conv2d_impl(fl_ctx* ctx, const fl_conv_geom* geom, int B, const uint32_t* w_hat_dev,
                          const uint32_t* ct_in_dev, const uint32_t* r_dev, uint32_t* ct_out_dev,
                          void* workspace_dev, size_t workspace_bytes, void* stream) {
  int rc;
  if ((rc = conv_checks(ctx, geom, B, workspace_bytes))) return rc;
  if (B == 0) return FL_OK;
  if ((rc = check_ptrs({w_hat_dev, ct_in_dev, ct_out_dev, workspace_dev}))) return rc;
  if (r_dev && (rc = check_ptrs({r_dev}))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = stage_ntt(ctx, geom, B, ct_in_dev, workspace_dev, st))) return rc;
  return stage_conv(ctx, geom, B, w_hat_dev, workspace_dev, r_dev, ct_out_dev, st);
}

int fl_he_conv2d_ntt_inputs(fl_ctx* ctx, const fl_conv_geom* geom, int B, const uint32_t* ct_in_dev,
                            void* workspace_dev, size_t workspace_bytes, void* stream) {
  int rc;
  if ((rc = conv_checks(ctx, geom, B, workspace_bytes))) return rc;
  if (B == 0) return FL_OK;
  if ((rc = check_ptrs({ct_in_dev, workspace_dev}))) return rc;
  return stage_ntt(ctx, geom, B, ct_in_dev, workspace_dev, (cudaStream_t)stream);
}

int fl_he_conv2d_from_ntt(fl_ctx* ctx, const fl_conv_geom* geom, int B, const uint32_t* w_hat_dev,
                          const void* workspace_dev, size_t workspace_bytes, const uint32_t* r_dev,
                          uint32_t* ct_out_dev, void* stream) {
  int rc;
  if ((rc = conv_checks(ctx, geom, B, workspace_bytes))) return rc;
  if (B == 0) return FL_OK;
  if ((rc = check_ptrs({w_hat_dev, workspace_dev, ct_out_dev}))) return rc;
  if (r_dev && (rc = check_ptrs({r_dev}))) return rc;
  return stage_conv(ctx, geom, B, w_hat_dev, workspace_dev, r_dev, ct_out_dev, (cudaStream_t)stream);
}

int fl_he_conv2d(fl_ctx* ctx, const fl_conv_geom* geom, int B, const uint32_t* w_hat_dev, const uint32_t* ct_in_dev,
                 uint32_t* ct_out_dev, void* workspace_dev, size_t workspace_bytes, void* stream) {
  return he_conv2d_impl(ctx, geom, B, w_hat_dev, ct_in_dev, nullptr, ct_out_dev, workspace_dev, workspace_bytes,
                        stream);
}

int fl_he_conv2d_mask(fl_ctx* ctx, const fl_conv_geom* geom, int B, const uint32_t* w_hat_dev,
                      const uint32_t* ct_in_dev, const uint32_t* r_dev, uint32_t* ct_out_dev, void* workspace_dev,
                      size_t workspace_bytes, void* stream) {
  if (!r_dev) return fail(FL_ERR_ARG, "null mask");
  return he_conv2d_impl(ctx, geom, B, w_hat_dev, ct_in_dev, r_dev, ct_out_dev, workspace_dev, workspace_bytes,
                        stream);
}

int fl_mod_switch(fl_ctx* ctx, int n, const uint32_t* ct_in_dev, int L_out, uint32_t* ct_out_dev, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx))) return rc;
  if (n < 0) return fail(FL_ERR_ARG, "n=%d", n);
  if (L_out < 1 || L_out > ctx->L) return fail(FL_ERR_ARG, "L_out=%d outside [1, %d]", L_out, ctx->L);
  if (n == 0) return FL_OK;
  if ((rc = check_ptrs({ct_in_dev, ct_out_dev}))) return rc;
  const char* a = (const char*)ct_in_dev;
  const char* b = (const char*)ct_out_dev;
  const size_t in_bytes = (size_t)n * 2 * ctx->L * ctx->N * 4, out_bytes = (size_t)n * 2 * L_out * ctx->N * 4;
  if (a < b + out_bytes && b < a + in_bytes) return fail(FL_ERR_ARG, "input and output overlap");
  fl::ModSwitchConst mc;
  memset(&mc, 0, sizeof mc);
  mc.L = ctx->L;
  mc.L_out = L_out;
  for (int d = 0; d < ctx->L; ++d) {
    const uint32_t p = ctx->cc.limb[d].q;
    mc.q[d] = p;
    for (int i = 0; i < d; ++i) {
      const uint32_t qi = ctx->cc.limb[i].q;
      mc.inv[d][i] = (uint32_t)powmod(p % qi, qi - 2, qi);
      mc.inv_sh[d][i] = shoup(mc.inv[d][i], qi);
    }
  }
  return launched(fl::launch_mod_switch(ct_in_dev, ct_out_dev, 2LL * n, ctx->N, mc, (cudaStream_t)stream),
                  "modulus switch");
}

int fl_he_conv2d_otf(fl_ctx* ctx, const fl_conv_geom* geom, int B, const int8_t* w_dev, const uint32_t* ct_in_dev,
                     const uint32_t* r_dev, uint32_t* ct_out_dev, void* workspace_dev, size_t workspace_bytes,
                     void* stream) {
  int rc;
  if ((rc = conv_checks(ctx, geom, B, workspace_bytes))) return rc;
  if (B == 0) return FL_OK;
  if (!w_dev) return fail(FL_ERR_ARG, "null filters");
  if ((rc = check_ptrs({ct_in_dev, ct_out_dev, workspace_dev}))) return rc;
  if (r_dev && (rc = check_ptrs({r_dev}))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = stage_ntt(ctx, geom, B, ct_in_dev, workspace_dev, st))) return rc;
  return launched(fl::launch_conv_otf(ctx->logN, B, dims_of(*geom), w_dev, (const uint32_t*)workspace_dev, ct_out_dev,
                                      r_dev, ctx->tw, ctx->cc, st),
                  "on-the-fly conv");
}

size_t fl_he_conv2d_tc_workspace_bytes(const fl_ctx* ctx, const fl_conv_geom* geom, int B) {
  if (!ctx || !geom || B < 0) return 0;
  return 2 * fl_he_conv2d_workspace_bytes(ctx, geom, B) +
         4 * fl::tc_scratch_words(B, fl::ConvDims{geom->Cout, geom->G, geom->n_in, geom->n_out, geom->bands}, ctx->L,
                                  ctx->N);
}

// Checks shared by the tensor-core entry points; the workspace holds the NTT
// images of the inputs, their slot-tiled copy, then the NTT-domain outputs
// in slot-tiled order (the scratch).
static int tc_checks(fl_ctx* ctx, const fl_conv_geom* geom, int B, size_t workspace_bytes) {
  int rc;
  if ((rc = conv_checks(ctx, geom, B, workspace_bytes))) return rc;
  const size_t need = fl_he_conv2d_tc_workspace_bytes(ctx, geom, B);
  if (workspace_bytes < need) return fail(FL_ERR_ARG, "workspace %zu bytes, need %zu", workspace_bytes, need);
  if (geom->G > FL_TC_MAX_G)
    return fail(FL_ERR_SHAPE, "G=%d input ciphertexts per band: above %d, the fp32 partial sums of the digit "
                "products would no longer be exact", geom->G, FL_TC_MAX_G);
  return FL_OK;
}

static uint32_t* tc_scratch(fl_ctx* ctx, const fl_conv_geom* geom, int B, const void* ws) {
  return (uint32_t*)ws + 2 * (fl_he_conv2d_workspace_bytes(ctx, geom, B) / 4);
}

// slot-tiled copy of the NTT images (the workspace's second part), then the
// tensor-core contraction into the scratch (its third part); the
// contraction follows the copy as a programmatic dependent launch
static int stage_tc(fl_ctx* ctx, const fl_conv_geom* geom, int B, const uint16_t* w_tc_dev, const void* ws,
                    cudaStream_t st) {
  const uint32_t* c_hat = (const uint32_t*)ws;
  uint32_t* c_tc = (uint32_t*)ws + fl_he_conv2d_workspace_bytes(ctx, geom, B) / 4;
  int rc;
  if ((rc = launched(fl::launch_tc_inputs(c_hat, c_tc, B, geom->n_in, ctx->L, ctx->N, st), "tensor-core input layout")))
    return rc;
  return launched(fl::launch_conv_tc(B, fl::ConvDims{geom->Cout, geom->G, geom->n_in, geom->n_out, geom->bands},
                                     w_tc_dev, c_tc, tc_scratch(ctx, geom, B, ws), ctx->N, ctx->cc, ctx->tc_err, st,
                                     true, ctx->tc_tile),
                  "tensor-core contraction");
}

// the output ciphertexts are gathered from the workspace: they may not
// overlap it, and their rows must fit one launch
static int tc_out_checks(fl_ctx* ctx, const fl_conv_geom* geom, int B, const void* ws, const uint32_t* ct_out_dev) {
  if ((long long)2 * B * geom->bands * geom->Cout > 0x7fffffffLL)
    return fail(FL_ERR_ARG, "B=%d: too many output rows for one launch", B);
  const char* a = (const char*)ws;
  const char* b = (const char*)ct_out_dev;
  const size_t ws_bytes = fl_he_conv2d_tc_workspace_bytes(ctx, geom, B),
               out_bytes = (size_t)B * geom->n_out * 2 * ctx->L * ctx->N * 4;
  if (a < b + out_bytes && b < a + ws_bytes) return fail(FL_ERR_ARG, "output ciphertexts overlap the workspace");
  return FL_OK;
}

// the inverse NTT + mask of every scratch row into the output ciphertexts
// (after tc_out_checks)
static int stage_intt_rows(fl_ctx* ctx, const fl_conv_geom* geom, int B, const void* ws, const uint32_t* r_dev,
                           uint32_t* ct_out_dev, cudaStream_t st, bool pdl) {
  return launched(fl::launch_intt_mask_rows(ctx->logN, B,
                                            fl::ConvDims{geom->Cout, geom->G, geom->n_in, geom->n_out, geom->bands},
                                            tc_scratch(ctx, geom, B, ws), ct_out_dev, r_dev, ctx->tw, ctx->cc, st, pdl,
                                            ctx->ntt_plan),
                  "output inverse ntt");
}

int fl_he_conv2d_tc(fl_ctx* ctx, const fl_conv_geom* geom, int B, const uint16_t* w_tc_dev, const uint32_t* ct_in_dev,
                    const uint32_t* r_dev, uint32_t* ct_out_dev, void* workspace_dev, size_t workspace_bytes,
                    void* stream) {
  int rc;
  if ((rc = tc_checks(ctx, geom, B, workspace_bytes))) return rc;
  if (B == 0) return FL_OK;
  if ((rc = check_ptrs({w_tc_dev, ct_in_dev, ct_out_dev, workspace_dev}))) return rc;
  if (r_dev && (rc = check_ptrs({r_dev}))) return rc;
  if ((rc = tc_out_checks(ctx, geom, B, workspace_dev, ct_out_dev))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = stage_ntt(ctx, geom, B, ct_in_dev, workspace_dev, st))) return rc;
  if ((rc = stage_tc(ctx, geom, B, w_tc_dev, workspace_dev, st))) return rc;
  return stage_intt_rows(ctx, geom, B, workspace_dev, r_dev, ct_out_dev, st, true);
}

int fl_he_conv2d_tc_from_ntt(fl_ctx* ctx, const fl_conv_geom* geom, int B, const uint16_t* w_tc_dev,
                             void* workspace_dev, size_t workspace_bytes, void* stream) {
  int rc;
  if ((rc = tc_checks(ctx, geom, B, workspace_bytes))) return rc;
  if (B == 0) return FL_OK;
  if ((rc = check_ptrs({w_tc_dev, workspace_dev}))) return rc;
  return stage_tc(ctx, geom, B, w_tc_dev, workspace_dev, (cudaStream_t)stream);
}

int fl_intt_mask_outputs(fl_ctx* ctx, const fl_conv_geom* geom, int B, const void* workspace_dev,
                         size_t workspace_bytes, const uint32_t* r_dev, uint32_t* ct_out_dev, void* stream) {
  int rc;
  if ((rc = tc_checks(ctx, geom, B, workspace_bytes))) return rc;
  if (B == 0) return FL_OK;
  if ((rc = check_ptrs({workspace_dev, ct_out_dev}))) return rc;
  if (r_dev && (rc = check_ptrs({r_dev}))) return rc;
  if ((rc = tc_out_checks(ctx, geom, B, workspace_dev, ct_out_dev))) return rc;
  return stage_intt_rows(ctx, geom, B, workspace_dev, r_dev, ct_out_dev, (cudaStream_t)stream, false);
}

size_t fl_tc_weights_bytes(const fl_ctx* ctx, const fl_conv_geom* geom) {
  if (!ctx || !geom || geom->G < 1 || geom->G > FL_TC_MAX_G) return 0;
  return fl::tc_weights_bytes(ctx->L, geom->Cout, geom->G, ctx->N);
}

int fl_tc_weights(fl_ctx* ctx, const fl_conv_geom* geom, const uint32_t* w_hat_dev, uint16_t* w_tc_dev, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx)) || (rc = check_geom(ctx, geom))) return rc;
  if (geom->G > FL_TC_MAX_G)
    return fail(FL_ERR_SHAPE, "G=%d input ciphertexts per band: above %d, the tensor-core form is not exact",
                geom->G, FL_TC_MAX_G);
  if ((rc = check_ptrs({w_hat_dev, w_tc_dev}))) return rc;
  const size_t in_bytes = fl_weights_bytes(ctx, geom), out_bytes = fl_tc_weights_bytes(ctx, geom);
  const uintptr_t a = (uintptr_t)w_hat_dev, b = (uintptr_t)w_tc_dev;
  if (a < b + out_bytes && b < a + in_bytes) return fail(FL_ERR_ARG, "w_hat and w_tc overlap");
  return launched(fl::launch_tc_weights(w_hat_dev, w_tc_dev, ctx->L, geom->Cout, geom->G, ctx->N, (cudaStream_t)stream),
                  "tensor-core weight tiles");
}

int fl_tc_error(fl_ctx* ctx, void* stream, uint64_t* error_host) {
  int rc;
  if ((rc = check_ctx(ctx))) return rc;
  if (!error_host) return fail(FL_ERR_ARG, "null error_host");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  unsigned long long v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, ctx->tc_err, sizeof v, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) e = cudaMemset(ctx->tc_err, 0, sizeof v);
  if (e != cudaSuccess) return cuda_fail(e, "error word");
  *error_host = v;
  return v ? fail(FL_ERR_TIMEOUT, "a bounded tensor-core wait gave up (error word 0x%llx)", v) : FL_OK;
}

int fl_he_conv2d_direct(fl_ctx* ctx, const fl_conv_geom* geom, int B, const int8_t* w_dev, const uint32_t* ct_in_dev,
                        const uint32_t* r_dev, uint32_t* ct_out_dev, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx)) || (rc = check_geom(ctx, geom))) return rc;
  if (B < 0) return fail(FL_ERR_ARG, "B=%d", B);
  if ((long long)geom->Cin * geom->k * geom->k > FL_DIRECT_MAX_TAPS)
    return fail(FL_ERR_SHAPE, "Cin*k*k=%lld above %d for the direct form",
                (long long)geom->Cin * geom->k * geom->k, FL_DIRECT_MAX_TAPS);
  if (B == 0) return FL_OK;
  if (!w_dev) return fail(FL_ERR_ARG, "null filters");
  if ((rc = check_ptrs({ct_in_dev, ct_out_dev}))) return rc;
  if (r_dev && (rc = check_ptrs({r_dev}))) return rc;
  return launched(fl::launch_direct(ctx->logN, B, dims_of(*geom), w_dev, ct_in_dev, ct_out_dev, r_dev, ctx->cc,
                                    (cudaStream_t)stream),
                  "direct conv");
}

int fl_mask_to_share(fl_ctx* ctx, int n, uint32_t* ct_dev, const uint32_t* r_dev, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx))) return rc;
  if (n < 0) return fail(FL_ERR_ARG, "n=%d", n);
  if (n == 0) return FL_OK;
  if ((rc = check_ptrs({ct_dev, r_dev}))) return rc;
  return launched(fl::launch_mask(ct_dev, r_dev, n, ctx->N, ctx->cc, (cudaStream_t)stream), "mask");
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
static const size_t kStackCtlBytes = 256;

size_t fl_stack_workspace_bytes(const fl_ctx* ctx, const fl_stack_layer* layers, int n_layers) {
  if (!ctx || !layers || n_layers < 0) return 0;
  size_t total = kStackCtlBytes;
  for (int i = 0; i < n_layers; ++i) {
    if (!layers[i].geom || layers[i].B < 0) return 0;
    total += align256((size_t)layers[i].B * layers[i].geom->n_in * 2 * ctx->L * ctx->N * 4);
  }
  return total;
}

// stages: 1 = input NTT, 2 = persistent kernel, 3 = both
static int stack_impl(fl_ctx* ctx, const fl_stack_layer* layers, int n_layers, void* workspace_dev,
                      size_t workspace_bytes, void* stream, int stages) {
  int rc;
  if ((rc = check_ctx(ctx))) return rc;
  if (n_layers < 0 || n_layers > FL_STACK_MAX_LAYERS)
    return fail(FL_ERR_ARG, "n_layers=%d outside [0, %d]", n_layers, FL_STACK_MAX_LAYERS);
  if (n_layers > 0 && !layers) return fail(FL_ERR_ARG, "null layers");
  if ((rc = check_ptrs({workspace_dev}))) return rc;
  const size_t need = fl_stack_workspace_bytes(ctx, layers, n_layers);
  if (need == 0 || workspace_bytes < need)
    return fail(FL_ERR_ARG, "workspace %zu bytes, need %zu", workspace_bytes, need);
  fl::StackArgs a;
  memset(&a, 0, sizeof a);
  fl::NttSegs segs;
  memset(&segs, 0, sizeof segs);
  char* ws = (char*)workspace_dev + kStackCtlBytes;
  long long items = 0;
  int rows = 0;
  for (int i = 0; i < n_layers; ++i) {
    const fl_stack_layer& y = layers[i];
    if ((rc = check_geom(ctx, y.geom))) return fail(rc, "layer %d: %s", i, g_err.c_str());
    if (y.B == 0) continue;
    if ((rc = check_ptrs({y.w_hat_dev, y.ct_in_dev, y.ct_out_dev})))
      return fail(rc, "layer %d: %s", i, g_err.c_str());
    if (y.r_dev && (rc = check_ptrs({y.r_dev}))) return fail(rc, "layer %d: %s", i, g_err.c_str());
    const fl_conv_geom& g = *y.geom;
    const size_t cbytes = (size_t)y.B * g.n_in * 2 * ctx->L * ctx->N * 4;
    const long long seg_rows = (long long)y.B * g.n_in * 2 * ctx->L;
    if (rows + seg_rows > 0x7fffffffLL) return fail(FL_ERR_ARG, "too many input rows");
    const int k = segs.n++;
    segs.src[k] = y.ct_in_dev;
    segs.dst[k] = (uint32_t*)ws;
    segs.row_begin[k] = rows;
    rows += (int)seg_rows;
    fl::StackLayer& s = a.layer[a.n_layers++];
    s.w_hat = y.w_hat_dev;
    s.c_hat = (const uint32_t*)ws;
    s.out = y.ct_out_dev;
    s.r = y.r_dev;
    s.Cout = g.Cout;
    s.G = g.G;
    s.n_in = g.n_in;
    s.n_out = g.n_out;
    s.bands = g.bands;
    s.BB = y.B * g.bands;
    s.item_begin = items;
    items += (long long)s.BB * g.Cout * ctx->L;
    ws += align256(cbytes);
  }
  segs.row_begin[segs.n] = rows;
  a.n_items = items;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* ctl = (unsigned long long*)workspace_dev;
  cudaError_t e;
  // queue head and error word: zeroed before the input NTT, so that the
  // queue kernel (or a single per-layer launch) follows the NTT directly as a
  // programmatic dependent; the persistent kernel's launcher zeroes its own
  if ((stages & 2) && ctx->stack_kernel != FL_STACK_PERSISTENT &&
      (e = cudaMemsetAsync(ctl, 0, 2 * sizeof(unsigned long long), st)) != cudaSuccess)
    return cuda_fail(e, "control reset");
  if ((stages & 1) &&
      (rc = launched(fl::launch_ntt_multi(ctx->logN, segs, ctx->tw, ctx->cc, st, ctx->ntt_plan), "stack input ntt")))
    return rc;
  if (!(stages & 2)) return FL_OK;
  if (ctx->stack_kernel == FL_STACK_PERSISTENT)
    return launched(fl::launch_stack(ctx->logN, a, ctl, ctx->tw, ctx->cc, ctx->sms, st), "stack");
  if (ctx->stack_kernel == FL_STACK_QUEUE)
    return launched(fl::launch_conv_queue(ctx->logN, a, ctl, ctx->tw, ctx->cc, ctx->sms, st), "stack queue");
  // per-layer fused launches; the error word stays 0 (these kernels never
  // wait).  The layers are independent, so they fan out over the context's
  // auxiliary streams and join back into `st`.
  const int fan = a.n_layers < kAuxStreams ? a.n_layers : kAuxStreams;
  if (fan > 1) {
    if ((e = cudaEventRecord(ctx->fork_ev, st)) != cudaSuccess) return cuda_fail(e, "fork");
    for (int k = 0; k < fan; ++k)
      if ((e = cudaStreamWaitEvent(ctx->aux[k], ctx->fork_ev, 0)) != cudaSuccess) return cuda_fail(e, "fork");
  }
  for (int k = 0; k < a.n_layers; ++k) {
    const fl::StackLayer& y = a.layer[k];
    fl::ConvDims cd{y.Cout, y.G, y.n_in, y.n_out, y.bands};
    cudaStream_t sk = fan > 1 ? ctx->aux[k % fan] : st;
    // on `st` itself (one layer) the launch follows the input NTT as a programmatic dependent
    if ((rc = launched(fl::launch_conv_intt(ctx->logN, y.BB / y.bands, cd, y.w_hat, y.c_hat, y.out, y.r, ctx->tw,
                                            ctx->cc, sk, fan <= 1),
                       "stack layer")))
      return rc;
  }
  if (fan > 1) {
    for (int k = 0; k < fan; ++k) {
      if ((e = cudaEventRecord(ctx->join_ev[k], ctx->aux[k])) != cudaSuccess) return cuda_fail(e, "join");
      if ((e = cudaStreamWaitEvent(st, ctx->join_ev[k], 0)) != cudaSuccess) return cuda_fail(e, "join");
    }
  }
  return FL_OK;
}

int fl_ctx_set_stack_kernel(fl_ctx* ctx, int kernel) {
  if (!ctx) return fail(FL_ERR_ARG, "null context");
  if (kernel != FL_STACK_PER_LAYER && kernel != FL_STACK_PERSISTENT && kernel != FL_STACK_QUEUE)
    return fail(FL_ERR_ARG, "kernel=%d", kernel);
  ctx->stack_kernel = kernel;
  return FL_OK;
}

int fl_ctx_get_stack_kernel(const fl_ctx* ctx) { return ctx ? ctx->stack_kernel : FL_ERR_ARG; }

int fl_ctx_set_ntt_plan(fl_ctx* ctx, int r1) {
  int rc;
  if ((rc = check_ctx(ctx))) return rc;
  if (!fl::plan_available(ctx->logN, r1))
    return fail(FL_ERR_ARG, "pass plan r1=%d is not available at N=%d", r1, ctx->N);
  ctx->ntt_plan = r1;
  return FL_OK;
}

int fl_ctx_get_ntt_plan(const fl_ctx* ctx) { return ctx ? (ctx->ntt_plan ? ctx->ntt_plan : fl::default_plan_r1(ctx->logN)) : 0; }

int fl_ctx_set_tc_tile(fl_ctx* ctx, int groups) {
  int rc;
  if ((rc = check_ctx(ctx))) return rc;
  if (groups != 0 && groups != 4 && groups != 8 && groups != 16 && groups != 32 && groups != 64)
    return fail(FL_ERR_ARG, "tensor-core tile of %d slot groups (4, 8, 16, 32 or 64)", groups);
  ctx->tc_tile = groups;
  return FL_OK;
}

int fl_ctx_get_tc_tile(const fl_ctx* ctx) { return ctx ? (ctx->tc_tile ? ctx->tc_tile : 32) : 0; }

int fl_he_conv2d_stack(fl_ctx* ctx, const fl_stack_layer* layers, int n_layers, void* workspace_dev,
                       size_t workspace_bytes, void* stream) {
  return stack_impl(ctx, layers, n_layers, workspace_dev, workspace_bytes, stream, 3);
}

int fl_he_conv2d_stack_ntt(fl_ctx* ctx, const fl_stack_layer* layers, int n_layers, void* workspace_dev,
                           size_t workspace_bytes, void* stream) {
  return stack_impl(ctx, layers, n_layers, workspace_dev, workspace_bytes, stream, 1);
}

int fl_he_conv2d_stack_run(fl_ctx* ctx, const fl_stack_layer* layers, int n_layers, void* workspace_dev,
                           size_t workspace_bytes, void* stream) {
  return stack_impl(ctx, layers, n_layers, workspace_dev, workspace_bytes, stream, 2);
}

int fl_stack_error(const void* workspace_dev, void* stream, uint64_t* error_host) {
  if (!workspace_dev || !error_host) return fail(FL_ERR_ARG, "null pointer");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream sync");
  unsigned long long v = 0;
  e = cudaMemcpy(&v, (const unsigned long long*)workspace_dev + 1, sizeof v, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "error word read");
  *error_host = v;
  return v ? fail(FL_ERR_TIMEOUT, "a bounded device wait gave up (error word 0x%llx)", v) : FL_OK;
}

int fl_selftest_wait_timeout(void* stream, uint64_t* error_host) {
  if (!error_host) return fail(FL_ERR_ARG, "null pointer");
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof *d);
  if (e != cudaSuccess) return cuda_fail(e, "error word");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long v = 0;
  if ((e = cudaMemsetAsync(d, 0, sizeof *d, st)) == cudaSuccess &&
      (e = fl::launch_wait_timeout_probe(d, st)) == cudaSuccess && (e = cudaStreamSynchronize(st)) == cudaSuccess)
    e = cudaMemcpy(&v, d, sizeof v, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "wait probe");
  *error_host = v;
  return v ? fail(FL_ERR_TIMEOUT, "the probe's wait gave up as designed (error word 0x%llx)", v) : FL_OK;
}

int fl_ntt_forward(fl_ctx* ctx, int n, uint32_t* data_dev, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx))) return rc;
  if (n < 0) return fail(FL_ERR_ARG, "n=%d", n);
  if (n == 0) return FL_OK;
  if ((rc = check_ptrs({data_dev})) || (rc = rows_ok((long long)n * ctx->L, "ntt"))) return rc;
  const int rows = n * ctx->L;
  return launched(fl::launch_ntt_fwd(ctx->logN, rows, data_dev, rows, 0, data_dev, rows, 0, 1, ctx->tw, ctx->cc,
                                     (cudaStream_t)stream, ctx->ntt_plan),
                  "ntt");
}

int fl_ntt_inverse(fl_ctx* ctx, int n, uint32_t* data_dev, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx))) return rc;
  if (n < 0) return fail(FL_ERR_ARG, "n=%d", n);
  if (n == 0) return FL_OK;
  if ((rc = check_ptrs({data_dev})) || (rc = rows_ok((long long)n * ctx->L, "intt"))) return rc;
  return launched(fl::launch_ntt_inv(ctx->logN, n * ctx->L, data_dev, ctx->tw, ctx->cc, (cudaStream_t)stream),
                  "intt");
}

// ---------------------------------------------------------------------------
// Batch encoding and the x^2 + x protocol, server side (Sec. 5.2)
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {
int check_batch(const fl_ctx* ctx) {
  if (!ctx->batch)
    return fail(FL_ERR_ARG, "batch encoding needs t prime with t = 1 mod 2N (t=%u, N=%d)", ctx->t, ctx->N);
  return FL_OK;
}
const uint32_t* tw_t(const fl_ctx* ctx) { return ctx->tw + (size_t)ctx->L * fl::twiddle_limb_words(ctx->logN); }
}  // namespace

extern "C" {

int fl_batch_encode(fl_ctx* ctx, int n, const uint32_t* slots_dev, uint32_t* m_dev, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx)) || (rc = check_batch(ctx))) return rc;
  if (n < 0) return fail(FL_ERR_ARG, "n=%d", n);
  if (n == 0) return FL_OK;
  if ((rc = check_ptrs({slots_dev, m_dev}))) return rc;
  return launched(fl::launch_batch_encode(ctx->logN, n, slots_dev, 1, m_dev, ctx->N, 0, tw_t(ctx), ctx->tc, ctx->cc,
                                          (cudaStream_t)stream),
                  "batch encode");
}

int fl_batch_decode(fl_ctx* ctx, int n, const uint32_t* m_dev, uint32_t* slots_dev, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx)) || (rc = check_batch(ctx))) return rc;
  if (n < 0) return fail(FL_ERR_ARG, "n=%d", n);
  if (n == 0) return FL_OK;
  if ((rc = check_ptrs({slots_dev, m_dev}))) return rc;
  return launched(fl::launch_batch_decode(ctx->logN, n, m_dev, slots_dev, tw_t(ctx), ctx->tc, (cudaStream_t)stream),
                  "batch decode");
}

size_t fl_x2x_prep_bytes(const fl_ctx* ctx, int n) {
  if (!ctx || n < 0) return 0;
  return (size_t)n * (ctx->L + 2) * ctx->N * sizeof(uint32_t);
}

int fl_x2x_prepare(fl_ctx* ctx, int n, const uint32_t* r_dev, const uint32_t* v_dev, uint32_t* prep_dev,
                   void* stream) {
  int rc;
  if ((rc = check_ctx(ctx)) || (rc = check_batch(ctx))) return rc;
  if (n < 0) return fail(FL_ERR_ARG, "n=%d", n);
  if (n == 0) return FL_OK;
  if ((rc = check_ptrs({r_dev, v_dev, prep_dev})) || (rc = rows_ok((long long)n * (ctx->L + 2), "x2x prepare")))
    return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int L = ctx->L, N = ctx->N;
  const long long stride = (long long)(L + 2) * N;
  cudaError_t e;
  // rows [0, L): lift of encode(2r) per limb, then NTT in place
  if ((e = fl::launch_batch_encode(ctx->logN, n, r_dev, 2, prep_dev, stride, L, tw_t(ctx), ctx->tc, ctx->cc, st)))
    return cuda_fail(e, "encode 2r");
  if ((e = fl::launch_ntt_fwd(ctx->logN, n * L, prep_dev, L, L + 2, prep_dev, L, L + 2, 1, ctx->tw, ctx->cc, st)))
    return cuda_fail(e, "ntt of 2r");
  // row L: encode(v) in [0, t); row L+1: r^2 - r + v mod t (direct encoding)
  if ((e = fl::launch_batch_encode(ctx->logN, n, v_dev, 1, prep_dev + (size_t)L * N, stride, 0, tw_t(ctx), ctx->tc,
                                   ctx->cc, st)))
    return cuda_fail(e, "encode v");
  return launched(fl::launch_x2x_const(r_dev, v_dev, prep_dev + (size_t)(L + 1) * N, stride, n, N, ctx->tc, st),
                  "r^2 - r + v");
}

int fl_x2x_round1(fl_ctx* ctx, int n, const uint32_t* prep_dev, const uint32_t* ct_z_dev, uint32_t* ct_out_dev,
                  void* stream) {
  int rc;
  if ((rc = check_ctx(ctx)) || (rc = check_batch(ctx))) return rc;
  if (n < 0) return fail(FL_ERR_ARG, "n=%d", n);
  if (n == 0) return FL_OK;
  if ((rc = check_ptrs({prep_dev, ct_z_dev, ct_out_dev})) || (rc = rows_ok((long long)n * 2 * ctx->L, "x2x round 1")))
    return rc;
  return launched(fl::launch_x2x_round1(ctx->logN, n, prep_dev, ct_z_dev, ct_out_dev, ctx->tw, ctx->cc,
                                        (cudaStream_t)stream),
                  "x2x round 1");
}

int fl_x2x_round2(fl_ctx* ctx, int n, const uint32_t* prep_dev, const uint32_t* ct_x_dev, const uint32_t* ct_y_dev,
                  uint32_t* ct_out_dev, void* stream) {
  int rc;
  if ((rc = check_ctx(ctx)) || (rc = check_batch(ctx))) return rc;
  if (n < 0) return fail(FL_ERR_ARG, "n=%d", n);
  if (n == 0) return FL_OK;
  if ((rc = check_ptrs({prep_dev, ct_x_dev, ct_y_dev, ct_out_dev}))) return rc;
  return launched(fl::launch_x2x_round2(prep_dev, ct_x_dev, ct_y_dev, ct_out_dev, n, ctx->N, ctx->cc,
                                        (cudaStream_t)stream),
                  "x2x round 2");
}

int fl_repack_outputs(const fl_conv_geom* prev, const fl_conv_geom* next, int B, const uint32_t* src_dev,
                      uint32_t* dst_dev, void* stream) {
  if (!prev || !next) return fail(FL_ERR_ARG, "null geometry");
  fl_conv_geom a, b;
  int rc;
  if ((rc = fl_conv_geom_make(prev->N, prev->Cin, prev->Cout, prev->H, prev->W, prev->k, prev->stride, prev->pad,
                              &a)) ||
      (rc = fl_conv_geom_make(next->N, next->Cin, next->Cout, next->H, next->W, next->k, next->stride, next->pad,
                              &b)))
    return rc;
  if (memcmp(&a, prev, sizeof a) || memcmp(&b, next, sizeof b))
    return fail(FL_ERR_SHAPE, "geometry fields are inconsistent (build them with fl_conv_geom_make)");
  if (prev->N != next->N || prev->Cout != next->Cin || prev->Ho != next->H || prev->Wo != next->W)
    return fail(FL_ERR_SHAPE, "layer outputs %dx%dx%d (N=%d) do not match next inputs %dx%dx%d (N=%d)", prev->Cout,
                prev->Ho, prev->Wo, prev->N, next->Cin, next->H, next->W, next->N);
  if (B < 0) return fail(FL_ERR_ARG, "B=%d", B);
  if (B == 0) return FL_OK;
  if ((rc = check_ptrs({src_dev, dst_dev}))) return rc;
  return launched(fl::launch_repack(src_dev, dst_dev, dims_of(*prev), dims_of(*next), B, next->N,
                                    (cudaStream_t)stream),
                  "repack");
}

}  // extern "C"
