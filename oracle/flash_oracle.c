/*
 * Flash HE-convolution oracle: a plain, slow, CPU restatement of what the
 * server-side homomorphic convolution computes, written from the paper
 * (Flash, arXiv 2401.16732) and nothing else.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this library.  It shares no source, table
 * or helper with the CUDA library; the two meet only through the seeded input
 * generator and the comparisons the tests make.
 *
 * Ring: R_q = Z_q[x]/(x^N + 1) (Sec. 2.2), q = prod q_l held as L residues
 * ("RNS limbs"), each q_l a prime below 2^30 with q_l = 1 mod 2N.
 * All arrays are limb-major: [L][N] for one polynomial, residues in [0, q_l).
 *
 * Each function names the passage it follows.  Nothing here is blocked,
 * fused or reordered beyond what those passages state.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

/* ------------------------------------------------------------------ */
/* Primes: the largest primes below 2^30 with q = 1 mod 2N, descending.  */
/* (RNS reading of the single ciphertext modulus q of Sec. 2.2, Table 1.) */
/* Primality by trial division: slow and obviously correct.             */
/* ------------------------------------------------------------------ */
int or_is_prime(uint32_t n)
{
    if (n < 2) return 0;
    if (n % 2 == 0) return n == 2;
    for (uint64_t d = 3; d * d <= n; d += 2)
        if (n % d == 0) return 0;
    return 1;
}

int or_find_primes(uint32_t N, int L, uint32_t *out)
{
    uint64_t step = 2ull * N;
    /* largest candidate below 2^30 that is 1 mod 2N */
    uint64_t c = ((((1ull << 30) - 1) - 1) / step) * step + 1;
    int found = 0;
    while (found < L && c > step) {
        if (or_is_prime((uint32_t)c)) out[found++] = (uint32_t)c;
        c -= step;
    }
    return found == L ? 0 : -1;
}

/* ------------------------------------------------------------------ */
/* Negacyclic schoolbook product out = a * b mod (x^N + 1, q).          */
/* Definition of multiplication in R_q (Sec. 2.2): x^N = -1, so a term  */
/* landing on exponent i + j >= N wraps to i + j - N with a minus sign.  */
/* Zero coefficients of `a` contribute nothing and are skipped.         */
/* ------------------------------------------------------------------ */
void or_negacyclic_mul(const uint32_t *a, const uint32_t *b, uint32_t N,
                       uint32_t q, uint32_t *out)
{
    i128 *acc = (i128 *)calloc(N, sizeof(i128));
    for (uint32_t i = 0; i < N; ++i) {
        if (a[i] == 0) continue;
        i128 ai = a[i];
        for (uint32_t j = 0; j < N; ++j) {
            uint32_t k = i + j;
            if (k < N) acc[k] += ai * b[j];
            else       acc[k - N] -= ai * b[j];
        }
    }
    for (uint32_t k = 0; k < N; ++k) {
        i128 r = acc[k] % (i128)q;
        if (r < 0) r += q;
        out[k] = (uint32_t)r;
    }
    free(acc);
}

/* ------------------------------------------------------------------ */
/* DRot (Eq. 2, proof in Appendix A): c'(x) = c(x) * x^{-step} mod       */
/* x^N + 1 for any step >= 0.  Since x^N = -1, x^{2N} = 1, so the step    */
/* counts modulo 2N, and coefficient i of the result is                  */
/* (-1)^floor((i+e)/N) * c[(i+e) mod N] with e = step mod 2N.  Here       */
/* i + e < 3N, so the sign flips once per multiple of N passed (zero, one */
/* or two times).  Every output coefficient is written.                  */
/* ------------------------------------------------------------------ */
static int64_t drot_coeff(const uint32_t *c, uint32_t N, uint32_t step,
                          uint32_t i)
{
    uint64_t idx = (uint64_t)i + step % (2ull * N);
    uint64_t wraps = idx / N;
    int64_t v = (int64_t)c[idx % N];
    return (wraps & 1) ? -v : v;
}

void or_drot(const uint32_t *c, uint32_t N, uint32_t q, uint32_t step,
             uint32_t *out)
{
    for (uint32_t i = 0; i < N; ++i) {
        int64_t v = drot_coeff(c, N, step, i);
        out[i] = (uint32_t)(v < 0 ? v + (int64_t)q : v) % q;
    }
}

/* ------------------------------------------------------------------ */
/* Private-key BFV encryption (Table 2, right column):                  */
/*   c0 = [-(a*s + e) + Delta*m]_q,  c1 = a.                             */
/* Per limb l: Delta_l = Delta mod q_l, s and e are small signed         */
/* polynomials, a is uniform in R_q (given as its residues).             */
/* ------------------------------------------------------------------ */
void or_encrypt(uint32_t N, int L, const uint32_t *q, const uint32_t *delta,
                const int8_t *s, const uint32_t *a, const int32_t *e,
                const uint32_t *m, uint32_t *c0, uint32_t *c1)
{
    uint32_t *sl = (uint32_t *)malloc(N * sizeof(uint32_t));
    uint32_t *as = (uint32_t *)malloc(N * sizeof(uint32_t));
    for (int l = 0; l < L; ++l) {
        uint32_t ql = q[l];
        for (uint32_t j = 0; j < N; ++j)
            sl[j] = (uint32_t)(((int64_t)s[j] % ql + ql) % ql);
        or_negacyclic_mul(sl, a + (size_t)l * N, N, ql, as);
        for (uint32_t j = 0; j < N; ++j) {
            int64_t v = -((int64_t)as[j] + e[j]) +
                        (int64_t)(((uint64_t)delta[l] * m[j]) % ql);
            v %= (int64_t)ql;
            if (v < 0) v += ql;
            c0[(size_t)l * N + j] = (uint32_t)v;
            c1[(size_t)l * N + j] = a[(size_t)l * N + j];
        }
    }
    free(sl);
    free(as);
}

/* Decryption phase per limb (Eq. in Appendix A, from [FV12]):            */
/*   [c1*s + c0]_{q_l}  =  (Delta*m + v) mod q_l.                          */
/* The CRT and the rounding to m are done with exact big integers by the   */
/* Python side.                                                            */
void or_phase(uint32_t N, int L, const uint32_t *q, const int8_t *s,
              const uint32_t *c0, const uint32_t *c1, uint32_t *out)
{
    uint32_t *sl = (uint32_t *)malloc(N * sizeof(uint32_t));
    uint32_t *cs = (uint32_t *)malloc(N * sizeof(uint32_t));
    for (int l = 0; l < L; ++l) {
        uint32_t ql = q[l];
        for (uint32_t j = 0; j < N; ++j)
            sl[j] = (uint32_t)(((int64_t)s[j] % ql + ql) % ql);
        or_negacyclic_mul(sl, c1 + (size_t)l * N, N, ql, cs);
        for (uint32_t j = 0; j < N; ++j)
            out[(size_t)l * N + j] =
                (uint32_t)(((uint64_t)cs[j] + c0[(size_t)l * N + j]) % ql);
    }
    free(sl);
    free(cs);
}

/* ------------------------------------------------------------------ */
/* Weight polynomial of output channel i and input ciphertext g:          */
/*   W_{i,g}(x) = sum_{jj < c_n, j = g*c_n + jj < Cin}                     */
/*                sum_{ky,kx} w[i][j][ky][kx] * x^{-(ky*Wp + kx + jj*P)}   */
/* This folds Algorithm 1's DRot(c, step_k) * filters[i][j][k] and the     */
/* alignment DRot(t, offset_j) into one plaintext polynomial, using        */
/* DRot(c, e) = c * x^{-e} (Eq. 2) and x^{-e} = -x^{N-e} for 0 < e < N.    */
/* Tap step ky*Wp + kx and offset jj*P are the readings of the paper's     */
/* DRot(c, k) and H*W*(j mod c_n) for a zero-padded plane of width Wp and  */
/* size P.  Output: residues mod q, length N.                              */
/* ------------------------------------------------------------------ */
void or_weight_poly(uint32_t N, uint32_t q, int Cin, int k, int Wp, int P,
                    int c_n, const int8_t *w_i /* [Cin][k][k] */, int g,
                    uint32_t *out)
{
    memset(out, 0, N * sizeof(uint32_t));
    for (int jj = 0; jj < c_n; ++jj) {
        int j = g * c_n + jj;
        if (j >= Cin) break;
        for (int ky = 0; ky < k; ++ky)
            for (int kx = 0; kx < k; ++kx) {
                int64_t wv = w_i[((size_t)j * k + ky) * k + kx];
                uint32_t e = (uint32_t)(ky * Wp + kx + jj * P);
                uint32_t pos;
                int64_t val;
                if (e == 0) { pos = 0; val = wv; }
                else        { pos = N - e; val = -wv; }
                int64_t cur = (int64_t)out[pos] + val;
                cur %= (int64_t)q;
                if (cur < 0) cur += q;
                out[pos] = (uint32_t)cur;
            }
    }
}

/* ------------------------------------------------------------------ */
/* Route O1 (the definition): output ciphertext (i, band) is              */
/*   y = ( sum_g W_{i,g} * c0_g , sum_g W_{i,g} * c1_g )  in R_q,           */
/* each product a negacyclic schoolbook product per limb.                  */
/* ct_in: [bands*G][2][L][N] for one image, input ct index band*G + g.     */
/* out:   [(i_hi - i_lo)*bands][2][L][N], output ct index (i-i_lo)*bands+b. */
/* ------------------------------------------------------------------ */
void or_conv_poly(uint32_t N, int L, const uint32_t *q, int Cin, int k,
                  int Wp, int P, int c_n, int G, int bands,
                  const int8_t *w /* [Cout][Cin][k][k] */,
                  const uint32_t *ct_in, int i_lo, int i_hi, uint32_t *out)
{
    size_t poly = N, ct = 2 * (size_t)L * N;
#pragma omp parallel
    {
        uint32_t *W = (uint32_t *)malloc(N * sizeof(uint32_t));
        uint32_t *prod = (uint32_t *)malloc(N * sizeof(uint32_t));
#pragma omp for collapse(2) schedule(dynamic)
        for (int i = i_lo; i < i_hi; ++i)
            for (int l = 0; l < L; ++l) {
                const int8_t *w_i = w + (size_t)i * Cin * k * k;
                for (int b = 0; b < bands; ++b)
                    for (int c = 0; c < 2; ++c) {
                        uint32_t *y = out + ((size_t)(i - i_lo) * bands + b) * ct +
                                      ((size_t)c * L + l) * poly;
                        memset(y, 0, N * sizeof(uint32_t));
                        for (int g = 0; g < G; ++g) {
                            or_weight_poly(N, q[l], Cin, k, Wp, P, c_n, w_i, g, W);
                            const uint32_t *x = ct_in + ((size_t)b * G + g) * ct +
                                                ((size_t)c * L + l) * poly;
                            or_negacyclic_mul(W, x, N, q[l], prod);
                            for (uint32_t u = 0; u < N; ++u)
                                y[u] = (uint32_t)(((uint64_t)y[u] + prod[u]) % q[l]);
                        }
                    }
            }
        free(W);
        free(prod);
    }
}

/* ------------------------------------------------------------------ */
/* Route O2: Algorithm 1 as the paper states it, with the lazy reduction  */
/* of Sec. 6.1 (accumulate unreduced, reduce once per partial sum) and    */
/* the output-channel parallelism of Sec. 6.2 (OpenMP over i).            */
/*   for i < c_o:  psum = 0                                                */
/*     for j < c_i:  c = x[j / c_n];  t = 0                                */
/*       for k < f_w^2:  t += DRot(c, step_k) * filters[i][j][k]           */
/*       psum += DRot(t, offset_j)                                         */
/*     y[i] = psum                                                         */
/* step_k = ky*Wp + kx and offset_j = (j mod c_n)*P (zero-padded planes).  */
/* Residues are below 2^30 and |w| <= 8, so |psum| < Cin*k^2*8*2^30 fits  */
/* a signed 64-bit word: 64-bit lazy accumulators play the role of the    */
/* paper's 128-bit ones for its 60-bit q.  Same layouts as or_conv_poly.  */
/* ------------------------------------------------------------------ */
void or_conv_alg1(uint32_t N, int L, const uint32_t *q, int Cin, int k,
                  int Wp, int P, int c_n, int G, int bands,
                  const int8_t *w, const uint32_t *ct_in, int i_lo, int i_hi,
                  uint32_t *out)
{
    size_t poly = N, ct = 2 * (size_t)L * N;
#pragma omp parallel
    {
        int64_t *t = (int64_t *)malloc(N * sizeof(int64_t));
        int64_t *psum = (int64_t *)malloc(N * sizeof(int64_t));
#pragma omp for collapse(2) schedule(dynamic)
        for (int i = i_lo; i < i_hi; ++i)
            for (int b = 0; b < bands; ++b)
                for (int c = 0; c < 2; ++c)
                    for (int l = 0; l < L; ++l) {
                        memset(psum, 0, N * sizeof(int64_t));
                        for (int j = 0; j < Cin; ++j) {
                            /* Let c = x[j / c_n] */
                            const uint32_t *x = ct_in + ((size_t)b * G + j / c_n) * ct +
                                                ((size_t)c * L + l) * poly;
                            memset(t, 0, N * sizeof(int64_t));
                            for (int ky = 0; ky < k; ++ky)
                                for (int kx = 0; kx < k; ++kx) {
                                    /* t += DRot(c, step_k) * filters[i][j][k] */
                                    int64_t wv = w[(((size_t)i * Cin + j) * k + ky) * k + kx];
                                    uint32_t step = (uint32_t)(ky * Wp + kx);
                                    for (uint32_t u = 0; u < N; ++u)
                                        t[u] += wv * drot_coeff(x, N, step, u);
                                }
                            /* psum += DRot(t, offset_j) */
                            uint32_t off = (uint32_t)((j % c_n) * P);
                            for (uint32_t u = 0; u < N; ++u) {
                                uint32_t idx = u + off;
                                psum[u] += idx < N ? t[idx] : -t[idx - N];
                            }
                        }
                        /* one reduction per partial sum (lazy reduction) */
                        uint32_t *y = out + ((size_t)(i - i_lo) * bands + b) * ct +
                                      ((size_t)c * L + l) * poly;
                        for (uint32_t u = 0; u < N; ++u) {
                            int64_t r = psum[u] % (int64_t)q[l];
                            y[u] = (uint32_t)(r < 0 ? r + q[l] : r);
                        }
                    }
        free(t);
        free(psum);
    }
}

/* ------------------------------------------------------------------ */
/* Mask addition (Sec. 5.2): the server adds the plaintext r to the       */
/* encrypted convolution result, c0 <- c0 + Delta*r (c1 unchanged), so    */
/* that the client decrypts a + r.  r is given (pre-generated offline,    */
/* Sec. 6.3), values in [0, t).  c0: [L][N].                              */
/* ------------------------------------------------------------------ */
void or_mask(uint32_t N, int L, const uint32_t *q, const uint32_t *delta,
             const uint32_t *r, uint32_t *c0)
{
    for (int l = 0; l < L; ++l)
        for (uint32_t u = 0; u < N; ++u) {
            uint64_t v = (uint64_t)c0[(size_t)l * N + u] +
                         ((uint64_t)delta[l] * r[u]) % q[l];
            c0[(size_t)l * N + u] = (uint32_t)(v % q[l]);
        }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Batch (SIMD) encoding over Z_t[x]/(x^N+1) (Sec. 2.2; used by the x^2+x */
/* protocol of Sec. 5.2).  Slot k of a plaintext m is its value at the    */
/* root psi_t^(2k+1), psi_t a primitive 2N-th root of unity mod t.         */
/*   decode: s_k = m(psi_t^(2k+1)) mod t                                   */
/*   encode: m_j = N^-1 * sum_k s_k * psi_t^(-(2k+1) j) mod t              */
/* (the interpolation formula: the N roots are distinct and x^N+1 splits). */
/* ------------------------------------------------------------------ */
static uint64_t or_powmod(uint64_t b, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = r * b % m;
        b = b * b % m;
        e >>= 1;
    }
    return r;
}

void or_batch_decode(uint32_t N, uint32_t t, uint32_t psi, const uint32_t *m, uint32_t *s)
{
    for (uint32_t k = 0; k < N; ++k) {
        uint64_t z = or_powmod(psi, 2ull * k + 1, t), zp = 1, acc = 0;
        for (uint32_t j = 0; j < N; ++j) {
            acc = (acc + (uint64_t)m[j] * zp) % t;
            zp = zp * z % t;
        }
        s[k] = (uint32_t)acc;
    }
}

void or_batch_encode(uint32_t N, uint32_t t, uint32_t psi, const uint32_t *s, uint32_t *m)
{
    uint64_t psi_inv = or_powmod(psi, t - 2, t);
    uint64_t n_inv = or_powmod(N, t - 2, t);
    for (uint32_t j = 0; j < N; ++j) {
        /* sum_k s_k * (psi^-(2k+1))^j = psi^-j * sum_k s_k * (psi^-2j)^k */
        uint64_t step = or_powmod(psi_inv, 2ull * j, t), zp = or_powmod(psi_inv, j, t), acc = 0;
        for (uint32_t k = 0; k < N; ++k) {
            acc = (acc + (uint64_t)s[k] * zp) % t;
            zp = zp * step % t;
        }
        m[j] = (uint32_t)(acc * n_inv % t);
    }
}
