"""Flash HE-convolution oracle (Python side).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The CUDA library never
imports, links or calls it, and it imports nothing from the CUDA library.

What it computes, and where the paper defines it (Flash, arXiv 2401.16732):

* ring and RNS primes ........ Sec. 2.2 / Table 1 (q held as L primes < 2^30)
* direct encoding ............ Eq. 1 (coefficient i holds m[i])
* zero-padded channel packing  Sec. 3.3 (client sends zero-padded inputs),
                               Algorithm 1 (c_n channels per ciphertext)
* private-key encryption ..... Table 2
* DRot ........................ Eq. 2 and the theorem of Appendix A
* convolution ................. Algorithm 1 (route O2) and its closed form
                               sum_g W_{i,g} * ct_g (route O1)
* lazy reduction .............. Sec. 6.1
* decryption / noise .......... Appendix A, Delta*m + v = [c1*s + c0]_q
* mask addition ................ Sec. 5.2 (HAdd of r) and Sec. 2.3 shares

Readings where the paper is silent or garbled are stated at each function.
Parity pins (tests/test_oracle_*.py) check every function here against
brute force, closed forms and textbook identities.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flash_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

T_DEFAULT = 65537


def build(force: bool = False) -> str:
    """Compile the C core of the oracle (plain gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", _LIB_PATH, _SRC])
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i8p = ctypes.POINTER(ctypes.c_int8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u32, i32 = ctypes.c_uint32, ctypes.c_int
        L.or_is_prime.argtypes = [u32]
        L.or_find_primes.argtypes = [u32, i32, u32p]
        L.or_negacyclic_mul.argtypes = [u32p, u32p, u32, u32, u32p]
        L.or_drot.argtypes = [u32p, u32, u32, u32, u32p]
        L.or_encrypt.argtypes = [u32, i32, u32p, u32p, i8p, u32p, i32p, u32p, u32p, u32p]
        L.or_phase.argtypes = [u32, i32, u32p, i8p, u32p, u32p, u32p]
        L.or_weight_poly.argtypes = [u32, u32, i32, i32, i32, i32, i32, i8p, i32, u32p]
        conv = [u32, i32, u32p, i32, i32, i32, i32, i32, i32, i32, i8p, u32p, i32, i32, u32p]
        L.or_conv_poly.argtypes = conv
        L.or_conv_alg1.argtypes = conv
        L.or_mask.argtypes = [u32, i32, u32p, u32p, u32p, u32p]
        L.or_num_threads.restype = ctypes.c_int
        L.or_batch_encode.argtypes = [u32, u32, u32, u32p, u32p]
        L.or_batch_decode.argtypes = [u32, u32, u32, u32p, u32p]
        _lib = L
    return _lib


def _p(a: np.ndarray, ctype):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------
def find_primes(N: int, L: int) -> list[int]:
    """Largest L primes below 2^30 with q = 1 mod 2N, descending (trial division)."""
    out = np.zeros(L, np.uint32)
    if lib().or_find_primes(N, L, _p(out, ctypes.c_uint32)) != 0:
        raise ValueError("not enough primes")
    return [int(v) for v in out]


def delta_residues(primes: list[int], t: int) -> list[int]:
    """Delta = floor(q/t) with q = prod q_l (Table 1), reduced per limb."""
    q = math.prod(primes)
    d = q // t
    return [d % ql for ql in primes]


@dataclass(frozen=True)
class Geometry:
    """Ciphertext layout of one convolution layer.

    Readings (the paper is silent or garbled on these points):
    * padded plane: the client zero-pads (Sec. 3.3), Hp = H + 2p, Wp = W + 2p;
    * DRot step of tap (ky, kx) is ky*Wp + kx (Algorithm 1 writes k, a 1-D index);
    * alignment offset of packed channel j is (j mod c_n) * P with P the padded
      plane size (Algorithm 1 writes H*W*(j mod c_n));
    * c_n = floor(N / P) channels per ciphertext (Algorithm 1 leaves c_n open);
    * stride s > 1: the stride-1 polynomial product is evaluated and output
      (oy, ox) is read at coefficient (s*oy)*Wp + s*ox;
    * a padded plane larger than N is split into row bands (Sec. 3.1 splits
      large inputs over several ciphertexts): Rin = floor(N / Wp) padded rows per
      ciphertext, Rout = floor((Rin - k)/s) + 1 output rows per band, band b
      starts at padded row b*Rout*s; one channel per ciphertext;
    * input ciphertext index band*G + g; output ciphertext index i*bands + band
      (one output ciphertext per output channel, Sec. 3.3).
    """
    N: int
    Cin: int
    Cout: int
    H: int
    W: int
    k: int
    s: int
    p: int
    Hp: int
    Wp: int
    Ho: int
    Wo: int
    Rin: int
    Rout: int
    bands: int
    P: int
    c_n: int
    G: int
    n_in: int
    n_out: int


def geometry(N, Cin, Cout, H, W, k, s=1, p=0) -> Geometry:
    Hp, Wp = H + 2 * p, W + 2 * p
    Ho, Wo = (Hp - k) // s + 1, (Wp - k) // s + 1
    if Hp * Wp <= N:
        Rin, Rout, bands = Hp, Ho, 1
    else:
        Rin = N // Wp
        if Rin < k:
            raise ValueError("padded row too long for one ciphertext")
        Rout = (Rin - k) // s + 1
        bands = -(-Ho // Rout)
    P = Rin * Wp
    c_n = N // P
    G = -(-Cin // c_n)
    return Geometry(N, Cin, Cout, H, W, k, s, p, Hp, Wp, Ho, Wo, Rin, Rout,
                    bands, P, c_n, G, bands * G, Cout * bands)


# ---------------------------------------------------------------------------
# Client side: packing (Eq. 1, zero padding, c_n channels per ct)
# ---------------------------------------------------------------------------
def pack_inputs(x: np.ndarray, geo: Geometry) -> np.ndarray:
    """Direct-encode one image x[Cin][H][W] (values in [0, t)) into
    geo.n_in plaintext polynomials [n_in][N] (uint32).

    Coefficient jj*P + y*Wp + xx of ciphertext band*G + g holds the zero-padded
    input of channel j = g*c_n + jj at padded row band*Rout*s + y, column xx.
    """
    Cin, H, W = x.shape
    xp = np.zeros((Cin, geo.Hp, geo.Wp), np.int64)
    xp[:, geo.p:geo.p + H, geo.p:geo.p + W] = x
    m = np.zeros((geo.n_in, geo.N), np.uint32)
    for band in range(geo.bands):
        r0 = band * geo.Rout * geo.s
        for j in range(Cin):
            g, jj = divmod(j, geo.c_n)
            plane = np.zeros((geo.Rin, geo.Wp), np.int64)
            rows = xp[j, r0:r0 + geo.Rin]
            plane[:rows.shape[0]] = rows
            m[band * geo.G + g, jj * geo.P: jj * geo.P + geo.P] = plane.ravel()
    return m


def extract_outputs(mpoly: np.ndarray, geo: Geometry) -> np.ndarray:
    """Read the convolution outputs [Cout][Ho][Wo] from decrypted output
    polynomials [n_out][N] (output ct i*bands + band)."""
    y = np.zeros((geo.Cout, geo.Ho, geo.Wo), np.int64)
    for i in range(geo.Cout):
        for band in range(geo.bands):
            poly = mpoly[i * geo.bands + band]
            for oyl in range(geo.Rout):
                oy = band * geo.Rout + oyl
                if oy >= geo.Ho:
                    break
                base = geo.s * oyl * geo.Wp
                y[i, oy] = poly[base: base + geo.s * geo.Wo: geo.s]
    return y


# ---------------------------------------------------------------------------
# Ring operations
# ---------------------------------------------------------------------------
def negacyclic_mul(a, b, q: int) -> np.ndarray:
    a, b = _u32(a), _u32(b)
    out = np.zeros_like(a)
    lib().or_negacyclic_mul(_p(a, ctypes.c_uint32), _p(b, ctypes.c_uint32),
                            a.shape[0], q, _p(out, ctypes.c_uint32))
    return out


def drot(c, step: int, q: int) -> np.ndarray:
    c = _u32(c)
    out = np.zeros_like(c)
    lib().or_drot(_p(c, ctypes.c_uint32), c.shape[0], q, step, _p(out, ctypes.c_uint32))
    return out


def weight_poly(w: np.ndarray, i: int, g: int, geo: Geometry, q: int) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.int8)
    out = np.zeros(geo.N, np.uint32)
    lib().or_weight_poly(geo.N, q, geo.Cin, geo.k, geo.Wp, geo.P, geo.c_n,
                         _p(w[i], ctypes.c_int8), g, _p(out, ctypes.c_uint32))
    return out


# ---------------------------------------------------------------------------
# BFV (Table 2, Appendix A)
# ---------------------------------------------------------------------------
def encrypt(s, a, e, m, primes, t=T_DEFAULT) -> np.ndarray:
    """Private-key encryption of plaintexts m[n][N] with randomness a[n][L][N]
    (uniform residues) and e[n][N]; secret s[N] ternary.  Returns [n][2][L][N]."""
    N, L = m.shape[-1], len(primes)
    q = _u32(primes)
    d = _u32(delta_residues(primes, t))
    s = np.ascontiguousarray(s, np.int8)
    n = m.shape[0]
    out = np.zeros((n, 2, L, N), np.uint32)
    for c in range(n):
        a_c = _u32(a[c])
        e_c = np.ascontiguousarray(e[c], np.int32)
        m_c = _u32(m[c])
        c0 = np.zeros((L, N), np.uint32)
        c1 = np.zeros((L, N), np.uint32)
        lib().or_encrypt(N, L, _p(q, ctypes.c_uint32), _p(d, ctypes.c_uint32),
                         _p(s, ctypes.c_int8), _p(a_c, ctypes.c_uint32),
                         _p(e_c, ctypes.c_int32), _p(m_c, ctypes.c_uint32),
                         _p(c0, ctypes.c_uint32), _p(c1, ctypes.c_uint32))
        out[c, 0], out[c, 1] = c0, c1
    return out


def phase(s, ct: np.ndarray, primes) -> np.ndarray:
    """[c1*s + c0] per limb for cts [n][2][L][N] -> [n][L][N]."""
    n, _, L, N = ct.shape
    q = _u32(primes)
    s = np.ascontiguousarray(s, np.int8)
    out = np.zeros((n, L, N), np.uint32)
    for c in range(n):
        c0, c1 = _u32(ct[c, 0]), _u32(ct[c, 1])
        o = np.zeros((L, N), np.uint32)
        lib().or_phase(N, L, _p(q, ctypes.c_uint32), _p(s, ctypes.c_int8),
                       _p(c0, ctypes.c_uint32), _p(c1, ctypes.c_uint32),
                       _p(o, ctypes.c_uint32))
        out[c] = o
    return out


def crt(res: np.ndarray, primes) -> np.ndarray:
    """Exact CRT of residues [..][L][N] -> Python-int object array [..][N] in [0, q)."""
    q = math.prod(primes)
    acc = np.zeros(res.shape[:-2] + res.shape[-1:], dtype=object)
    for l, ql in enumerate(primes):
        Ql = q // ql
        coef = Ql * pow(Ql, -1, ql)
        acc = acc + res[..., l, :].astype(np.int64).astype(object) * coef
    return acc % q


def decrypt(s, ct, primes, t=T_DEFAULT) -> np.ndarray:
    """m = round(t * [c0 + c1*s]_q / q) mod t, exact (big integers)."""
    q = math.prod(primes)
    x = crt(phase(s, ct, primes), primes)
    m = (2 * t * x + q) // (2 * q)
    return (m % t).astype(np.int64)


def noise_inf(s, ct, m_expected, primes, t=T_DEFAULT) -> int:
    """||v||_inf with v = [c0 + c1*s]_q - Delta*m, centred in (-q/2, q/2]."""
    q = math.prod(primes)
    delta = q // t
    x = crt(phase(s, ct, primes), primes)
    v = (x - np.asarray(m_expected).astype(np.int64).astype(object) * delta) % q
    v = np.where(v > q // 2, v - q, v)
    return int(max(abs(int(z)) for z in v.ravel()))


def mod_switch(ct, primes, L_out) -> np.ndarray:
    """BFV modulus switching (Fan and Vercauteren's scale-and-round by q'/q),
    dropping the last RNS primes one at a time: each step replaces the CRT
    value x in [0, q) of every coefficient of both components by the nearest
    integer to x / q_last (never a tie: q_last is odd), reduced mod q' = q /
    q_last.  The result decrypts under the first L_out primes.  The paper
    keeps one modulus and does not switch; this reduces the volume of output
    ciphertexts.  ct [..][2][L][N] -> [..][2][L_out][N]."""
    cur = list(primes)
    res = _u32(ct)
    while len(cur) > L_out:
        ql, nxt = cur[-1], cur[:-1]
        x = crt(res, cur)
        xr = ((2 * x + ql) // (2 * ql)) % math.prod(nxt)
        out = np.empty(res.shape[:-2] + (len(nxt), res.shape[-1]), np.uint32)
        for i, qi in enumerate(nxt):
            out[..., i, :] = (xr % qi).astype(np.int64)
        res, cur = out, nxt
    return res


def mask(ct: np.ndarray, r: np.ndarray, primes, t=T_DEFAULT) -> np.ndarray:
    """c0 <- c0 + Delta*r for cts [n][2][L][N], r[n][N] in [0, t)."""
    ct = _u32(ct).copy()
    n, _, L, N = ct.shape
    q = _u32(primes)
    d = _u32(delta_residues(primes, t))
    for c in range(n):
        c0 = np.ascontiguousarray(ct[c, 0])
        rr = _u32(r[c])
        lib().or_mask(N, L, _p(q, ctypes.c_uint32), _p(d, ctypes.c_uint32),
                      _p(rr, ctypes.c_uint32), _p(c0, ctypes.c_uint32))
        ct[c, 0] = c0
    return ct


# ---------------------------------------------------------------------------
# Convolution routes
# ---------------------------------------------------------------------------
def _conv(fn, ct_in, w, geo: Geometry, primes, i_lo, i_hi):
    ct_in = _u32(ct_in)
    assert ct_in.shape == (geo.n_in, 2, len(primes), geo.N), ct_in.shape
    w = np.ascontiguousarray(w, np.int8)
    q = _u32(primes)
    out = np.zeros(((i_hi - i_lo) * geo.bands, 2, len(primes), geo.N), np.uint32)
    fn(geo.N, len(primes), _p(q, ctypes.c_uint32), geo.Cin, geo.k, geo.Wp, geo.P,
       geo.c_n, geo.G, geo.bands, _p(w, ctypes.c_int8), _p(ct_in, ctypes.c_uint32),
       i_lo, i_hi, _p(out, ctypes.c_uint32))
    return out


def conv_alg1(ct_in, w, geo, primes, i_lo=0, i_hi=None):
    """Route O2: Algorithm 1 with lazy reduction, one image; output cts of
    channels [i_lo, i_hi) -> [(i_hi-i_lo)*bands][2][L][N]."""
    return _conv(lib().or_conv_alg1, ct_in, w, geo, primes, i_lo,
                 geo.Cout if i_hi is None else i_hi)


def conv_poly(ct_in, w, geo, primes, i_lo=0, i_hi=None):
    """Route O1: sum_g W_{i,g} * ct_g by schoolbook negacyclic products."""
    return _conv(lib().or_conv_poly, ct_in, w, geo, primes, i_lo,
                 geo.Cout if i_hi is None else i_hi)


def conv2d_int(x: np.ndarray, w: np.ndarray, s: int, p: int) -> np.ndarray:
    """Plain integer cross-correlation (the CNN convolution Algorithm 1
    evaluates): y[i][oy][ox] = sum_{j,ky,kx} w[i][j][ky][kx] *
    xpad[j][s*oy+ky][s*ox+kx], exact in int64."""
    Cin, H, W = x.shape
    Cout, _, k, _ = w.shape
    xp = np.zeros((Cin, H + 2 * p, W + 2 * p), np.int64)
    xp[:, p:p + H, p:p + W] = x
    Ho = (H + 2 * p - k) // s + 1
    Wo = (W + 2 * p - k) // s + 1
    y = np.zeros((Cout, Ho, Wo), np.int64)
    w64 = w.astype(np.int64)
    for ky in range(k):
        for kx in range(k):
            patch = xp[:, ky: ky + s * (Ho - 1) + 1: s, kx: kx + s * (Wo - 1) + 1: s]
            y += np.einsum("ij,jhw->ihw", w64[:, :, ky, kx], patch)
    return y


def noise_bound(w: np.ndarray, primes, t=T_DEFAULT, x_max=255, e_max=21,
                masked=False) -> int:
    """Analytic bound on ||v||_inf of an output ciphertext of the conv.

    Input cts satisfy c0 + c1*s = Delta*m - e (Table 2).  With Delta*t = q - r_t
    (r_t = q mod t), M_i = sum_g W_{i,g} m_g over Z[x]/(x^N+1) and
    K_i = floor(M_i / t), the output decrypts as Delta*[M_i]_t + v_i with
    v_i = -r_t*K_i - sum_g W_{i,g} e_g, so ||v_i|| <= r_t*ceil(x_max*S_i/t)
    + e_max*S_i where S_i = sum |w_i|.  The mask adds at most r_t more
    (the carry of [M]_t + r).
    """
    q = math.prod(primes)
    r_t = q % t
    S = int(np.abs(w.astype(np.int64)).reshape(w.shape[0], -1).sum(1).max())
    b = r_t * (-(-x_max * S // t) + 1) + e_max * S
    return b + (r_t if masked else 0)


# ---------------------------------------------------------------------------
# Batch encoding and the server side of the x^2 + x protocol (Sec. 5.2)
# ---------------------------------------------------------------------------
def plain_root(N: int, t: int = T_DEFAULT) -> int:
    """Reading: psi_t is the first g^((t-1)/2N), g = 2, 3, ..., with
    psi_t^N = -1 mod t (a primitive 2N-th root of unity; t = 1 mod 2N)."""
    assert (t - 1) % (2 * N) == 0
    for g in range(2, t):
        psi = pow(g, (t - 1) // (2 * N), t)
        if pow(psi, N, t) == t - 1:
            return psi
    raise ValueError("no root")


def batch_encode(slots, N, t=T_DEFAULT) -> np.ndarray:
    s = _u32(np.asarray(slots) % t)
    out = np.zeros(N, np.uint32)
    lib().or_batch_encode(N, t, plain_root(N, t), _p(s, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def batch_decode(m, N, t=T_DEFAULT) -> np.ndarray:
    m = _u32(np.asarray(m) % t)
    out = np.zeros(N, np.uint32)
    lib().or_batch_decode(N, t, plain_root(N, t), _p(m, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def lift_centered(m, q: int, t: int = T_DEFAULT) -> np.ndarray:
    """Plaintext coefficients in [0, t) as integers in (-t/2, t/2], mod q."""
    m = np.asarray(m).astype(np.int64)
    c = np.where(m > t // 2, m - t, m)
    return (c % q).astype(np.uint32)


def pmult(ct, m, primes, t=T_DEFAULT) -> np.ndarray:
    """PMult (Sec. 2.2): both components times the plaintext polynomial m
    (coefficients lifted to (-t/2, t/2]) in R_q.  ct [n][2][L][N], m [n][N]."""
    ct = _u32(ct)
    out = np.zeros_like(ct)
    for c in range(ct.shape[0]):
        for l, ql in enumerate(primes):
            mm = lift_centered(m[c], ql, t)
            for j in range(2):
                out[c, j, l] = negacyclic_mul(mm, ct[c, j, l], ql)
    return out


def add_plain(ct, m, primes, t=T_DEFAULT) -> np.ndarray:
    """HAdd with a plaintext: c0 <- c0 + Delta*m (m in [0, t))."""
    return mask(ct, np.asarray(m, dtype=np.uint32), primes, t)


def sub_ct(a, b, primes) -> np.ndarray:
    """HAdd of a and the negation of b, limb by limb."""
    a, b = _u32(a), _u32(b)
    out = np.empty_like(a)
    for l, ql in enumerate(primes):
        out[..., l, :] = ((a[..., l, :].astype(np.int64) - b[..., l, :]) % ql).astype(np.uint32)
    return out


def x2x_server_round1(ct_batch, r, v, primes, t=T_DEFAULT) -> np.ndarray:
    """Server step of Sec. 5.2 on <a+r> (batch encoded): PMult by the batch
    encoding of 2r, then add v (batch encoded): <2ar + 2r^2 + v>.
    ct_batch [n][2][L][N]; r, v [n][N] slot vectors mod t."""
    N = ct_batch.shape[-1]
    pm = np.stack([batch_encode((2 * np.asarray(r[c], np.int64)) % t, N, t) for c in range(ct_batch.shape[0])])
    pv = np.stack([batch_encode(v[c], N, t) for c in range(ct_batch.shape[0])])
    return add_plain(pmult(ct_batch, pm, primes, t), pv, primes, t)


def x2x_server_round2(ct_x, ct_y, r, v, primes, t=T_DEFAULT) -> np.ndarray:
    """Final server step of Sec. 5.2: with <X> = <a^2 + 2ar + r^2 + a + r> and
    <Y> = <2ar + 2r^2 + v> (both direct encoded), <a^2 + a> = <X> - <Y> +
    (r^2 - r + v) (direct encoded plaintext)."""
    r = np.asarray(r, np.int64)
    c = (r * r - r + np.asarray(v, np.int64)) % t
    return add_plain(sub_ct(ct_x, ct_y, primes), c, primes, t)


def num_threads() -> int:
    return int(lib().or_num_threads())
