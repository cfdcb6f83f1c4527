"""Pins for the CPU oracle: every oracle function is checked against something
other than itself -- brute force on tiny rings, textbook identities, a library
routine, or a fact the paper states.  No GPU needed."""
import json
import math
import os

import numpy as np
import pytest

from paper_2401_16732_gb300 import synth

T = 65537
HERE = os.path.dirname(os.path.abspath(__file__))


def textbook_negacyclic(a, b, q):
    """Pure-Python schoolbook product in Z[x], then reduction by x^N = -1."""
    N = len(a)
    full = [0] * (2 * N - 1)
    for i in range(N):
        for j in range(N):
            full[i + j] += int(a[i]) * int(b[j])
    return [(full[k] - (full[k + N] if k + N < 2 * N - 1 else 0)) % q for k in range(N)]


def primitive_2n_root(q, N):
    """Brute force: smallest psi with psi^N = -1 mod q (order exactly 2N)."""
    for g in range(2, q):
        psi = pow(g, (q - 1) // (2 * N), q)
        if pow(psi, N, q) == q - 1:
            return psi
    raise AssertionError


# ----------------------------------------------------------------- primes
@pytest.mark.parametrize("N,L", [(4096, 2), (8192, 3), (16384, 4), (64, 3)])
def test_primes_are_the_largest_ntt_friendly_primes(oracle, N, L):
    sympy = pytest.importorskip("sympy")
    qs = oracle.find_primes(N, L)
    assert qs == sorted(qs, reverse=True)
    for q in qs:
        assert q < 2 ** 30 and q % (2 * N) == 1 and sympy.isprime(q)
    # no prime 1 mod 2N was skipped between 2^30 and the smallest one chosen
    c = (2 ** 30 - 1) // (2 * N) * (2 * N) + 1
    while c > qs[-1]:
        assert sympy.isprime(c) == (c in qs)
        c -= 2 * N


def test_is_prime_matches_sympy(oracle):
    sympy = pytest.importorskip("sympy")
    for n in list(range(0, 2000)) + [2 ** 30 - 35, 2 ** 30 - 1, 1073692673, 1073692671]:
        assert bool(oracle.lib().or_is_prime(n)) == bool(sympy.isprime(n)), n


# ----------------------------------------------------------------- ring
@pytest.mark.parametrize("N,q", [(8, 97), (16, 97), (32, 193), (64, 1073692673)])
def test_negacyclic_mul_matches_textbook(oracle, N, q):
    g = np.random.default_rng(N)
    for _ in range(3):
        a = g.integers(0, q, N)
        b = g.integers(0, q, N)
        a[g.integers(0, N, N // 3)] = 0  # exercise the zero skip
        assert list(oracle.negacyclic_mul(a, b, q)) == textbook_negacyclic(a, b, q)


@pytest.mark.parametrize("N,q", [(16, 97), (64, 1073692673)])
def test_negacyclic_mul_is_pointwise_at_odd_powers_of_psi(oracle, N, q):
    """a*b mod x^N+1 is characterised by its values at the N roots of
    x^N + 1, the odd powers of a primitive 2N-th root psi."""
    psi = primitive_2n_root(q, N)
    g = np.random.default_rng(1)
    a, b = g.integers(0, q, N), g.integers(0, q, N)
    c = oracle.negacyclic_mul(a, b, q)

    def ev(p, z):
        return sum(int(p[j]) * pow(z, j, q) for j in range(N)) % q

    for k in range(N):
        z = pow(psi, 2 * k + 1, q)
        assert ev(c, z) == ev(a, z) * ev(b, z) % q


def test_monomials_wrap_with_minus_sign(oracle):
    N, q = 16, 97
    for i in range(N):
        for j in range(N):
            a = np.zeros(N, np.int64); a[i] = 1
            b = np.zeros(N, np.int64); b[j] = 1
            c = oracle.negacyclic_mul(a, b, q)
            want = np.zeros(N, np.int64)
            want[(i + j) % N] = 1 if i + j < N else q - 1
            assert list(c) == list(want)


# ----------------------------------------------------------------- DRot
def test_drot_golden_examples(oracle):
    with open(os.path.join(HERE, "golden", "drot_example.json")) as f:
        fx = json.load(f)
    q = 97
    for case in fx["cases"]:
        got = oracle.drot(np.array(case["m"]) % q, case["step"], q)
        assert list(got) == [v % q for v in case["shifted"]]


def test_drot_is_multiplication_by_x_minus_step(oracle):
    """Eq. 2: DRot(c, step) = c * x^{-step}, and x^{-step} = -x^{N-step}."""
    N, q = 32, 193
    c = np.random.default_rng(2).integers(0, q, N)
    for step in range(N):
        mono = np.zeros(N, np.int64)
        if step == 0:
            mono[0] = 1
        else:
            mono[N - step] = q - 1
        assert list(oracle.drot(c, step, q)) == list(oracle.negacyclic_mul(mono, c, q))


def test_drot_beyond_one_wrap(oracle):
    """Eq. 2 for steps of N and more: x^N = -1, so x^{-step} is the monomial
    x^e with e = -step mod 2N, read as -x^{e-N} when e >= N.  Steps compose:
    DRot(DRot(c, a), b) = DRot(c, a + b), and a step of 2N is the identity.
    Every coefficient is written (no step leaves the output untouched)."""
    N, q = 16, 97
    c = np.random.default_rng(3).integers(1, q, N)
    for step in (N - 1, N, N + 3, 2 * N - 1, 2 * N, 2 * N + 5, 3 * N + 1):
        e = (-step) % (2 * N)
        mono = np.zeros(N, np.int64)
        if e < N:
            mono[e] = 1
        else:
            mono[e - N] = q - 1
        got = oracle.drot(c, step, q)
        assert list(got) == list(oracle.negacyclic_mul(mono, c, q)), step
        assert (got != 0).all()  # c has no zero coefficient, so neither has its shift
    for a_step, b_step in ((3, N - 1), (N, N), (N + 2, 2 * N - 3)):
        two = oracle.drot(oracle.drot(c, a_step, q), b_step, q)
        assert list(two) == list(oracle.drot(c, a_step + b_step, q))
    assert list(oracle.drot(c, 2 * N, q)) == list(c)


def test_drot_theorem_on_ciphertexts(oracle):
    """Appendix A: decrypting DRot(ct, step) gives the signed shift of m and
    the noise norm is unchanged."""
    N = 64
    primes = oracle.find_primes(N, 2)
    s = synth.secret_key(5, N)
    m = synth.activations(5, (1, N)).astype(np.uint32)
    a = synth.uniform_residues(5, primes, (1, 2, N))
    e = synth.cbd_noise(5, (1, N))
    ct = oracle.encrypt(s, a, e, m, primes)
    n0 = oracle.noise_inf(s, ct, m, primes)
    for step in (0, 1, 5, 63):
        rot = np.stack([np.stack([oracle.drot(ct[0, c, l], step, primes[l])
                                  for l in range(2)]) for c in range(2)])[None]
        want = np.array([(-1) ** ((i + step) // N) * int(m[0, (i + step) % N]) for i in range(N)])
        assert list(oracle.decrypt(s, rot, primes)[0]) == list(want % T)
        # the plaintext is the integer polynomial m(x)*x^{-step} (signed coefficients)
        assert oracle.noise_inf(s, rot, want[None], primes) == n0


# ----------------------------------------------------------------- BFV
@pytest.mark.parametrize("N,L", [(64, 2), (128, 3), (256, 4)])
def test_encrypt_decrypt_and_exact_fresh_noise(oracle, N, L):
    primes = oracle.find_primes(N, L)
    s = synth.secret_key(9, N)
    m = synth.masks(9, (2, N), T)
    a = synth.uniform_residues(9, primes, (2, L, N))
    e = synth.cbd_noise(9, (2, N))
    ct = oracle.encrypt(s, a, e, m, primes)
    assert (ct[:, 1] == a).all()  # c1 = a (Table 2)
    assert (oracle.decrypt(s, ct, primes) == m).all()
    # c0 + c1*s = Delta*m - e exactly, so the noise is -e
    q = math.prod(primes)
    delta = q // T
    x = oracle.crt(oracle.phase(s, ct, primes), primes)
    v = (x - m.astype(np.int64).astype(object) * delta) % q
    v = np.where(v > q // 2, v - q, v)
    assert (v.astype(np.int64) == -e).all()


def test_online_encryption_algorithm2(oracle):
    """Algorithm 2: Enc(m) = Enc(0) + Delta*m for the same (a, e)."""
    N, L = 128, 3
    primes = oracle.find_primes(N, L)
    s = synth.secret_key(3, N)
    m = synth.masks(3, (1, N), T)
    a = synth.uniform_residues(3, primes, (1, L, N))
    e = synth.cbd_noise(3, (1, N))
    ct = oracle.encrypt(s, a, e, m, primes)
    ct0 = oracle.encrypt(s, a, e, np.zeros_like(m), primes)
    delta = math.prod(primes) // T
    for l, ql in enumerate(primes):
        want = (ct0[0, 0, l].astype(object) + (delta % ql) * m[0].astype(object)) % ql
        assert (ct[0, 0, l].astype(object) == want).all()
    assert (ct[0, 1] == ct0[0, 1]).all()


def test_decrypt_rounds_to_nearest(oracle):
    """Decryption of a hand-made phase Delta*m + v: since t*Delta = q - r_t,
    t*(Delta*m + v)/q = m + (t*v - r_t*m)/q, so m comes back exactly while
    |t*v - r_t*m| < q/2, and the neighbour just outside either edge."""
    N, L = 16, 2
    primes = oracle.find_primes(N, L)
    q = math.prod(primes)
    delta, r_t = q // T, q % T
    s = np.zeros(N, np.int8)  # phase = c0
    m = 1234
    v_hi = (q // 2 + r_t * m) // T
    v_lo = -((q // 2 - r_t * m) // T)
    for v, shift in ((v_hi, 0), (v_hi + 1, 1), (v_lo, 0), (v_lo - 1, -1), (0, 0)):
        x = (delta * m + v) % q
        c0 = np.array([[x % ql] * N for ql in primes], np.uint32)
        ct = np.stack([c0, np.zeros_like(c0)])[None]
        assert (oracle.decrypt(s, ct, primes) == (m + shift) % T).all(), (v, shift)


# ----------------------------------------------------------------- conv
def brute_conv2d(x, w, s, p):
    Cin, H, W = x.shape
    Cout, _, k, _ = w.shape
    Ho = (H + 2 * p - k) // s + 1
    Wo = (W + 2 * p - k) // s + 1
    y = [[[0] * Wo for _ in range(Ho)] for _ in range(Cout)]
    for i in range(Cout):
        for oy in range(Ho):
            for ox in range(Wo):
                acc = 0
                for j in range(Cin):
                    for ky in range(k):
                        for kx in range(k):
                            yy, xx = s * oy + ky - p, s * ox + kx - p
                            if 0 <= yy < H and 0 <= xx < W:
                                acc += int(w[i, j, ky, kx]) * int(x[j, yy, xx])
                y[i][oy][ox] = acc
    return np.array(y)


def test_conv2d_int_matches_brute_force_and_torch(oracle):
    torch = pytest.importorskip("torch")
    for (Cin, Cout, H, k, s, p) in [(3, 4, 6, 3, 1, 1), (2, 3, 7, 3, 2, 1), (4, 2, 5, 1, 2, 0), (2, 2, 9, 7, 2, 3)]:
        x = synth.activations(1, (Cin, H, H))
        w = synth.weights(1, (Cout, Cin, k, k))
        y = oracle.conv2d_int(x, w, s, p)
        assert (y == brute_conv2d(x, w, s, p)).all()
        yt = torch.nn.functional.conv2d(torch.tensor(x, dtype=torch.float64)[None],
                                        torch.tensor(w, dtype=torch.float64), stride=s, padding=p)[0]
        assert (yt.numpy().astype(np.int64) == y).all()


GEOS = [
    # N, Cin, Cout, H, k, s, p
    (256, 3, 4, 6, 3, 1, 1),     # c_n = 4, one ct
    (256, 7, 3, 6, 3, 1, 1),     # c_n = 4, G = 2, ragged last ct
    (256, 5, 3, 7, 3, 2, 1),     # stride 2
    (256, 9, 2, 8, 1, 2, 0),     # 1x1 stride-2 shortcut
    (64, 2, 3, 10, 3, 1, 1),     # row bands (plane 144 > N = 64)
    (256, 3, 2, 20, 7, 2, 3),    # 7x7/2 stem with bands
    (64, 1, 1, 6, 3, 1, 1),      # single channel
]


def test_pack_inputs_places_padded_pixels(oracle):
    for (N, Cin, Cout, H, k, s, p) in GEOS:
        geo = oracle.geometry(N, Cin, Cout, H, H, k, s, p)
        x = synth.activations(4, (Cin, H, H))
        m = oracle.pack_inputs(x, geo)
        seen = np.zeros_like(m, dtype=bool)
        for band in range(geo.bands):
            for j in range(Cin):
                g, jj = divmod(j, geo.c_n)
                for y in range(geo.Rin):
                    for xx in range(geo.Wp):
                        yy, xo = band * geo.Rout * s + y - p, xx - p
                        v = x[j, yy, xo] if (0 <= yy < H and 0 <= xo < H) else 0
                        pos = jj * geo.P + y * geo.Wp + xx
                        assert m[band * geo.G + g, pos] == v
                        seen[band * geo.G + g, pos] = True
        assert (m[~seen] == 0).all()


def test_geometry_outputs_never_wrap(oracle):
    """With the readings above every valid output of every band is computed
    from coefficients below N (no negacyclic wrap), and the bands tile the
    output rows exactly once."""
    for (N, Cin, Cout, H, k, s, p) in GEOS + [(8192, 512, 512, 4, 3, 1, 1), (16384, 3, 64, 224, 7, 2, 3),
                                               (16384, 256, 64, 56, 1, 1, 0), (4096, 16, 16, 16, 3, 1, 1)]:
        geo = oracle.geometry(N, Cin, Cout, H, H, k, s, p)
        top = (s * (geo.Rout - 1) + k - 1) * geo.Wp + s * (geo.Wo - 1) + k - 1 + (geo.c_n - 1) * geo.P
        assert top < N and geo.c_n * geo.P <= N
        rows = [b * geo.Rout + r for b in range(geo.bands) for r in range(geo.Rout) if b * geo.Rout + r < geo.Ho]
        assert rows == list(range(geo.Ho))


def test_stem_and_cifar_geometries(oracle):
    g = oracle.geometry(16384, 3, 64, 224, 224, 7, 2, 3)
    assert (g.Rin, g.Rout, g.bands, g.c_n, g.n_in, g.n_out) == (71, 33, 4, 1, 12, 256)
    g = oracle.geometry(4096, 16, 16, 16, 16, 3, 1, 1)
    assert (g.P, g.c_n, g.G) == (324, 12, 2)


@pytest.mark.parametrize("geo_args", GEOS)
def test_conv_routes_O1_O2_agree_bit_exact(oracle, geo_args):
    N, Cin, Cout, H, k, s, p = geo_args
    geo = oracle.geometry(N, Cin, Cout, H, H, k, s, p)
    primes = oracle.find_primes(N, 3)
    w = synth.weights(7, (Cout, Cin, k, k))
    ct = synth.raw_ciphertexts(7, primes, (geo.n_in, 2, 3, N))
    y1 = oracle.conv_poly(ct, w, geo, primes)
    y2 = oracle.conv_alg1(ct, w, geo, primes)
    assert (y1 == y2).all()
    # and on a sub-range of output channels
    if Cout > 1:
        assert (oracle.conv_alg1(ct, w, geo, primes, 1, Cout) == y2[geo.bands:]).all()


@pytest.mark.parametrize("geo_args", GEOS)
def test_conv_decrypts_to_integer_conv2d_mod_t(oracle, geo_args):
    """O3: decrypt(conv(Enc(x))) == conv2d(x, w) mod t at every valid output,
    and the measured noise stays below the analytic bound."""
    N, Cin, Cout, H, k, s, p = geo_args
    geo = oracle.geometry(N, Cin, Cout, H, H, k, s, p)
    primes = oracle.find_primes(N, 2)
    sk = synth.secret_key(11, N)
    x = synth.activations(11, (Cin, H, H))
    w = synth.weights(11, (Cout, Cin, k, k))
    m = oracle.pack_inputs(x, geo)
    a = synth.uniform_residues(11, primes, (geo.n_in, 2, N))
    e = synth.cbd_noise(11, (geo.n_in, N))
    ct = oracle.encrypt(sk, a, e, m, primes)
    y = oracle.conv_alg1(ct, w, geo, primes)
    dec = oracle.decrypt(sk, y, primes)
    assert (oracle.extract_outputs(dec, geo) == oracle.conv2d_int(x, w, s, p) % T).all()
    # noise bound: expected plaintext is M_i mod t over all N coefficients
    M = oracle.decrypt(sk, y, primes)
    assert oracle.noise_inf(sk, y, M, primes) <= oracle.noise_bound(w, primes)
    # mask -> shares (Sec. 5.2, Sec. 2.3): client decrypts a + r, server keeps t - r
    r = synth.masks(11, (geo.n_out, N), T)
    ym = oracle.mask(y, r, primes)
    client = oracle.decrypt(sk, ym, primes)
    assert (client == (M + r) % T).all()
    server = (T - r.astype(np.int64)) % T
    assert ((client + server) % T == M).all()
    assert oracle.noise_inf(sk, ym, client, primes) <= oracle.noise_bound(w, primes, masked=True)


def test_planted_mistakes_are_caught(oracle):
    """A wrong tap sign, a transposed filter or a dropped wrap sign in the
    weight polynomial breaks the decrypt == conv2d pin."""
    N, Cin, Cout, H, k, s, p = 256, 3, 2, 6, 3, 1, 1
    geo = oracle.geometry(N, Cin, Cout, H, H, k, s, p)
    primes = oracle.find_primes(N, 2)
    sk = synth.secret_key(12, N)
    x = synth.activations(12, (Cin, H, H))
    w = synth.weights(12, (Cout, Cin, k, k))
    m = oracle.pack_inputs(x, geo)
    ct = oracle.encrypt(sk, synth.uniform_residues(12, primes, (geo.n_in, 2, N)),
                        synth.cbd_noise(12, (geo.n_in, N)), m, primes)
    want = oracle.conv2d_int(x, w, s, p) % T

    def conv_with(Wfun):
        y = np.zeros((Cout, 2, 2, N), np.uint32)
        for i in range(Cout):
            for l, ql in enumerate(primes):
                for c in range(2):
                    acc = np.zeros(N, np.int64)
                    for g in range(geo.G):
                        acc = (acc + oracle.negacyclic_mul(Wfun(i, g, ql), ct[g, c, l], ql)) % ql
                    y[i, c, l] = acc
        return oracle.extract_outputs(oracle.decrypt(sk, y, primes), geo)

    good = lambda i, g, ql: oracle.weight_poly(w, i, g, geo, ql)
    assert (conv_with(good) == want).all()
    flipped = lambda i, g, ql: (ql - oracle.weight_poly(w, i, g, geo, ql).astype(np.int64)) % ql
    assert not (conv_with(flipped) == want).all()
    wt = np.ascontiguousarray(w.transpose(0, 1, 3, 2))
    transposed = lambda i, g, ql: oracle.weight_poly(wt, i, g, geo, ql)
    assert not (conv_with(transposed) == want).all()

    def unsigned(i, g, ql):  # x^{-e} taken as +x^{N-e}: the negacyclic sign dropped
        W = oracle.weight_poly(w, i, g, geo, ql).astype(np.int64)
        W[1:] = (ql - W[1:]) % ql
        return W
    assert not (conv_with(unsigned) == want).all()


# ----------------------------------------------------------------- batch encoding and x^2 + x
@pytest.mark.parametrize("N", [8, 16, 64])
def test_batch_encoding_is_slotwise(oracle, N):
    """decode(encode(s)) = s, and the negacyclic product of two encodings
    decodes to the slot-wise product (the defining property of SIMD slots)."""
    g = np.random.default_rng(N)
    s1, s2 = g.integers(0, T, N), g.integers(0, T, N)
    m1, m2 = oracle.batch_encode(s1, N), oracle.batch_encode(s2, N)
    assert (oracle.batch_decode(m1, N) == s1).all()
    prod = oracle.negacyclic_mul(m1, m2, T)
    assert (oracle.batch_decode(prod, N) == (s1 * s2) % T).all()
    # direct check of decode against the definition on one slot
    psi = oracle.plain_root(N)
    k = 3 % N
    z = pow(psi, 2 * k + 1, T)
    assert int(oracle.batch_decode(m1, N)[k]) == sum(int(m1[j]) * pow(z, j, T) for j in range(N)) % T


def test_x2x_protocol_end_to_end(oracle):
    """Sec. 5.2: starting from <a> (direct), mask with r, let the client square,
    run both server rounds, and the result decrypts to a^2 + a mod t."""
    N, L = 256, 3
    primes = oracle.find_primes(N, L)
    s = synth.secret_key(51, N)
    a = synth.masks(51, (1, N), T)
    r = synth.masks(52, (1, N), T)
    v = synth.masks(53, (1, N), T)
    enc = lambda m, k: oracle.encrypt(s, synth.uniform_residues(60 + k, primes, (1, L, N)),
                                      synth.cbd_noise(60 + k, (1, N)), np.asarray(m, np.uint32), primes)
    ct_a = enc(a, 0)
    z = oracle.decrypt(s, oracle.mask(ct_a, r, primes), primes)          # client: a + r
    assert (z == (a + r) % T).all()
    X = (z * z + z) % T                                                  # client: x^2 + x
    ct_x = enc(X, 1)                                                     # direct encoding
    ct_zb = enc(oracle.batch_encode(z[0], N)[None], 2)                   # batch encoding
    ct_y_b = oracle.x2x_server_round1(ct_zb, r, v, primes)              # server round 1
    Yb = oracle.batch_decode(oracle.decrypt(s, ct_y_b, primes)[0], N)    # client decrypts slots
    assert (Yb == (2 * r[0] * z[0] + v[0]) % T).all()
    ct_y = enc(Yb[None], 3)                                              # re-encrypt, direct
    out = oracle.x2x_server_round2(ct_x, ct_y, r, v, primes)             # server round 2
    assert (oracle.decrypt(s, out, primes) == (a * a + a) % T).all()


# ----------------------------------------------------------------- modulus switching
def test_mod_switch_rounds_to_nearest(oracle):
    """Each dropped prime leaves x' with |q_last * x' - x| <= q_last / 2 on the
    CRT values (the defining property of rounding to the nearest integer),
    checked against big-integer CRT of input and output."""
    N, L = 64, 3
    primes = oracle.find_primes(2048, L)
    ct = synth.raw_ciphertexts(70, primes, (2, 2, L, N))
    out = oracle.mod_switch(ct, primes, L - 1)
    x = oracle.crt(ct, primes)
    xp = oracle.crt(out, primes[:-1])
    ql, qn = primes[-1], math.prod(primes[:-1])
    for a, b in zip(x.ravel(), xp.ravel()):
        d = ql * int(b) - int(a)
        # x' is taken mod q'; undo a wrap at the top of the range
        if d < -(ql // 2):
            d += ql * qn
        assert abs(d) <= ql // 2


@pytest.mark.parametrize("L,L_out", [(3, 2), (4, 2), (4, 3)])
def test_mod_switch_keeps_the_message(oracle, L, L_out):
    """Decrypting under the first L_out primes after switching gives the same
    plaintext, including after a convolution and the mask; the noise is the
    scaled noise plus at most (1 + ||s||_1)/2 of rounding."""
    N, T_ = 256, T
    primes = oracle.find_primes(N, L)
    geo = oracle.geometry(N, 2, 3, 6, 6, 3, 1, 1)
    s = synth.secret_key(71, N)
    x = synth.activations(71, (2, 6, 6))
    w = synth.weights(71, (3, 2, 3, 3))
    m = oracle.pack_inputs(x, geo)
    ct = oracle.encrypt(s, synth.uniform_residues(71, primes, (geo.n_in, L, N)),
                        synth.cbd_noise(71, (geo.n_in, N)), m, primes)
    r = synth.masks(71, (geo.n_out, N), T_)
    y = oracle.mask(oracle.conv_alg1(ct, w, geo, primes), r, primes)
    want = oracle.decrypt(s, y, primes)
    ys = oracle.mod_switch(y, primes, L_out)
    assert ys.shape == (geo.n_out, 2, L_out, N)
    assert (oracle.decrypt(s, ys, primes[:L_out]) == want).all()
    q, qs = math.prod(primes), math.prod(primes[:L_out])
    v = oracle.noise_inf(s, y, want, primes)
    vs = oracle.noise_inf(s, ys, want, primes[:L_out])
    # Delta' m differs from (q'/q) Delta m by less than t; rounding adds (1+||s||_1)/2 per drop
    steps = L - L_out
    assert vs <= v * qs // q + steps * (1 + int(np.abs(s).sum())) // 2 + T_ + steps


def test_pmult_lifts_plaintexts_centred(oracle):
    """PMult by the constant t - 1 is multiplication by -1 (the centred lift
    of t - 1), so it negates the ciphertext exactly; by 1 it is the identity;
    by x it is the negacyclic shift (a DRot by N - 1)."""
    N, L = 64, 3
    primes = oracle.find_primes(2048, L)
    ct = synth.raw_ciphertexts(72, primes, (1, 2, L, N))
    one, minus_one, xpoly = np.zeros((1, N), np.uint32), np.zeros((1, N), np.uint32), np.zeros((1, N), np.uint32)
    one[0, 0], minus_one[0, 0], xpoly[0, 1] = 1, T - 1, 1
    assert (oracle.pmult(ct, one, primes) == ct).all()
    neg = oracle.pmult(ct, minus_one, primes)
    for l, q in enumerate(primes):
        assert (neg[0, :, l] == (q - ct[0, :, l].astype(np.int64)) % q).all()
    shifted = oracle.pmult(ct, xpoly, primes)
    for l, q in enumerate(primes):
        for c in range(2):
            a = ct[0, c, l].astype(np.int64)
            want = np.concatenate([[(q - a[-1]) % q], a[:-1]])
            assert (shifted[0, c, l] == want).all()


def test_plaintext_addition_and_ciphertext_subtraction_are_homomorphic(oracle):
    """decrypt(add_plain(Enc(m1), m2)) = m1 + m2 mod t and
    decrypt(sub_ct(Enc(m1), Enc(m2))) = m1 - m2 mod t (fresh noise stays far
    inside the decryption bound).  Delta = floor(q/t) satisfies
    Delta * t + (q mod t) = q, so every residue Delta_l * t + (q mod t) is 0
    mod q_l."""
    N, L = 256, 2
    primes = oracle.find_primes(N, L)
    s = synth.secret_key(81, N)
    m1, m2 = synth.masks(81, (1, N), T, 1), synth.masks(81, (1, N), T, 2)
    ct1 = oracle.encrypt(s, synth.uniform_residues(81, primes, (1, L, N), 1), synth.cbd_noise(81, (1, N), 1), m1,
                         primes)
    ct2 = oracle.encrypt(s, synth.uniform_residues(81, primes, (1, L, N), 2), synth.cbd_noise(81, (1, N), 2), m2,
                         primes)
    m1, m2 = m1.astype(np.int64), m2.astype(np.int64)
    assert (oracle.decrypt(s, oracle.add_plain(ct1, m2, primes), primes) == (m1 + m2) % T).all()
    assert (oracle.decrypt(s, oracle.sub_ct(ct1, ct2, primes), primes) == (m1 - m2) % T).all()
    q = math.prod(primes)
    for d, ql in zip(oracle.delta_residues(primes, T), primes):
        assert (d * T + q % T) % ql == 0


def test_centred_lift(oracle):
    """lift_centered sends [0, t) to its representatives in (-t/2, t/2],
    written mod q: each is congruent to its input mod t and the ends of the
    range map to 0, t//2, -(t//2) and -1."""
    q = oracle.find_primes(2048, 1)[0]
    m = np.array([0, 1, T // 2, T // 2 + 1, T - 1])
    got = oracle.lift_centered(m, q).astype(np.int64)
    ints = np.where(got > q // 2, got - q, got)
    assert list(ints) == [0, 1, T // 2, -(T // 2), -1]
    r = synth.masks(82, (4096,), T).astype(np.int64)
    li = oracle.lift_centered(r, q).astype(np.int64)
    li = np.where(li > q // 2, li - q, li)
    assert (np.abs(li) <= T // 2).all() and ((li - r) % T == 0).all()
