"""Parity of batch encoding and of the server steps of the x^2 + x protocol
(Sec. 5.2) with the oracle, through the C-ABI, and the protocol end to end
between two encrypted convolutions.  Comparisons of ciphertexts and
plaintexts are bit-exact."""
import numpy as np
import pytest

from paper_2401_16732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
T = 65537


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def dev(a, dtype=torch.int32):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda()
    return torch.from_numpy(a).to(dtype).cuda()


@pytest.fixture(scope="module")
def fg():
    from paper_2401_16732_gb300 import flashgpu
    return flashgpu


_ctx = {}


def ctx(fg, N, L):
    if (N, L) not in _ctx:
        _ctx[(N, L)] = fg.Context(N, L)
    return _ctx[(N, L)]


def encrypt_polys(c, sk, m, seed):
    """GPU private-key encryption of plaintext polynomials m [n][N] (values in
    [0, t)): a 1 x N 'image' with a 1x1 kernel packs coefficient u = m[u]."""
    n, N, L = m.shape[0], c.N, c.L
    g = c.geom(1, 1, 1, N, 1)
    a = synth.uniform_residues(seed, c.primes, (n, 1, L, N))
    e = synth.cbd_noise(seed, (n, 1, N))
    ct = c.encrypt(sk, g, dev(m.reshape(n, 1, 1, N).astype(np.int32)), dev(a), dev(e))
    return ct.view(n, 2, L, N)


# ------------------------------------------------------------------ batch encoding
@pytest.mark.parametrize("N,L,n", [(2048, 1, 3), (4096, 2, 2), (8192, 3, 2), (16384, 1, 1)])
def test_batch_encode_decode_match_oracle(fg, oracle, N, L, n):
    c = ctx(fg, N, L)
    s = synth.masks(5, (n, N), T)
    m = u32(c.batch_encode(dev(s)))
    for i in range(n):
        assert (m[i] == oracle.batch_encode(s[i], N)).all()
    assert (u32(c.batch_decode(dev(m))) == s).all()
    p = synth.masks(6, (n, N), T)
    d = u32(c.batch_decode(dev(p)))
    for i in range(n):
        assert (d[i] == oracle.batch_decode(p[i], N)).all()
    # slot values are reduced mod t first
    assert (u32(c.batch_encode(dev(s + T))) == m).all()


def test_batch_encoding_needs_t_one_mod_2n(fg):
    c = fg.Context(2048, 1, 257)  # 257 - 1 is not a multiple of 4096
    x = torch.zeros(2048, dtype=torch.int32, device="cuda")
    with pytest.raises(fg.FlashError, match="t = 1 mod 2N"):
        c.batch_encode(x)


# ------------------------------------------------------------------ server steps
@pytest.mark.parametrize("N,L", [(4096, 2), (8192, 3)])
def test_x2x_prepare_rows(fg, oracle, N, L):
    c = ctx(fg, N, L)
    n = 2
    r, v = synth.masks(7, (n, N), T, 1), synth.masks(7, (n, N), T, 2)
    prep = c.x2x_prepare(dev(r), dev(v))
    got = u32(prep).copy()
    lifted = dev(got[:, :L].copy())
    c.ntt_inverse(lifted)
    lifted = u32(lifted)
    for i in range(n):
        e2r = oracle.batch_encode((2 * r[i].astype(np.int64)) % T, N)
        for l, q in enumerate(c.primes):
            # rows [0, L) carry N^-1 (round 1's inverse NTT leaves it out)
            back = lifted[i, l].astype(np.int64) * N % q
            assert (back == oracle.lift_centered(e2r, q)).all()
        assert (got[i, L] == oracle.batch_encode(v[i], N)).all()
        rr = r[i].astype(np.int64)
        assert (got[i, L + 1] == (rr * rr - rr + v[i]) % T).all()


@pytest.mark.parametrize("N,L,n", [(2048, 1, 3), (4096, 2, 3), (8192, 3, 2), (16384, 2, 1)])
def test_x2x_round1_matches_oracle(fg, oracle, N, L, n):
    """PMult by the batch encoding of 2r plus encode(v) on uniform residues
    (the step is linear in the ciphertext, so any residues exercise it)."""
    c = ctx(fg, N, L)
    ct = synth.raw_ciphertexts(8, c.primes, (n, 2, L, N))
    r, v = synth.masks(8, (n, N), T, 1), synth.masks(8, (n, N), T, 2)
    prep = c.x2x_prepare(dev(r), dev(v))
    want = oracle.x2x_server_round1(ct, r, v, c.primes)
    assert (u32(c.x2x_round1(prep, dev(ct))) == want).all()
    d = dev(ct)
    c.x2x_round1(prep, d, out=d)  # in place
    assert (u32(d) == want).all()


@pytest.mark.parametrize("N,L,n", [(2048, 1, 5), (8192, 3, 3), (16384, 4, 1)])
def test_x2x_round2_matches_oracle(fg, oracle, N, L, n):
    c = ctx(fg, N, L)
    X = synth.raw_ciphertexts(9, c.primes, (n, 2, L, N), 1)
    Y = synth.raw_ciphertexts(9, c.primes, (n, 2, L, N), 2)
    r, v = synth.masks(9, (n, N), T, 1), synth.masks(9, (n, N), T, 2)
    r[0, :4] = [0, 1, T - 1, 2]  # r^2 at the ends of [0, t)
    prep = c.x2x_prepare(dev(r), dev(v))
    want = oracle.x2x_server_round2(X, Y, r, v, c.primes)
    assert (u32(c.x2x_round2(prep, dev(X), dev(Y))) == want).all()
    dx = dev(X)
    c.x2x_round2(prep, dx, dev(Y), out=dx)  # in place on X
    assert (u32(dx) == want).all()


def test_x2x_empty_batch(fg):
    c = ctx(fg, 2048, 1)
    z = torch.empty((0, 2048), dtype=torch.int32, device="cuda")
    prep = c.x2x_prepare(z, z)
    assert prep.shape == (0, 3, 2048)
    assert c.x2x_round1(prep, torch.empty((0, 2, 1, 2048), dtype=torch.int32, device="cuda")).shape[0] == 0


# ------------------------------------------------------------------ repacking
REPACK = [
    # (N, prev layer, next layer) as (Cin, Cout, H, W, k, s, p)
    (2048, (3, 4, 16, 16, 3, 1, 1), (4, 5, 16, 16, 3, 2, 1)),     # packed channels, next stride 2
    (2048, (2, 2, 60, 60, 3, 1, 1), (2, 3, 60, 60, 3, 2, 1)),     # row bands on both sides
    (2048, (3, 4, 33, 33, 3, 2, 1), (4, 4, 17, 17, 3, 1, 1)),     # prev stride 2, ragged
    (8192, (64, 64, 8, 8, 3, 1, 1), (64, 128, 8, 8, 3, 2, 1)),    # ResNet-18 stage-4 shape
]


@pytest.mark.parametrize("N,prev,nxt", REPACK)
def test_repack_matches_oracle(fg, oracle, N, prev, nxt):
    gp, gn = fg.fl_conv_geom_make(N, *prev), fg.fl_conv_geom_make(N, *nxt)
    B = 2
    src = synth.masks(10, (B, gp.n_out, N), T)
    got = u32(fg.repack_outputs(gp, gn, dev(src)))
    op, on = oracle.geometry(N, *prev), oracle.geometry(N, *nxt)
    for b in range(B):
        assert (got[b] == oracle.pack_inputs(oracle.extract_outputs(src[b].astype(np.int64), op), on)).all()


def test_repack_rejects_mismatched_layers(fg):
    gp = fg.fl_conv_geom_make(2048, 3, 4, 16, 16, 3, 1, 1)
    gn = fg.fl_conv_geom_make(2048, 5, 4, 16, 16, 3, 1, 1)
    src = torch.zeros((1, gp.n_out, 2048), dtype=torch.int32, device="cuda")
    with pytest.raises(fg.FlashError, match="do not match"):
        fg.repack_outputs(gp, gn, src)


# ------------------------------------------------------------------ the protocol end to end
def test_x2x_protocol_between_two_convolutions(fg, oracle):
    """conv -> mask r -> client computes x^2 + x on a + r -> server rounds 1
    and 2 -> next conv: the result decrypts to conv2(f(conv1(x))) mod t with
    f(a) = a^2 + a, and each server step matches the oracle bit for bit."""
    N, L, B = 8192, 3, 2
    c = ctx(fg, N, L)
    g1 = c.geom(3, 4, 16, 16, 3, 1, 1)
    g2 = c.geom(4, 5, 16, 16, 3, 2, 1)
    s = synth.secret_key(41, N)
    sk = c.keygen(dev(s, torch.int8))
    x = synth.activations(41, (B, 3, 16, 16))
    w1, w2 = synth.weights(41, (4, 3, 3, 3), 1), synth.weights(41, (5, 4, 3, 3), 2)
    a1 = synth.uniform_residues(41, c.primes, (B, g1.n_in, L, N))
    e1 = synth.cbd_noise(41, (B, g1.n_in, N))
    ct1 = c.encrypt(sk, g1, dev(x), dev(a1), dev(e1))
    r1 = synth.masks(41, (B, g1.n_out, N), T)
    y1 = c.he_conv2d(g1, c.encode_weights(g1, dev(w1, torch.int8)), ct1, r=dev(r1))

    # client: a + r in the next layer's input layout, X = z^2 + z, <X>, <z>_batch
    z = fg.repack_outputs(g1, g2, c.decrypt(sk, y1))
    zn = u32(z).astype(np.int64)
    n = B * g2.n_in
    X = ((zn * zn + zn) % T).reshape(n, N)
    ct_x = encrypt_polys(c, sk, X, 42)
    ct_z = encrypt_polys(c, sk, u32(c.batch_encode(z.view(n, N))).astype(np.int64), 43)

    # server round 1 on its mask in the same layout and a fresh mask v
    r2 = fg.repack_outputs(g1, g2, dev(r1)).view(n, N)
    v = synth.masks(44, (n, N), T)
    prep = c.x2x_prepare(r2, dev(v))
    ct_y_b = c.x2x_round1(prep, ct_z)
    assert (u32(ct_y_b) == oracle.x2x_server_round1(u32(ct_z), u32(r2), v, c.primes)).all()

    # client: Y = 2rz + v, re-encrypted under direct encoding
    Y = u32(c.batch_decode(c.decrypt(sk, ct_y_b))).astype(np.int64)
    rn = u32(r2).astype(np.int64)
    assert (Y == (2 * rn * zn.reshape(n, N) + v) % T).all()
    ct_yd = encrypt_polys(c, sk, Y, 45)

    # server round 2 -> the next convolution's input
    act = c.x2x_round2(prep, ct_x, ct_yd)
    assert (u32(act) == oracle.x2x_server_round2(u32(ct_x), u32(ct_yd), u32(r2), v, c.primes)).all()
    y2 = c.he_conv2d(g2, c.encode_weights(g2, dev(w2, torch.int8)), act.view(B, g2.n_in, 2, L, N))
    got = u32(c.extract_outputs(g2, c.decrypt(sk, y2))).astype(np.int64)
    for b in range(B):
        a = oracle.conv2d_int(x[b], w1, 1, 1) % T
        f = (a * a + a) % T
        assert (got[b] == oracle.conv2d_int(f, w2, 2, 1) % T).all()
