"""Parity of the two other GPU forms of the convolution with the oracle's
Algorithm 1 (route O2) and with the NTT route: the direct form (DRot + CMult,
no NTT) and on-the-fly weights (weight polynomials rebuilt and transformed
in shared memory, no encoded weights).  All comparisons are bit-exact."""
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


CASES = [
    # N, L, (Cin, Cout, H, W, k, s, p), B
    (4096, 2, (16, 16, 16, 16, 3, 1, 1), 2),     # single-layer workload shape
    (2048, 3, (7, 5, 9, 9, 3, 2, 1), 2),         # stride 2, ragged last ct, Cout not a multiple of 4
    (2048, 2, (9, 6, 12, 12, 1, 2, 0), 1),       # 1x1 stride-2 shortcut
    (2048, 2, (160, 3, 14, 14, 3, 1, 1), 1),     # G = 20
    (2048, 2, (3, 4, 40, 40, 7, 2, 3), 2),       # 7x7/2 stem with row bands
    (8192, 3, (3, 64, 32, 32, 3, 1, 1), 1),      # ResNet-18 stem
    (16384, 4, (5, 3, 30, 30, 3, 1, 1), 1),      # N = 16384, L = 4
]


@pytest.mark.parametrize("N,L,shape,B", CASES)
def test_direct_form_bit_exact(fg, oracle, N, L, shape, B):
    c = ctx(fg, N, L)
    g = c.geom(*shape)
    geo = oracle.geometry(N, *shape)
    w = synth.weights(12, (g.Cout, g.Cin, g.k, g.k))
    ct = synth.raw_ciphertexts(12, c.primes, (B, g.n_in, 2, L, N))
    r = synth.masks(12, (B, g.n_out, N), T)
    dw, dct, dr = dev(w, torch.int8), dev(ct), dev(r)
    y = u32(c.he_conv2d_direct(g, dw, dct))
    ym = u32(c.he_conv2d_direct(g, dw, dct, r=dr))
    ntt = u32(c.he_conv2d(g, c.encode_weights(g, dw), dct, r=dr))
    assert (ym == ntt).all()  # the two GPU routes agree
    assert (u32(dct) == ct).all()
    for b in range(B):
        # sampled output channels against the oracle's Algorithm 1 (all of them when small)
        chans = range(g.Cout) if g.Cout * N <= 64 * 4096 else [0, g.Cout // 2, g.Cout - 1]
        for i in chans:
            want = oracle.conv_alg1(ct[b], w, geo, c.primes, i, i + 1)
            sl = slice(i * g.bands, (i + 1) * g.bands)
            assert (y[b, sl] == want).all()
            assert (ym[b, sl] == oracle.mask(want, r[b, sl], c.primes)).all()


def test_direct_form_extreme_values(fg, oracle):
    """All residues q - 1 with all weights -128 or 127: the largest signed
    accumulations the kernel's offset has to cover."""
    N, L = 2048, 2
    c = ctx(fg, N, L)
    g = c.geom(64, 4, 6, 6, 3, 1, 1)
    geo = oracle.geometry(N, 64, 4, 6, 6, 3, 1, 1)
    ct = np.empty((1, g.n_in, 2, L, N), np.uint32)
    for l, q in enumerate(c.primes):
        ct[:, :, :, l, :] = q - 1
    for wv in (-128, 127):
        w = np.full((g.Cout, g.Cin, g.k, g.k), wv, np.int8)
        got = u32(c.he_conv2d_direct(g, dev(w, torch.int8), dev(ct)))
        assert (got[0] == oracle.conv_alg1(ct[0], w, geo, c.primes)).all()


def test_direct_form_limits(fg):
    c = ctx(fg, 2048, 1)
    g = c.geom(2048, 1, 1, 1, 3, 1, 1)  # 2048 * 9 taps > FL_DIRECT_MAX_TAPS
    w = torch.zeros((1, 2048, 3, 3), dtype=torch.int8, device="cuda")
    ct = torch.zeros((1, g.n_in, 2, 1, 2048), dtype=torch.int32, device="cuda")
    with pytest.raises(fg.FlashError, match="direct form"):
        c.he_conv2d_direct(g, w, ct)
    g2 = c.geom(3, 2, 8, 8, 3, 1, 1)
    empty = torch.empty((0, g2.n_in, 2, 1, 2048), dtype=torch.int32, device="cuda")
    assert c.he_conv2d_direct(g2, torch.zeros((2, 3, 3, 3), dtype=torch.int8, device="cuda"), empty).shape[0] == 0


# ------------------------------------------------------------------ on-the-fly weights
OTF_CASES = CASES + [
    (2048, 3, (8, 101, 6, 6, 3, 1, 1), 2),       # odd Cout, many CTAs, G = 1
    (4096, 2, (40, 7, 8, 8, 1, 1, 0), 1),        # 1x1, 40 taps per polynomial
]


@pytest.mark.parametrize("N,L,shape,B", OTF_CASES)
def test_otf_weights_bit_exact(fg, oracle, N, L, shape, B):
    c = ctx(fg, N, L)
    g = c.geom(*shape)
    geo = oracle.geometry(N, *shape)
    w = synth.weights(13, (g.Cout, g.Cin, g.k, g.k))
    ct = synth.raw_ciphertexts(13, c.primes, (B, g.n_in, 2, L, N))
    r = synth.masks(13, (B, g.n_out, N), T)
    dw, dct, dr = dev(w, torch.int8), dev(ct), dev(r)
    ym = u32(c.he_conv2d_otf(g, dw, dct, r=dr))
    y = u32(c.he_conv2d_otf(g, dw, dct))
    assert (ym == u32(c.he_conv2d(g, c.encode_weights(g, dw), dct, r=dr))).all()
    for b in range(B):
        for i in ([0, g.Cout - 1] if g.Cout > 1 else [0]):
            want = oracle.conv_alg1(ct[b], w, geo, c.primes, i, i + 1)
            sl = slice(i * g.bands, (i + 1) * g.bands)
            assert (y[b, sl] == want).all()
            assert (ym[b, sl] == oracle.mask(want, r[b, sl], c.primes)).all()


# ------------------------------------------------------------------ byte-split tensor-core contraction
TC_CASES = CASES + [
    (2048, 2, (8, 40, 6, 6, 3, 1, 1), 9),        # 18 columns: three column groups, the last ragged; 3 row tiles
    (4096, 3, (96, 17, 8, 8, 3, 1, 1), 3),       # several K steps, Cout 17
]


@pytest.mark.parametrize("N,L,shape,B", TC_CASES)
def test_tc_form_bit_exact(fg, oracle, N, L, shape, B):
    """The tensor-core form gives the plain form's ciphertexts from the same
    encoded weights, with and without the mask, and matches the oracle's
    Algorithm 1 on sampled output channels."""
    c = ctx(fg, N, L)
    g = c.geom(*shape)
    geo = oracle.geometry(N, *shape)
    w = synth.weights(14, (g.Cout, g.Cin, g.k, g.k))
    ct = synth.raw_ciphertexts(14, c.primes, (B, g.n_in, 2, L, N))
    r = synth.masks(14, (B, g.n_out, N), T)
    dw, dct, dr = dev(w, torch.int8), dev(ct), dev(r)
    wh = c.encode_weights(g, dw)
    ym = u32(c.he_conv2d_tc(g, wh, dct, r=dr))
    y = u32(c.he_conv2d_tc(g, wh, dct))
    assert (ym == u32(c.he_conv2d(g, wh, dct, r=dr))).all()
    assert (y == u32(c.he_conv2d(g, wh, dct))).all()
    assert (u32(dct) == ct).all()
    for b in (0, B - 1):
        for i in ([0, g.Cout - 1] if g.Cout > 1 else [0]):
            want = oracle.conv_alg1(ct[b], w, geo, c.primes, i, i + 1)
            sl = slice(i * g.bands, (i + 1) * g.bands)
            assert (y[b, sl] == want).all()
            assert (ym[b, sl] == oracle.mask(want, r[b, sl], c.primes)).all()


def test_tc_form_extreme_digits(fg):
    """Weights and inputs whose three low bytes are all 255 (the largest digit
    products) and G = 20, so every tensor-core partial sum is at its bound:
    the tensor-core form still equals the plain form."""
    N, L = 2048, 2
    c = ctx(fg, N, L)
    g = c.geom(160, 20, 14, 14, 3, 1, 1)  # 8 channels of 16 x 16 padded rows per ciphertext
    assert g.G == 20
    big = [((q >> 24) << 24) - 1 for q in c.primes]  # bytes ff ff ff, then the top byte minus one
    wh = torch.empty((L, g.Cout, g.G, N), dtype=torch.int32, device="cuda")
    ct = torch.empty((1, g.n_in, 2, L, N), dtype=torch.int32, device="cuda")
    for l, v in enumerate(big):
        wh[l] = int(np.uint32(v).view(np.int32))
        ct[:, :, :, l] = int(np.uint32(v).view(np.int32))
    r = dev(synth.masks(15, (1, g.n_out, N), T))
    assert torch.equal(c.he_conv2d_tc(g, wh, ct, r=r), c.he_conv2d(g, wh, ct, r=r))


def test_tc_form_empty_batch(fg):
    c = ctx(fg, 2048, 2)
    g = c.geom(3, 4, 8, 8, 3, 1, 1)
    wh = c.encode_weights(g, torch.zeros((4, 3, 3, 3), dtype=torch.int8, device="cuda"))
    empty = torch.empty((0, g.n_in, 2, 2, 2048), dtype=torch.int32, device="cuda")
    assert c.he_conv2d_tc(g, wh, empty, workspace=torch.empty(16, dtype=torch.int32, device="cuda")).shape[0] == 0


def test_tc_form_refuses_g_beyond_shared_memory(fg):
    """G = 200 input ciphertexts do not fit one CTA's shared memory in the
    tensor-core form: refused on the host before any launch; the plain form
    still takes the layer."""
    N, L = 2048, 1
    c = ctx(fg, N, L)
    g = c.geom(1600, 1, 14, 14, 3, 1, 1)  # 8 channels of 16 x 16 padded rows per ciphertext
    assert g.G == 200
    wh = torch.zeros((L, g.Cout, g.G, N), dtype=torch.int32, device="cuda")
    ct = torch.zeros((1, g.n_in, 2, L, N), dtype=torch.int32, device="cuda")
    with pytest.raises(fg.FlashError, match="shared memory"):
        c.he_conv2d_tc(g, wh, ct)
    assert int(c.he_conv2d(g, wh, ct).abs().sum()) == 0
