"""Parity of the two other GPU forms of the convolution with the oracle's
Algorithm 1 (route O2) and with the NTT route: the direct form (DRot + CMult,
no NTT) and on-the-fly weights (weight polynomials rebuilt and transformed
in shared memory, no encoded weights).  All comparisons are bit-exact."""
import ctypes

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


# ------------------------------------------------------------------ tensor-core contraction (tcgen05)
TC_CASES = CASES + [
    (2048, 2, (8, 40, 6, 6, 3, 1, 1), 9),        # 18 columns: two column tiles, the second ragged
    (4096, 3, (96, 17, 8, 8, 3, 1, 1), 3),       # several K steps, Cout 17
    (2048, 2, (8, 300, 6, 6, 3, 1, 1), 2),       # three output-channel tiles, the last ragged
    (2048, 1, (512, 8, 14, 14, 3, 1, 1), 1),     # G = 64, the exactness limit (bias in its own K step)
    (2048, 2, (504, 5, 14, 14, 3, 1, 1), 2),     # G = 63 (bias in the last K step)
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
    ym = u32(c.he_conv2d_tc(g, c.tc_weights(g, wh), dct, r=dr))
    y = u32(c.he_conv2d_tc(g, c.tc_weights(g, wh), dct))
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
    """G = 64 (the exactness limit) with weights and inputs made of residues
    whose balanced digits are extreme (q - 1, 2^24 - 1, and byte patterns
    0x80 / 0x7f that give digits of -128 and 127): the tensor-core form
    still equals the plain form.  No bounded wait ran out."""
    N, L = 2048, 2
    c = ctx(fg, N, L)
    g = c.geom(512, 20, 14, 14, 3, 1, 1)  # 8 channels of 16 x 16 padded rows per ciphertext
    assert g.G == 64
    rng = np.random.default_rng(16)
    for pat in range(3):
        wh = torch.empty((L, g.Cout, g.G, N), dtype=torch.int32, device="cuda")
        ct = torch.empty((1, g.n_in, 2, L, N), dtype=torch.int32, device="cuda")
        for l, q in enumerate(c.primes):
            vals = [q - 1, (1 << 24) - 1, 0x00808080, 0x007F7F7F, 0x3F808080 % q, ((q >> 24) << 24) - 1]
            a = rng.choice(vals, size=(g.Cout, g.G, N)) if pat == 2 else np.full((g.Cout, g.G, N), vals[pat])
            x = rng.choice(vals, size=(1, g.n_in, 2, N)) if pat == 2 else np.full((1, g.n_in, 2, N), vals[pat])
            wh[l] = torch.from_numpy(a.astype(np.uint32).view(np.int32)).cuda()
            ct[:, :, :, l] = torch.from_numpy(x.astype(np.uint32).view(np.int32)).cuda()
        r = dev(synth.masks(15 + pat, (1, g.n_out, N), T))
        assert torch.equal(c.he_conv2d_tc(g, c.tc_weights(g, wh), ct, r=r), c.he_conv2d(g, wh, ct, r=r)), pat
    assert c.tc_error() == 0


def test_tc_form_empty_batch(fg):
    c = ctx(fg, 2048, 2)
    g = c.geom(3, 4, 8, 8, 3, 1, 1)
    wh = c.encode_weights(g, torch.zeros((4, 3, 3, 3), dtype=torch.int8, device="cuda"))
    empty = torch.empty((0, g.n_in, 2, 2, 2048), dtype=torch.int32, device="cuda")
    ws = torch.empty(16, dtype=torch.int32, device="cuda")
    assert c.he_conv2d_tc(g, c.tc_weights(g, wh), empty, workspace=ws).shape[0] == 0


def test_tc_form_stages_equal_the_one_call_form(fg):
    """Input NTT, tensor-core contraction and inverse NTT + mask as three calls
    give fl_he_conv2d_tc's ciphertexts (B = 3, two output-channel tiles)."""
    N, L, B = 2048, 2, 3
    c = ctx(fg, N, L)
    g = c.geom(24, 130, 8, 8, 3, 1, 1)
    wt = c.tc_weights(g, c.encode_weights(g, dev(synth.weights(4, (g.Cout, g.Cin, g.k, g.k)), torch.int8)))
    ct = dev(synth.raw_ciphertexts(4, c.primes, (B, g.n_in, 2, L, N)))
    r = dev(synth.masks(4, (B, g.n_out, N), T))
    want = c.he_conv2d_tc(g, wt, ct, r=r)
    ws = c.tc_workspace(g, B)
    out = torch.full_like(want, -1)
    c.he_conv2d_ntt_inputs(g, ct, ws)
    c.he_conv2d_tc_from_ntt(g, B, wt, ws)
    c.intt_mask_outputs(g, ws, out, r=r)
    assert torch.equal(out, want)
    assert c.tc_error() == 0
    # the outputs are gathered from the workspace: an output buffer inside it
    # is refused before any launch, by the staged call and the one-call form
    inside = ws[ws.numel() - out.numel():].view(out.shape)
    with pytest.raises(fg.FlashError, match="overlap"):
        c.intt_mask_outputs(g, ws, inside, r=r)
    with pytest.raises(fg.FlashError, match="overlap"):
        c.he_conv2d_tc(g, wt, ct, out=inside, workspace=ws, r=r)
    assert torch.equal(c.he_conv2d_tc(g, wt, ct, workspace=ws, r=r), want)


def decode_tc_weights(wt, L, Cout, G, N):
    """Digits of the weight tiles back to [L][rows][4 ceil(G/4)][N] integers
    sum_a d_a 256^a, following the layout fl_tc_weights documents (16 KB per
    (limb, 128-row tile, 4-slot group, K step), slot s at 2048 halves, row r
    and K index k = 4 (g % 4) + a at half ((r / 8) * 2 + k / 8) * 64 +
    (r % 8) * 8 + k % 8), plus the digits themselves."""
    mt, nch = (Cout + 127) // 128, (G + 3) // 4
    h = wt.cpu().numpy().view(np.float16).astype(np.float64)
    assert (h == np.round(h)).all() and h.min() >= -128 and h.max() <= 127
    # [l][mt][u4][kc][s][r/8][k/8][r%8][k%8] -> [l][mt][r/8][r%8][kc][k/8][k%8][u4][s]
    h = h.reshape(L, mt, N // 4, nch, 4, 16, 2, 8, 8).transpose(0, 1, 5, 7, 3, 6, 8, 2, 4)
    d = h.reshape(L, mt * 128, nch * 4, 4, N)  # [l][row][g][a][u]
    v = sum(d[:, :, :, a].astype(np.int64) << (8 * a) for a in range(4))
    return v, d


def test_tc_weights_are_the_digits_of_the_encoded_weights(fg):
    """tc_weights' tiles hold the balanced base-256 digits of every encoded
    weight (in [-128, 127], summing back to the residue) and zeros in the
    padding rows and ciphertexts; two row tiles (the second ragged) and G = 9
    (three K steps, the last ragged)."""
    N, L = 2048, 2
    c = ctx(fg, N, L)
    g = c.geom(180, 130, 8, 8, 3, 1, 1)
    assert g.G == 9
    wh = c.encode_weights(g, dev(synth.weights(3, (g.Cout, g.Cin, g.k, g.k)), torch.int8))
    wt = c.tc_weights(g, wh)
    assert wt.numel() * 2 == fg._lib.fl_tc_weights_bytes(c.h, ctypes.byref(g))
    v, d = decode_tc_weights(wt, L, g.Cout, g.G, N)
    w = wh.cpu().numpy().view(np.uint32).astype(np.int64)
    assert (v[:, :g.Cout, :g.G] == w).all()
    assert (d[:, :g.Cout, g.G:] == 0).all() and (d[:, g.Cout:] == 0).all()


def test_tc_form_refuses_g_beyond_the_exact_range(fg):
    """G = 65 input ciphertexts would let the fp32 digit sums leave the exact
    integer range: refused on the host before any launch (FL_ERR_SHAPE);
    the plain form still takes the layer."""
    N, L = 2048, 1
    c = ctx(fg, N, L)
    g = c.geom(520, 1, 14, 14, 3, 1, 1)  # 8 channels of 16 x 16 padded rows per ciphertext
    assert g.G == fg.FL_TC_MAX_G + 1
    wh = torch.zeros((L, g.Cout, g.G, N), dtype=torch.int32, device="cuda")
    ct = torch.zeros((1, g.n_in, 2, L, N), dtype=torch.int32, device="cuda")
    with pytest.raises(fg.FlashError, match="exact"):
        c.tc_weights(g, wh)
    # the C entry points refuse it too, before touching any buffer
    buf = torch.zeros(1 << 20, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert fg._lib.fl_tc_weights_bytes(c.h, ctypes.byref(g)) == 0
    assert fg._lib.fl_tc_weights(c.h, ctypes.byref(g), p, p, None) == fg.FL_ERR_SHAPE
    assert fg._lib.fl_he_conv2d_tc(c.h, ctypes.byref(g), 1, p, p, None, p, p, buf.numel() * 4, None) != 0
    assert int(c.he_conv2d(g, wh, ct).abs().sum()) == 0
