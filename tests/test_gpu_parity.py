"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

All comparisons are bit-exact: the whole path is exact modular arithmetic.
Inputs come from the seeded generators in paper_2401_16732_gb300.synth and
are handed unchanged to both sides."""
import math

import numpy as np
import pytest

from paper_2401_16732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
T = 65537


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def dev(a, dtype=torch.int32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda() if a.dtype != np.uint32 else \
        torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


@pytest.fixture(scope="module")
def fg():
    from paper_2401_16732_gb300 import flashgpu
    return flashgpu


_ctx = {}


def ctx(fg, N, L):
    if (N, L) not in _ctx:
        _ctx[(N, L)] = fg.Context(N, L)
    return _ctx[(N, L)]


# ------------------------------------------------------------------ params
@pytest.mark.parametrize("N,L", [(2048, 1), (4096, 2), (8192, 3), (16384, 4)])
def test_context_parameters_match_oracle(fg, oracle, N, L):
    c = ctx(fg, N, L)
    assert c.primes == oracle.find_primes(N, L)
    assert c.delta == oracle.delta_residues(c.primes, T)
    for q, psi in zip(c.primes, c.psi):
        assert pow(psi, N, q) == q - 1  # primitive 2N-th root


# ------------------------------------------------------------------ NTT
@pytest.mark.parametrize("N,L", [(2048, 2), (4096, 2), (8192, 3), (16384, 4)])
def test_ntt_roundtrip_and_definition(fg, N, L):
    c = ctx(fg, N, L)
    a = synth.raw_ciphertexts(1, c.primes, (3, L, N))
    d = dev(a)
    c.ntt_forward(d)
    A = u32(d).copy()
    c.ntt_inverse(d)
    assert (u32(d) == a).all()
    # forward slot k = a(psi^(2 brev(k) + 1)) on sampled slots
    logn = N.bit_length() - 1
    rng = np.random.default_rng(0)
    for l, (q, psi) in enumerate(zip(c.primes, c.psi)):
        coeffs = [int(v) for v in a[1, l]]
        for k in list(rng.integers(0, N, 6)) + [0, N - 1]:
            br = int(format(int(k), f"0{logn}b")[::-1], 2)
            z = pow(psi, 2 * br + 1, q)
            acc, zp = 0, 1
            for cf in coeffs:
                acc = (acc + cf * zp) % q
                zp = zp * z % q
            assert A[1, l, k] == acc


@pytest.mark.parametrize("N,L", [(2048, 1), (8192, 3)])
def test_ntt_product_is_negacyclic_product(fg, oracle, N, L):
    c = ctx(fg, N, L)
    a = synth.raw_ciphertexts(2, c.primes, (1, L, N))
    b = synth.raw_ciphertexts(3, c.primes, (1, L, N))
    da, db = dev(a), dev(b)
    c.ntt_forward(da)
    c.ntt_forward(db)
    q = torch.tensor(c.primes, dtype=torch.int64, device="cuda").view(1, L, 1)
    prod = (da.to(torch.int64) * db.to(torch.int64)) % q
    p32 = prod.to(torch.int32).contiguous()
    c.ntt_inverse(p32)
    got = u32(p32)
    for l in range(L):
        assert (got[0, l] == oracle.negacyclic_mul(a[0, l], b[0, l], c.primes[l])).all()


# ------------------------------------------------------------------ client side
def encrypt_both(fg, oracle, c, g, B, seed):
    N, L = c.N, c.L
    s = synth.secret_key(seed, N)
    x = synth.activations(seed, (B, g.Cin, g.H, g.W))
    a = synth.uniform_residues(seed, c.primes, (B, g.n_in, L, N))
    e = synth.cbd_noise(seed, (B, g.n_in, N))
    sk = c.keygen(dev(s, torch.int8))
    ct = c.encrypt(sk, g, dev(x), dev(a), dev(e))
    geo = oracle.geometry(N, g.Cin, g.Cout, g.H, g.W, g.k, g.stride, g.pad)
    want = np.stack([oracle.encrypt(s, a[b], e[b], oracle.pack_inputs(x[b], geo), c.primes) for b in range(B)])
    return s, x, sk, ct, want, geo


@pytest.mark.parametrize("N,L,shape", [
    (4096, 2, (16, 16, 16, 16, 3, 1, 1)),   # the single-layer workload
    (2048, 3, (5, 3, 9, 9, 3, 2, 1)),       # stride 2, ragged last ct
    (2048, 2, (2, 2, 40, 40, 3, 1, 1)),     # row bands
])
def test_encrypt_decrypt_match_oracle(fg, oracle, N, L, shape):
    c = ctx(fg, N, L)
    g = c.geom(*shape)
    s, x, sk, ct, want, geo = encrypt_both(fg, oracle, c, g, 2, 21)
    assert (u32(ct) == want).all()
    m = u32(c.decrypt(sk, ct))
    for b in range(2):
        assert (m[b] == oracle.pack_inputs(x[b], geo)).all()
        assert (m[b] == oracle.decrypt(s, want[b], c.primes)).all()


def test_online_encryption_algorithm2(fg, oracle):
    c = ctx(fg, 4096, 2)
    g = c.geom(16, 16, 16, 16, 3, 1, 1)
    N, L = c.N, c.L
    s = synth.secret_key(4, N)
    x = synth.activations(4, (1, 16, 16, 16))
    a = synth.uniform_residues(4, c.primes, (1, g.n_in, L, N))
    e = synth.cbd_noise(4, (1, g.n_in, N))
    sk = c.keygen(dev(s, torch.int8))
    enc0 = c.encrypt(sk, g, dev(np.zeros_like(x)), dev(a), dev(e))
    ct = c.encrypt_online(g, dev(x), enc0)
    geo = oracle.geometry(N, 16, 16, 16, 16, 3, 1, 1)
    assert (u32(ct)[0] == oracle.encrypt(s, a[0], e[0], oracle.pack_inputs(x[0], geo), c.primes)).all()


# ------------------------------------------------------------------ weights
@pytest.mark.parametrize("N,L,shape", [(4096, 2, (16, 16, 16, 16, 3, 1, 1)), (2048, 3, (40, 3, 6, 6, 3, 1, 1)),
                                       (2048, 2, (3, 4, 40, 40, 7, 2, 3))])
def test_encode_weights_matches_weight_polynomials(fg, oracle, N, L, shape):
    c = ctx(fg, N, L)
    g = c.geom(*shape)
    w = synth.weights(5, (g.Cout, g.Cin, g.k, g.k))
    wh = c.encode_weights(g, dev(w, torch.int8))
    coeff = wh.clone().view(L * g.Cout * g.G, N)
    # back to coefficients, limb by limb (rows of one limb share the limb's prime)
    got = np.empty((L, g.Cout, g.G, N), np.uint32)
    for l in range(L):
        blk = coeff[l * g.Cout * g.G:(l + 1) * g.Cout * g.G]
        tmp = torch.zeros(blk.shape[0], L, N, dtype=torch.int32, device="cuda")
        tmp[:, l] = blk
        c.ntt_inverse(tmp)
        got[l] = u32(tmp[:, l]).reshape(g.Cout, g.G, N)
    geo = oracle.geometry(N, *shape)
    # the encoded weights are NTT(W_{i,g}) * N^-1 (the fused kernel's inverse NTT leaves N^-1 out)
    for l, q in enumerate(c.primes):
        for i in range(g.Cout):
            for gg in range(g.G):
                back = got[l, i, gg].astype(np.int64) * N % q
                assert (back == oracle.weight_poly(w, i, gg, geo, q)).all()


# ------------------------------------------------------------------ the hot path
CONV_CASES = [
    # N, L, (Cin, Cout, H, W, k, s, p), B
    (4096, 2, (16, 16, 16, 16, 3, 1, 1), 1),     # single-layer workload, full
    (4096, 2, (16, 16, 16, 16, 3, 1, 1), 3),     # batch
    (2048, 3, (7, 5, 9, 9, 3, 2, 1), 2),         # stride 2, ragged last ct
    (2048, 2, (9, 6, 12, 12, 1, 2, 0), 2),       # 1x1 stride-2 shortcut
    (2048, 2, (160, 3, 14, 14, 3, 1, 1), 1),     # G = 20 > 16: a fold in the 64-bit accumulator
    (2048, 2, (3, 4, 40, 40, 7, 2, 3), 2),       # 7x7/2 stem with row bands
    (8192, 3, (3, 8, 32, 32, 3, 1, 1), 1),       # ResNet-18 stem shape, N = 8192
    (16384, 4, (5, 3, 30, 30, 3, 1, 1), 1),      # N = 16384, L = 4
    (2048, 3, (8, 101, 6, 6, 3, 1, 1), 2),       # odd Cout, grid beyond two waves
    (8192, 3, (40, 150, 8, 8, 3, 1, 1), 1),      # 450 CTAs at N = 8192
]


@pytest.mark.parametrize("N,L,shape,B", CONV_CASES)
def test_he_conv2d_bit_exact_vs_oracle(fg, oracle, N, L, shape, B):
    c = ctx(fg, N, L)
    g = c.geom(*shape)
    geo = oracle.geometry(N, *shape)
    w = synth.weights(6, (g.Cout, g.Cin, g.k, g.k))
    ct = synth.raw_ciphertexts(6, c.primes, (B, g.n_in, 2, L, N))
    r = synth.masks(6, (B, g.n_out, N), T)
    wh = c.encode_weights(g, dev(w, torch.int8))
    d_ct, d_r = dev(ct), dev(r)
    y = u32(c.he_conv2d(g, wh, d_ct))
    ym = u32(c.he_conv2d(g, wh, d_ct, r=d_r))
    y2 = c.he_conv2d(g, wh, d_ct)
    ys = u32(c.mask_to_share(y2, d_r))
    ws = c.workspace(g, B)
    c.he_conv2d_ntt_inputs(g, d_ct, ws)
    yst = u32(c.he_conv2d_from_ntt(g, B, wh, ws, torch.empty_like(y2), r=d_r))
    assert (yst == ym).all()  # the two staged calls equal the fused call
    assert (u32(d_ct) == ct).all()  # input untouched
    for b in range(B):
        want = oracle.conv_alg1(ct[b], w, geo, c.primes)
        assert (y[b] == want).all()
        if b == 0:
            assert (want == oracle.conv_poly(ct[b], w, geo, c.primes)).all()
        wm = oracle.mask(want, r[b], c.primes)
        assert (ym[b] == wm).all()
        assert (ys[b] == wm).all()


@pytest.mark.parametrize("N,L,shape", [(4096, 2, (16, 16, 16, 16, 3, 1, 1)), (2048, 2, (3, 4, 40, 40, 7, 2, 3)),
                                       (2048, 3, (7, 5, 9, 9, 3, 2, 1))])
def test_decrypt_of_gpu_conv_is_integer_conv2d(fg, oracle, N, L, shape):
    """O3 end to end on the GPU: encrypt, convolve, mask, decrypt; the shares
    reconstruct conv2d(x, w) mod t and the noise stays within its bound."""
    c = ctx(fg, N, L)
    g = c.geom(*shape)
    B = 2
    s, x, sk, ct, want_ct, geo = encrypt_both(fg, oracle, c, g, B, 31)
    w = synth.weights(31, (g.Cout, g.Cin, g.k, g.k))
    r = synth.masks(31, (B, g.n_out, N), T)
    wh = c.encode_weights(g, dev(w, torch.int8))
    y = c.he_conv2d(g, wh, ct, r=dev(r))
    client = c.decrypt(sk, y)
    yo = u32(c.extract_outputs(g, client)).astype(np.int64)
    server = (T - r.astype(np.int64)) % T
    for b in range(B):
        ref = oracle.conv2d_int(x[b], w, g.stride, g.pad) % T
        share_sum = (u32(client)[b].astype(np.int64) + server[b]) % T
        assert (oracle.extract_outputs(share_sum, geo) == ref).all()
        assert ((yo[b] - oracle.extract_outputs(r[b].astype(np.int64), geo)) % T == ref).all()
        yb = u32(y)[b]
        assert oracle.noise_inf(s, yb, u32(client)[b], c.primes) <= oracle.noise_bound(w, c.primes, masked=True)


# ------------------------------------------------------------------ full size, sampled
RESNET18_SAMPLED = [
    # (Cin, Cout, H, W, k, s, p) of ResNet-18 CIFAR layers at N = 8192
    (3, 64, 32, 32, 3, 1, 1), (64, 64, 32, 32, 3, 1, 1), (64, 128, 32, 32, 3, 2, 1), (64, 128, 32, 32, 1, 2, 0),
    (128, 256, 16, 16, 3, 2, 1), (256, 256, 8, 8, 3, 1, 1), (512, 512, 4, 4, 3, 1, 1),
]


@pytest.mark.parametrize("shape", RESNET18_SAMPLED)
def test_full_size_resnet18_layers_sampled(fg, oracle, shape):
    c = ctx(fg, 8192, 3)
    g = c.geom(*shape)
    geo = oracle.geometry(8192, *shape)
    w = synth.weights(7, (g.Cout, g.Cin, g.k, g.k))
    ct = synth.raw_ciphertexts(7, c.primes, (1, g.n_in, 2, 3, 8192))
    r = synth.masks(7, (1, g.n_out, 8192), T)
    wh = c.encode_weights(g, dev(w, torch.int8))
    y = u32(c.he_conv2d(g, wh, dev(ct), r=dev(r)))
    for i in (0, g.Cout // 2 + 1, g.Cout - 1):
        want = oracle.mask(oracle.conv_alg1(ct[0], w, geo, c.primes, i, i + 1), r[0, i:i + 1], c.primes)
        assert (y[0, i:i + 1] == want).all(), i


def test_full_size_resnet50_stem_sampled(fg, oracle):
    """7x7/2 stem on 3x224x224 at N = 16384: four row bands per channel."""
    c = ctx(fg, 16384, 4)
    shape = (3, 64, 224, 224, 7, 2, 3)
    g = c.geom(*shape)
    assert (g.bands, g.n_in, g.n_out) == (4, 12, 256)
    geo = oracle.geometry(16384, *shape)
    w = synth.weights(8, (64, 3, 7, 7))
    ct = synth.raw_ciphertexts(8, c.primes, (1, g.n_in, 2, 4, 16384))
    wh = c.encode_weights(g, dev(w, torch.int8))
    y = u32(c.he_conv2d(g, wh, dev(ct)))
    for i in (0, 37):
        want = oracle.conv_alg1(ct[0], w, geo, c.primes, i, i + 1)
        assert (y[0, i * 4:(i + 1) * 4] == want).all()


# ------------------------------------------------------------------ edges and errors
def test_empty_batch_and_argument_errors(fg):
    c = ctx(fg, 4096, 2)
    g = c.geom(16, 16, 16, 16, 3, 1, 1)
    wh = torch.zeros(2, 16, g.G, 4096, dtype=torch.int32, device="cuda")
    ws = c.workspace(g, 1)
    out = torch.zeros(1, g.n_out, 2, 2, 4096, dtype=torch.int32, device="cuda")
    ct = torch.zeros(1, g.n_in, 2, 2, 4096, dtype=torch.int32, device="cuda")
    import ctypes
    lib = fg._lib
    # B = 0 is a no-op
    assert lib.fl_he_conv2d(c.h, ctypes.byref(g), 0, fg._ptr(wh), fg._ptr(ct), fg._ptr(out), fg._ptr(ws), 0,
                            None) == 0
    # short workspace
    assert lib.fl_he_conv2d(c.h, ctypes.byref(g), 1, fg._ptr(wh), fg._ptr(ct), fg._ptr(out), fg._ptr(ws), 16,
                            None) == fg.FL_ERR_ARG
    # misaligned pointer
    assert lib.fl_he_conv2d(c.h, ctypes.byref(g), 1, fg._ptr(wh), ctypes.c_void_p(ct.data_ptr() + 4), fg._ptr(out),
                            fg._ptr(ws), ws.numel() * 4, None) == fg.FL_ERR_ARG
    # geometry of another ring degree
    g2 = fg.fl_conv_geom_make(8192, 16, 16, 16, 16, 3, 1, 1)
    assert lib.fl_he_conv2d(c.h, ctypes.byref(g2), 1, fg._ptr(wh), fg._ptr(ct), fg._ptr(out), fg._ptr(ws),
                            ws.numel() * 4, None) == fg.FL_ERR_SHAPE
    # tampered geometry
    g3 = c.geom(16, 16, 16, 16, 3, 1, 1)
    g3.G = 1
    assert lib.fl_he_conv2d(c.h, ctypes.byref(g3), 1, fg._ptr(wh), fg._ptr(ct), fg._ptr(out), fg._ptr(ws),
                            ws.numel() * 4, None) == fg.FL_ERR_SHAPE
    assert "inconsistent" in fg.fl_last_error()
    # a batch whose row count does not fit one launch is refused before any pointer is used
    huge = (1 << 31) // (g.n_in * 2 * 2) + 1
    assert lib.fl_he_conv2d(c.h, ctypes.byref(g), huge, None, None, None, None, ctypes.c_size_t(-1).value,
                            None) == fg.FL_ERR_ARG
    assert "exceed one launch" in fg.fl_last_error()
    with pytest.raises(fg.FlashError):
        fg.Context(1000, 2)
    with pytest.raises(fg.FlashError):
        fg.Context(4096, 5)
    torch.cuda.synchronize()


def test_maximum_residues(fg, oracle):
    """All inputs at q_l - 1 and all weights at -8: the largest products and
    accumulators the contraction can see."""
    c = ctx(fg, 2048, 2)
    shape = (40, 2, 6, 6, 3, 1, 1)
    g = c.geom(*shape)
    geo = oracle.geometry(2048, *shape)
    ct = np.empty((1, g.n_in, 2, 2, 2048), np.uint32)
    for l, q in enumerate(c.primes):
        ct[..., l, :] = q - 1
    w = np.full((2, 40, 3, 3), -8, np.int8)
    wh = c.encode_weights(g, dev(w, torch.int8))
    y = u32(c.he_conv2d(g, wh, dev(ct)))
    assert (y[0] == oracle.conv_alg1(ct[0], w, geo, c.primes)).all()


# ------------------------------------------------------------------ many layers in one launch
STACKS = [
    (2048, 2, [((7, 5, 9, 9, 3, 2, 1), 2, True), ((160, 3, 14, 14, 3, 1, 1), 1, False),
               ((3, 4, 40, 40, 7, 2, 3), 2, True), ((9, 6, 12, 12, 1, 2, 0), 0, True)]),
    (4096, 2, [((16, 16, 16, 16, 3, 1, 1), 1, True), ((16, 16, 16, 16, 3, 1, 1), 3, True),
               ((40, 7, 8, 8, 1, 1, 0), 2, False)]),
    (8192, 3, [((3, 8, 32, 32, 3, 1, 1), 1, True), ((64, 12, 32, 32, 3, 2, 1), 2, True),
               ((128, 9, 16, 16, 1, 2, 0), 1, False), ((512, 5, 4, 4, 3, 1, 1), 1, True)]),
    (16384, 4, [((5, 3, 30, 30, 3, 1, 1), 1, True), ((3, 6, 224, 224, 7, 2, 3), 1, True)]),
]


@pytest.mark.parametrize("kernel", ["per_layer", "persistent", "queue"])
@pytest.mark.parametrize("N,L,layers", STACKS)
def test_stack_equals_single_layer_and_oracle(fg, oracle, N, L, layers, kernel):
    c = ctx(fg, N, L)
    c.stack_kernel = {"per_layer": fg.FL_STACK_PER_LAYER, "persistent": fg.FL_STACK_PERSISTENT,
                      "queue": fg.FL_STACK_QUEUE}[kernel]
    specs, ref = [], []
    for li, (shape, B, masked) in enumerate(layers):
        g = c.geom(*shape)
        w = synth.weights(40 + li, (g.Cout, g.Cin, g.k, g.k))
        ct = synth.raw_ciphertexts(40 + li, c.primes, (B, g.n_in, 2, L, N))
        r = synth.masks(40 + li, (B, g.n_out, N), T) if masked else None
        wh = c.encode_weights(g, dev(w, torch.int8))
        sp = {"g": g, "w_hat": wh, "ct_in": dev(ct), "r": dev(r) if masked else None,
              "out": torch.full((B, g.n_out, 2, L, N), -1, dtype=torch.int32, device="cuda"),
              "w": w, "ct": ct, "rr": r, "shape": shape}
        specs.append(sp)
    arr = c.stack_layers(specs)
    ws = c.stack_workspace(arr)
    c.he_conv2d_stack(arr, ws)
    assert c.stack_error(ws) == 0
    for sp in specs:
        B = sp["ct_in"].shape[0]
        if B == 0:
            continue
        single = u32(c.he_conv2d(sp["g"], sp["w_hat"], sp["ct_in"], r=sp["r"]))
        got = u32(sp["out"])
        assert (got == single).all(), sp["shape"]
        geo = oracle.geometry(N, *sp["shape"])
        i_hi = min(sp["g"].Cout, 2)
        want = oracle.conv_alg1(sp["ct"][B - 1], sp["w"], geo, c.primes, 0, i_hi)
        if sp["rr"] is not None:
            want = oracle.mask(want, sp["rr"][B - 1, :i_hi * geo.bands], c.primes)
        assert (got[B - 1, :i_hi * geo.bands] == want).all(), sp["shape"]
    # a second run through the split stages gives the same outputs
    outs = [sp["out"].clone() for sp in specs]
    for sp in specs:
        sp["out"].fill_(-1)
    c.he_conv2d_stack(arr, ws, stage="ntt")
    c.he_conv2d_stack(arr, ws, stage="run")
    assert c.stack_error(ws) == 0
    for sp, o in zip(specs, outs):
        assert torch.equal(sp["out"], o)
    c.stack_kernel = fg.FL_STACK_PER_LAYER


@pytest.mark.parametrize("kernel", ["per_layer", "persistent", "queue"])
def test_stack_at_the_layer_limit(fg, kernel):
    """FL_STACK_MAX_LAYERS (64) layers of four alternating shapes, some
    masked, some with B = 0, in one stack call: every output equals the
    single-layer call; one layer more is refused before any launch."""
    N, L = 2048, 2
    c = ctx(fg, N, L)
    c.stack_kernel = {"per_layer": fg.FL_STACK_PER_LAYER, "persistent": fg.FL_STACK_PERSISTENT,
                      "queue": fg.FL_STACK_QUEUE}[kernel]
    shapes = [(3, 4, 8, 8, 3, 1, 1), (8, 5, 10, 10, 1, 2, 0), (20, 3, 6, 6, 3, 1, 1), (4, 17, 12, 12, 3, 2, 1)]
    geoms = [c.geom(*sh) for sh in shapes]
    whs = [c.encode_weights(g, dev(synth.weights(96, (g.Cout, g.Cin, g.k, g.k), k), torch.int8))
           for k, g in enumerate(geoms)]
    specs, want = [], []
    for li in range(fg.FL_STACK_MAX_LAYERS):
        g, wh = geoms[li % 4], whs[li % 4]
        B = (li % 3) if li % 7 else 0
        ct = dev(synth.raw_ciphertexts(97, c.primes, (B, g.n_in, 2, L, N), li))
        r = dev(synth.masks(97, (B, g.n_out, N), T, li)) if li % 2 else None
        out = torch.full((B, g.n_out, 2, L, N), -1, dtype=torch.int32, device="cuda")
        specs.append({"g": g, "w_hat": wh, "ct_in": ct, "r": r, "out": out})
        want.append(c.he_conv2d(g, wh, ct, r=r) if B else out.clone())
    arr = c.stack_layers(specs)
    ws = c.stack_workspace(arr)
    c.he_conv2d_stack(arr, ws)
    assert c.stack_error(ws) == 0
    for sp, w in zip(specs, want):
        assert torch.equal(sp["out"], w)
    over = c.stack_layers(specs + specs[:1])
    with pytest.raises(fg.FlashError, match="n_layers"):
        c.he_conv2d_stack(over, ws)
    c.stack_kernel = fg.FL_STACK_PER_LAYER


def test_stack_empty(fg):
    c = ctx(fg, 4096, 2)
    arr = c.stack_layers([])
    ws = torch.empty(64, dtype=torch.int32, device="cuda")
    c.he_conv2d_stack(arr, ws)
    assert c.stack_error(ws) == 0


def test_stack_keeps_inline_tensors_alive(fg):
    """A mask built inline in the layer specs must stay allocated while the
    layer array exists: otherwise the workspace allocated next reuses its
    memory and every masked output differs."""
    N, L = 4096, 2
    c = ctx(fg, N, L)
    g = c.geom(16, 16, 16, 16, 3, 1, 1)
    w = synth.weights(90, (16, 16, 3, 3))
    ct = dev(synth.raw_ciphertexts(90, c.primes, (1, g.n_in, 2, L, N)))
    r = synth.masks(90, (1, g.n_out, N), T)
    wh = c.encode_weights(g, dev(w, torch.int8))
    want = c.he_conv2d(g, wh, ct, r=dev(r))
    for kernel in (fg.FL_STACK_PER_LAYER, fg.FL_STACK_QUEUE, fg.FL_STACK_PERSISTENT):
        c.stack_kernel = kernel
        outs = [torch.zeros_like(want) for _ in range(2)]
        arr = c.stack_layers([{"g": g, "w_hat": wh, "ct_in": ct, "r": dev(r), "out": o} for o in outs])
        ws = c.stack_workspace(arr)  # would reuse the masks' memory if they had been freed
        ws.fill_(-1)
        c.he_conv2d_stack(arr, ws)
        assert c.stack_error(ws) == 0
        for o in outs:
            assert torch.equal(o, want)
    c.stack_kernel = fg.FL_STACK_PER_LAYER


@pytest.mark.parametrize("graph", [False, True])
def test_autotune_sets_the_fastest_kernel(fg, graph):
    """The autotuner times every stack kernel (eager calls or graph replays),
    leaves the fastest set on the context, and the stack then still gives the
    single-layer result."""
    from paper_2401_16732_gb300.autotune import KERNELS, tune_stack
    N, L = 4096, 2
    c = ctx(fg, N, L)
    g = c.geom(16, 16, 16, 16, 3, 1, 1)
    wh = c.encode_weights(g, dev(synth.weights(93, (16, 16, 3, 3)), torch.int8))
    ct = dev(synth.raw_ciphertexts(93, c.primes, (1, g.n_in, 2, L, N)))
    r = dev(synth.masks(93, (1, g.n_out, N), T))
    want = c.he_conv2d(g, wh, ct, r=r)
    outs = [torch.zeros_like(want) for _ in range(2)]
    arr = c.stack_layers([{"g": g, "w_hat": wh, "ct_in": ct, "r": r, "out": o} for o in outs])
    ws = c.stack_workspace(arr)
    res = tune_stack(c, [{"g": g, "ct_in": ct, "r": r}] * 2, arr, ws, cache=None, graph=graph)
    assert set(res["ms"]) == {name for _, name in KERNELS} and all(v > 0 for v in res["ms"].values())
    assert res["kernel"] == min(res["ms"], key=res["ms"].get)
    assert c.stack_kernel == dict((name, k) for k, name in KERNELS)[res["kernel"]]
    for o in outs:
        o.zero_()
    c.he_conv2d_stack(arr, ws)
    assert c.stack_error(ws) == 0
    for o in outs:
        assert torch.equal(o, want)
    c.stack_kernel = fg.FL_STACK_PER_LAYER


@pytest.mark.parametrize("kernel", ["queue", "per_layer"])
def test_graph_replay_matches_eager(fg, oracle, kernel):
    """A stack (one call: input NTT, then the conv kernel as a programmatic
    dependent launch) and a single-layer conv captured in CUDA graphs and
    replayed on fresh inputs give the eager results bit for bit."""
    N, L = 4096, 2
    c = ctx(fg, N, L)
    c.stack_kernel = fg.FL_STACK_QUEUE if kernel == "queue" else fg.FL_STACK_PER_LAYER
    shapes = [(16, 16, 16, 16, 3, 1, 1), (16, 8, 16, 16, 1, 2, 0)]
    geos = [c.geom(*sh) for sh in shapes]
    whs = [c.encode_weights(g, dev(synth.weights(95, (g.Cout, g.Cin, g.k, g.k), li), torch.int8))
           for li, g in enumerate(geos)]
    cts = [dev(synth.raw_ciphertexts(95, c.primes, (2, g.n_in, 2, L, N), li)) for li, g in enumerate(geos)]
    rs = [dev(synth.masks(95, (2, g.n_out, N), T, li)) for li, g in enumerate(geos)]
    outs = [torch.zeros((2, g.n_out, 2, L, N), dtype=torch.int32, device="cuda") for g in geos]
    arr = c.stack_layers([{"g": g, "w_hat": wh, "ct_in": ct, "r": r, "out": o}
                          for g, wh, ct, r, o in zip(geos, whs, cts, rs, outs)])
    ws = c.stack_workspace(arr)
    single_out = torch.zeros_like(outs[0])
    single_ws = c.workspace(geos[0], 2)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):  # warm-up outside the capture
        c.he_conv2d_stack(arr, ws, stream=st)
        c.he_conv2d(geos[0], whs[0], cts[0], out=single_out, workspace=single_ws, r=rs[0], stream=st)
    st.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        c.he_conv2d_stack(arr, ws, stream=st)
        c.he_conv2d(geos[0], whs[0], cts[0], out=single_out, workspace=single_ws, r=rs[0], stream=st)
    for trial in range(2):
        for li, (g, ct) in enumerate(zip(geos, cts)):  # fresh inputs, same buffers
            ct.copy_(dev(synth.raw_ciphertexts(96 + trial, c.primes, (2, g.n_in, 2, L, N), li)))
        for o in outs:
            o.zero_()
        single_out.zero_()
        with torch.cuda.stream(st):
            graph.replay()
        st.synchronize()
        assert c.stack_error(ws) == 0
        for g, wh, ct, r, o in zip(geos, whs, cts, rs, outs):
            assert torch.equal(o, c.he_conv2d(g, wh, ct, r=r))
        assert torch.equal(single_out, outs[0])
    c.stack_kernel = fg.FL_STACK_PER_LAYER
