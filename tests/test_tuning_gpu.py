"""Every tuning choice the autotuner can make gives bit-identical results.

The NTT pass plan (radix of the two row-strided passes) of the input NTT and
of the tensor-core form's inverse-NTT-rows kernel, and the tensor-core tile
(slot groups per CTA), are checked against the default choice and against
the oracle's Algorithm 1; the autotuner's own choices are checked the same
way after it has set them."""
import numpy as np
import pytest

from paper_2401_16732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
T = 65537


@pytest.fixture(scope="module")
def fg():
    from paper_2401_16732_gb300 import flashgpu
    return flashgpu


def dev(a, dtype=torch.int32):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(dtype).cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("N,L", [(2048, 1), (4096, 2), (8192, 3), (16384, 4)])
def test_every_ntt_plan_gives_the_same_transform(fg, N, L):
    """fl_ntt_forward under every available pass plan equals the default
    plan's transform, and the inverse transform brings it back."""
    c = fg.Context(N, L)
    x = dev(synth.raw_ciphertexts(21, c.primes, (3, L, N)))
    c.ntt_plan = 0
    ref = x.clone()
    c.ntt_forward(ref)
    for r1 in fg.NTT_PLANS[N.bit_length() - 1]:
        c.ntt_plan = r1
        assert c.ntt_plan == r1
        y = x.clone()
        c.ntt_forward(y)
        assert torch.equal(y, ref), r1
        c.ntt_inverse(y)
        assert torch.equal(y, x), r1
    with pytest.raises(fg.FlashError):
        c.ntt_plan = 6
    c.ntt_plan = 0


@pytest.mark.parametrize("N,L,shape,B", [(8192, 3, (64, 24, 32, 32, 3, 1, 1), 2),
                                         (16384, 2, (40, 130, 30, 30, 3, 1, 1), 1),
                                         (4096, 2, (16, 16, 16, 16, 3, 1, 1), 3)])
def test_every_plan_and_tile_is_bit_exact_against_the_oracle(fg, oracle, N, L, shape, B):
    """The plain and tensor-core forms under every pass plan (input NTT,
    inverse-NTT rows) and tile (slot groups per CTA) give the same masked
    ciphertexts, equal to the oracle's Algorithm 1 on the first and last
    output channel of the last image."""
    c = fg.Context(N, L)
    g = c.geom(*shape)
    geo = oracle.geometry(N, *shape)
    w = synth.weights(22, (g.Cout, g.Cin, g.k, g.k))
    ct = synth.raw_ciphertexts(22, c.primes, (B, g.n_in, 2, L, N))
    r = synth.masks(22, (B, g.n_out, N), T)
    wh = c.encode_weights(g, dev(w, torch.int8))
    wt = c.tc_weights(g, wh)
    dct, dr = dev(ct), dev(r)
    want = None
    for r1 in fg.NTT_PLANS[N.bit_length() - 1]:
        c.ntt_plan = r1
        plain = c.he_conv2d(g, wh, dct, r=dr)
        if want is None:
            want = plain
            b = B - 1
            for i in (0, g.Cout - 1):
                sl = slice(i * g.bands, (i + 1) * g.bands)
                ref = oracle.mask(oracle.conv_alg1(ct[b], w, geo, c.primes, i, i + 1), r[b, sl], c.primes)
                assert (u32(plain)[b, sl] == ref).all(), i
        assert torch.equal(plain, want), ("plain", r1)
        for tile in fg.TC_TILES:
            c.tc_tile = tile
            assert c.tc_tile == tile
            assert torch.equal(c.he_conv2d_tc(g, wt, dct, r=dr), want), ("tc", r1, tile)
    assert c.tc_error() == 0
    with pytest.raises(fg.FlashError):
        c.tc_tile = 6
    c.ntt_plan = 0
    c.tc_tile = 0


def test_autotuner_choices_stay_bit_exact(fg, oracle):
    """The autotuner times every pass plan, tile (for the whole step and per
    layer) and per-layer form, leaves valid choices set, and the two-layer
    workload it tuned still gives the plain form's ciphertexts (and the
    oracle's on a sampled channel)."""
    from paper_2401_16732_gb300.autotune import tune_forms, tune_ntt_plan, tune_tc_tile, tune_tc_tiles
    N, L, B = 4096, 2, 2
    c = fg.Context(N, L)
    shapes = [(16, 16, 16, 16, 3, 1, 1), (64, 130, 8, 8, 3, 1, 1)]
    layers, want = [], []
    for li, sh in enumerate(shapes):
        g = c.geom(*sh)
        w = synth.weights(23, (g.Cout, g.Cin, g.k, g.k), li)
        lay = {"g": g, "w": w, "w_hat": c.encode_weights(g, dev(w, torch.int8)),
               "ct_in": dev(synth.raw_ciphertexts(23, c.primes, (B, g.n_in, 2, L, N), li)),
               "r": dev(synth.masks(23, (B, g.n_out, N), T, li)),
               "out": torch.empty((B, g.n_out, 2, L, N), dtype=torch.int32, device="cuda")}
        want.append(c.he_conv2d(lay["g"], lay["w_hat"], lay["ct_in"], r=lay["r"]))
        layers.append(lay)

    def step(st):
        for lay in layers:
            c.he_conv2d(lay["g"], lay["w_hat"], lay["ct_in"], out=lay["out"], r=lay["r"], stream=st)

    plan = tune_ntt_plan(c, step, reps=1)
    assert plan["choice"] in fg.NTT_PLANS[12] and set(plan["ms"]) == {str(p) for p in fg.NTT_PLANS[12]}
    assert c.ntt_plan == plan["choice"]
    lay1 = layers[1]
    wt = c.tc_weights(lay1["g"], lay1["w_hat"])
    tile = tune_tc_tile(c, lambda st: c.he_conv2d_tc(lay1["g"], wt, lay1["ct_in"], out=lay1["out"], r=lay1["r"],
                                                      stream=st), reps=1)
    assert tile["choice"] in fg.TC_TILES and c.tc_tile == tile["choice"]
    per_layer = tune_tc_tiles(c, [dict(lay, w_tc=c.tc_weights(lay["g"], lay["w_hat"])) for lay in layers], reps=1)
    assert all(t["choice"] in fg.TC_TILES and set(t["ms"]) == {str(x) for x in fg.TC_TILES} for t in per_layer)
    assert c.tc_tile == tile["choice"]  # the per-layer timing leaves the context's tile as it was
    forms = tune_forms(c, layers, reps=1, cache=None)
    assert [f["form"] for f in forms] == [lay["form"] for lay in layers]
    for lay, wnt, f in zip(layers, want, forms):
        assert f["form"] in ("plain", "tc") and all(v > 0 for v in f["ms"].values())
        assert f["tc_tile"] in fg.TC_TILES
        if lay["form"] == "tc":
            assert lay["tc_tile"] == f["tc_tile"]
            c.tc_tile = lay["tc_tile"]
            got = c.he_conv2d_tc(lay["g"], lay["w_tc"], lay["ct_in"], r=lay["r"])
        else:
            got = c.he_conv2d(lay["g"], lay["w_hat"], lay["ct_in"], r=lay["r"])
        assert torch.equal(got, wnt)
    geo = oracle.geometry(N, *shapes[1])
    ref = oracle.mask(oracle.conv_alg1(u32(layers[1]["ct_in"])[0], layers[1]["w"], geo, c.primes, 0, 1),
                      u32(layers[1]["r"])[0, :1], c.primes)
    assert (u32(want[1])[0, :1] == ref).all()
    assert c.tc_error() == 0
