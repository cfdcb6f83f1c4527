"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times.  The whole ResNet-18 CIFAR conv stack (20 layers, N = 8192, L = 3)
runs as one stack call (input NTT of every layer, then the fused contraction
/ inverse NTT / mask kernel) captured in a CUDA graph and replayed.  At B = 1
it runs on the queue kernel, at B = 64 on per-layer launches, the kernels the
autotuner keeps for these workloads; the ResNet-50 ImageNet stack (53
layers, N = 16384, L = 4, B = 8) runs on per-layer launches too.  The
tensor-core form runs the batched stacks per layer as bench.py --form tc
does, and the ResNet-50 stack runs once more with both forms mixed the way
bench.py --form auto runs it.  Sampled outputs, two output channels of every
layer for the last image, are compared bit for bit with the oracle's Algorithm 1 plus the
mask.  The x^2 + x server rounds run over the 1808
activation ciphertexts of bench.py's x2x workload."""
import numpy as np
import pytest

from paper_2401_16732_gb300 import synth
from paper_2401_16732_gb300.workloads import WORKLOADS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
T = 65537


@pytest.fixture(scope="module")
def fg():
    from paper_2401_16732_gb300 import flashgpu
    return flashgpu


def _bench_layers(c, wl, seed, tc=False):
    """Every layer of a workload as bench.py sets it up: encoded weights (as
    tensor-core weight tiles, made right after the encoding, when tc),
    fresh uniform-residue inputs and masks of the layer's shape, and output
    buffers; returns the layer specs and the int8 filters."""
    N, L, B = wl.N, wl.L, wl.B
    specs, filters = [], []
    for li, shape in enumerate(wl.layers):
        g = c.geom(*shape)
        w = synth.weights(seed, (g.Cout, g.Cin, g.k, g.k), li)
        w_hat = c.encode_weights(g, torch.from_numpy(w).to(torch.int8).cuda())
        wk = {"w_tc": c.tc_weights(g, w_hat)} if tc else {"w_hat": w_hat}
        del w_hat
        specs.append({"g": g, **wk,
                      "ct_in": synth.device_uniform_residues(seed, c.primes, (B, g.n_in, 2, L, N), li),
                      "r": synth.device_masks(seed, (B, g.n_out, N), T, li),
                      "out": torch.empty((B, g.n_out, 2, L, N), dtype=torch.int32, device="cuda")})
        filters.append((shape, w))
    return specs, filters


def _replay_once(step):
    """Capture `step(stream)` in a CUDA graph (after one eager run) and
    replay it once, as bench.py's timed step does."""
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        step(stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step(stream)
    return stream, graph


def _check_sampled(oracle, c, wl, specs, filters, channels):
    """Output channels channels(li, Cout) of every layer, for the last image,
    against the oracle's Algorithm 1 plus the mask, bit for bit.  Only those
    rows leave the device."""
    b = wl.B - 1
    for li, (sp, (shape, w)) in enumerate(zip(specs, filters)):
        g = sp["g"]
        geo = oracle.geometry(wl.N, *shape)
        ct_b = sp["ct_in"][b].cpu().numpy().view(np.uint32)
        for i in channels(li, g):
            sl = slice(i * g.bands, (i + 1) * g.bands)
            r_b = sp["r"][b, sl].cpu().numpy().view(np.uint32)
            got = sp["out"][b, sl].cpu().numpy().view(np.uint32)
            want = oracle.mask(oracle.conv_alg1(ct_b, w, geo, c.primes, i, i + 1), r_b, c.primes)
            assert (got == want).all(), (wl.name, li, i)


def _two_channels(li, g):
    return sorted({li % g.Cout, g.Cout - 1})


@pytest.mark.parametrize("config,kernel", [("resnet18", "queue"), ("resnet18-b64", "per_layer"),
                                           ("resnet50-b8", "per_layer")])
def test_full_stack_in_the_bench_configuration(fg, oracle, config, kernel):
    wl = WORKLOADS[config]
    c = fg.Context(wl.N, wl.L)
    c.stack_kernel = {"queue": fg.FL_STACK_QUEUE, "per_layer": fg.FL_STACK_PER_LAYER}[kernel]
    specs, filters = _bench_layers(c, wl, 5)
    arr = c.stack_layers(specs)
    ws = c.stack_workspace(arr)
    stream, graph = _replay_once(lambda st: c.he_conv2d_stack(arr, ws, stream=st))
    for sp in specs:
        sp["out"].fill_(-1)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        graph.replay()
    stream.synchronize()
    assert c.stack_error(ws) == 0
    _check_sampled(oracle, c, wl, specs, filters, _two_channels)
    del arr, ws, graph, specs


@pytest.mark.parametrize("config", ["resnet18-b64", "resnet50-b8"])
def test_tc_form_full_stack_in_the_bench_configuration(fg, oracle, config):
    """The tensor-core form over a whole batched stack, as bench.py --form tc
    runs it (per layer: input NTT, tensor-core contraction, inverse NTT +
    mask; one CUDA graph per step), against the oracle on two output channels
    of every layer.  ResNet-50's layers reach G = 52 input ciphertexts."""
    wl = WORKLOADS[config]
    torch.cuda.empty_cache()  # ResNet-50's weight tiles, outputs and masks take most of the device
    c = fg.Context(wl.N, wl.L)
    specs, filters = _bench_layers(c, wl, 7, tc=True)
    assert max(sp["g"].G for sp in specs) == (52 if config == "resnet50-b8" else 10)
    ws = c.tc_workspace(max((sp["g"] for sp in specs), key=lambda g: c.tc_workspace_bytes(g, wl.B)), wl.B)  # shared
    for sp in specs:
        sp["ws"] = ws

    def step(st):
        for sp in specs:
            c.he_conv2d_tc(sp["g"], sp["w_tc"], sp["ct_in"], out=sp["out"], workspace=sp["ws"], r=sp["r"],
                           stream=st)

    stream, graph = _replay_once(step)
    for sp in specs:
        sp["out"].fill_(-1)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        graph.replay()
    stream.synchronize()
    _check_sampled(oracle, c, wl, specs, filters, _two_channels)
    del graph, specs


def test_mixed_forms_full_stack_as_the_autotuned_step(fg, oracle):
    """ResNet-50 B=8 as bench.py --form auto runs it: the plain layers as one
    stack call on the queue kernel, then the tensor-core layers one by one
    with a shared workspace, all in one CUDA graph.  The forms follow the
    layers' shapes the way the autotuner measures them to fall (tensor
    cores where G >= 7 and Cout >= 128), so that both forms cover many layers
    and the queue kernel runs over a full-size N = 16384 stack with gaps
    between its layers.  Two output channels of every layer against the
    oracle."""
    wl = WORKLOADS["resnet50-b8"]
    torch.cuda.empty_cache()
    c = fg.Context(wl.N, wl.L)
    c.stack_kernel = fg.FL_STACK_QUEUE
    N, L, B = wl.N, wl.L, wl.B
    specs, filters = [], []
    for li, shape in enumerate(wl.layers):
        g = c.geom(*shape)
        w = synth.weights(9, (g.Cout, g.Cin, g.k, g.k), li)
        w_hat = c.encode_weights(g, torch.from_numpy(w).to(torch.int8).cuda())
        tc = g.G >= 7 and g.Cout >= 128
        wk = {"w_tc": c.tc_weights(g, w_hat)} if tc else {"w_hat": w_hat}
        del w_hat
        specs.append({"g": g, "tc": tc, **wk,
                      "ct_in": synth.device_uniform_residues(9, c.primes, (B, g.n_in, 2, L, N), li),
                      "r": synth.device_masks(9, (B, g.n_out, N), T, li),
                      "out": torch.empty((B, g.n_out, 2, L, N), dtype=torch.int32, device="cuda")})
        filters.append((shape, w))
    tc_specs = [sp for sp in specs if sp["tc"]]
    assert 10 <= len(tc_specs) <= len(specs) - 10
    arr = c.stack_layers([{k: sp[k] for k in ("g", "w_hat", "ct_in", "r", "out")} for sp in specs if not sp["tc"]])
    ws = c.stack_workspace(arr)
    wst = c.tc_workspace(max((sp["g"] for sp in tc_specs), key=lambda g: c.tc_workspace_bytes(g, B)), B)

    def step(st):
        c.he_conv2d_stack(arr, ws, stream=st)
        for sp in tc_specs:
            c.he_conv2d_tc(sp["g"], sp["w_tc"], sp["ct_in"], out=sp["out"], workspace=wst, r=sp["r"], stream=st)

    stream, graph = _replay_once(step)
    for sp in specs:
        sp["out"].fill_(-1)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        graph.replay()
    stream.synchronize()
    assert c.stack_error(ws) == 0 and c.tc_error() == 0
    _check_sampled(oracle, c, wl, specs, filters, _two_channels)
    del arr, ws, wst, graph, specs


def test_x2x_rounds_at_the_bench_size(fg, oracle):
    """The x^2 + x server rounds over the benchmark's 1808 activation
    ciphertexts (every packed input of ResNet-18 CIFAR's convolutions but the
    stem, B = 16, N = 8192, L = 3), launched as bench.py does; the first, a
    middle and the last ciphertext against the oracle's two rounds."""
    wl = WORKLOADS["resnet18"]
    N, L = wl.N, wl.L
    c = fg.Context(N, L)
    n = 16 * sum(c.geom(*sh).n_in for sh in wl.layers[1:])
    assert n == 1808
    r, v = synth.device_masks(6, (n, N), T, 1), synth.device_masks(6, (n, N), T, 2)
    prep = c.x2x_prepare(r, v)
    ct_z, ct_x, ct_y = (synth.device_uniform_residues(6, c.primes, (n, 2, L, N), k) for k in (3, 4, 5))
    stream = torch.cuda.Stream()
    out1, out2 = torch.empty_like(ct_z), torch.empty_like(ct_z)
    torch.cuda.synchronize()  # inputs and prepared rows come from the default stream
    c.x2x_round1(prep, ct_z, out1, stream=stream)
    c.x2x_round2(prep, ct_x, ct_y, out2, stream=stream)
    stream.synchronize()

    def h(t, k):
        return t[k:k + 1].cpu().numpy().view(np.uint32)

    for k in (0, n // 2, n - 1):
        assert (h(out1, k) == oracle.x2x_server_round1(h(ct_z, k), h(r, k), h(v, k), c.primes)).all(), k
        assert (h(out2, k) == oracle.x2x_server_round2(h(ct_x, k), h(ct_y, k), h(r, k), h(v, k), c.primes)).all(), k
