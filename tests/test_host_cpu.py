"""Host-side logic that needs no GPU: the benchmark workloads, the serving
loop's request generation and statistics, the synthetic input ranges, and the
bench's algorithmic byte counts."""
import math
import os
import sys

import numpy as np
import pytest

from paper_2401_16732_gb300 import synth
from paper_2401_16732_gb300.workloads import WORKLOADS, resnet18_cifar, resnet50_imagenet

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
T = 65537


def conv_params(layers):
    return sum(cin * cout * k * k for cin, cout, h, w, k, s, p in layers)


def test_resnet18_cifar_has_the_published_parameter_count():
    """The widely published ResNet-18 CIFAR total of 11,173,962 parameters is
    the conv weights plus batch-norm (2 per channel of each BN) plus the
    512x10 classifier; the conv part is what the stack must contain."""
    layers = resnet18_cifar()
    bn_channels = 64 + 4 * 64 + 5 * 128 + 5 * 256 + 5 * 512
    assert conv_params(layers) + 2 * bn_channels + 512 * 10 + 10 == 11_173_962
    # spatial sizes: 32 -> 16 -> 8 -> 4, strides only on the first conv of stages 2-4
    assert [l[2] for l in layers] == [32] * 7 + [16] * 5 + [8] * 5 + [4] * 3
    assert sum(1 for l in layers if l[5] == 2) == 6


def test_resnet50_imagenet_has_the_published_parameter_count():
    """torchvision's ResNet-50 has 25,557,032 parameters: conv weights, batch
    norm (2 per channel) and the 2048x1000 classifier."""
    layers = resnet50_imagenet()
    bn_channels = sum(l[1] for l in layers)  # one BN after every conv
    assert conv_params(layers) + 2 * bn_channels + 2048 * 1000 + 1000 == 25_557_032
    assert layers[0] == (3, 64, 224, 224, 7, 2, 3)
    assert layers[-1][1] == 2048 and layers[-1][2] == 7


def test_workloads_match_their_configurations():
    assert (WORKLOADS["single"].N, WORKLOADS["single"].L, WORKLOADS["single"].B) == (4096, 2, 1)
    assert (WORKLOADS["resnet18"].N, WORKLOADS["resnet18"].L, WORKLOADS["resnet18"].B) == (8192, 3, 1)
    assert WORKLOADS["resnet18-b64"].B == 64
    assert (WORKLOADS["resnet50-b8"].N, WORKLOADS["resnet50-b8"].L, WORKLOADS["resnet50-b8"].B) == (16384, 4, 8)


def test_poisson_requests_are_seeded_and_shaped():
    from paper_2401_16732_gb300.serve import poisson_requests
    a = poisson_requests(400, 200.0, {"x": 0.7, "y": 0.3}, bmax=8, seed=3)
    b = poisson_requests(400, 200.0, {"x": 0.7, "y": 0.3}, bmax=8, seed=3)
    assert [(q.arrival, q.model, q.B) for q in a] == [(q.arrival, q.model, q.B) for q in b]
    arr = np.array([q.arrival for q in a])
    assert (np.diff(arr) > 0).all()
    assert abs(len(a) / arr[-1] - 200.0) < 40.0          # mean rate
    assert all(1 <= q.B <= 8 for q in a)
    share = sum(q.model == "x" for q in a) / len(a)
    assert 0.6 < share < 0.8


def test_latency_stats_percentiles():
    from paper_2401_16732_gb300.serve import Request, latency_stats
    reqs = []
    for i in range(100):
        q = Request(rid=i, model="x", B=1, arrival=0.0)
        q.done = (i + 1) / 1000.0  # 1 .. 100 ms
        reqs.append(q)
    st = latency_stats(reqs)
    assert st["p50_ms"] == pytest.approx(50.0) and st["p99_ms"] == pytest.approx(99.0)
    assert st["max_ms"] == pytest.approx(100.0)
    assert latency_stats([]) == {"p50_ms": None, "p99_ms": None}


def test_synthetic_draws_have_the_stated_ranges():
    x = synth.activations(1, (4, 16, 16))
    w = synth.weights(1, (8, 4, 3, 3))
    s = synth.secret_key(1, 4096)
    e = synth.cbd_noise(1, (2, 4096))
    r = synth.masks(1, (2, 4096), T)
    assert x.min() >= 0 and x.max() <= 255
    assert w.min() >= -8 and w.max() <= 7 and w.dtype == np.int8
    assert set(np.unique(s)) <= {-1, 0, 1}
    assert np.abs(e).max() <= 21 and abs(e.mean()) < 0.2
    assert r.max() < T
    primes = [1073692673, 1073668097]
    a = synth.uniform_residues(1, primes, (3, 2, 4096))
    assert all(a[:, l].max() < q for l, q in enumerate(primes))
    # every purpose and index has its own stream
    assert not np.array_equal(synth.masks(1, (64,), T, 1), synth.masks(1, (64,), T, 2))


def test_bench_algorithmic_bytes_count_every_buffer_once(oracle):
    """layer_bytes (the roofline numerator) counts the encoded weights, the
    NTT-domain inputs, the outputs and the masks once each."""
    sys.path.insert(0, ROOT)
    import bench
    N, L, B = 8192, 3, 2
    g = oracle.geometry(N, 64, 128, 16, 16, 3, 1, 1)
    words = L * g.Cout * g.G * N + B * g.n_in * 2 * L * N + B * g.n_out * 2 * L * N + B * g.n_out * N
    assert bench.layer_bytes(g, B, L, N) == 4 * words
    assert bench.intt_butterflies(g, B, L, N) == B * g.n_out * 2 * L * (N // 2) * int(math.log2(N))


def test_clock_record_uses_the_timed_region_reads():
    """bench.py's clock record: NVML reads taken while the timed steps run
    are preferred; the reasons the record must flag come from their bits."""
    import types
    sys.path.insert(0, ROOT)
    import bench
    reads = iter([(2070.0, 0), (1965.0, 0x4), (2070.0, 0x1)])

    class Ev:
        n = 0

        def query(self):
            Ev.n += 1
            return Ev.n == 3

    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.samples, cs.win = [], []
    cs.nvml = types.SimpleNamespace(read=lambda: next(reads), max_mhz=2070.0)
    cs.poll_until(Ev())
    s = cs.summary()
    assert s["samples_timed_region"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]  # 0x1 (idle) is not a throttle reason
    cs.win = [(1500.0, 0x8 | 0x40)]
    assert cs.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    cs.nvml, cs.win = None, []
    assert cs.summary()["reasons"] == ["no nvidia-smi samples"]  # neither source: said so, no number


def test_reference_arm_prints_one_contract_line(oracle):
    """bench.py --impl reference (the oracle on the host cores) prints one
    JSON line with the keys the benchmark contract asks of that arm."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "single",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "layers/s" and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
