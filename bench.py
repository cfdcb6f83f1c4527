"""Throughput of the homomorphic convolution path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config resnet18]
    python bench.py --impl reference ...    (the CPU oracle, timed on host cores)

A step is one pass of the hot path (forward NTT of the inputs, per-slot
contraction, inverse NTT, mask addition) over every conv layer of the
workload for one batch of synthetic encrypted inputs.  The default workload
is the ResNet-18 CIFAR conv stack, B = 1, N = 8192, L = 3, t = 65537.  Each
rank runs the full workload on its own GPU (independent images: weak
scaling, no data-path collective).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The batched ResNet-50 stack in the tensor-core form holds most of the device
# (weight tiles, outputs, masks of all 53 layers); growable segments keep
# freed blocks of one size usable for allocations of another.  Read when
# CUDA starts.
os.environ.setdefault("PYTORCH_ALLOC_CONF", "expandable_segments:True")

from paper_2401_16732_gb300 import synth  # noqa: E402
from paper_2401_16732_gb300.workloads import WORKLOADS, Workload  # noqa: E402

T_PLAIN = 65537
FALLBACK_HBM_GBS = 6800.0
FALLBACK_TENSOR_FLOPS = 1.9e15
L2_BYTES = 129e6
# Integer-ALU roofline of the inverse NTT: a lazy Gentleman-Sande butterfly
# with Shoup multiplication needs 4 ALU-pipe operations (sum, conditional
# subtract as add + min, difference) and 3 multiplies; the ALU pipe retires 16
# lanes per clock per SM sub-partition.  152 SMs x 4 x 16 x 2.07 GHz / 4.
ALU_BFLY_DERIVED = 152 * 4 * 16 * 2.07e9 / 4
_ALU = {}


def alu_peak():
    """(butterflies/s, source): the lazy Gentleman-Sande butterfly rate
    measured on this GPU by the roofline-ceiling library (libflpeaks, once
    per process), else the derived figure above."""
    if "v" not in _ALU:
        import ctypes
        try:
            lib = ctypes.CDLL(os.path.join(ROOT, "paper_2401_16732_gb300", "libflpeaks.so"))
            lib.fl_measure_butterfly_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
            v = ctypes.c_double()
            if lib.fl_measure_butterfly_rate(20000, ctypes.byref(v)) != 0 or v.value <= 0:
                raise RuntimeError("measurement failed")
            _ALU["v"] = (v.value, "measured: lazy Gentleman-Sande butterflies from registers on every SM "
                                   "(libflpeaks fl_measure_butterfly_rate), "
                                   f"derived pipe bound {ALU_BFLY_DERIVED / 1e12:.2f} T/s")
        except Exception as exc:  # the figure is reported with its source either way
            _ALU["v"] = (ALU_BFLY_DERIVED, f"derived: 152 SMs x 4 x 16 ALU lanes x 2.07 GHz / 4 ALU ops per "
                                           f"butterfly (measurement unavailable: {exc})")
    return _ALU["v"]
# Direct form: one signed 32x32->64-bit multiply-add per lane per clock on the
# 16-lane integer multiply pipe (an upper bound).
DIRECT_MAC_PEAK = 152 * 4 * 16 * 2.07e9
# DRAM bytes (read + write) of one step's launches of the dominant kernel,
# from one ncu capture of the same command, each with the SHA-256 (first 16
# hex digits) of the kernel sources it was captured from.  The figure is
# reported only while those sources still hash the same; any edit to them
# makes it null until it is captured again.
KERNEL_SOURCES = {  # the kernel's own file and the shared device header
    "queue": ("fl_kernels.cu", "fl_device.cuh"),
    "round1": ("fl_act.cu", "fl_device.cuh"),
    "round2": ("fl_act.cu", "fl_device.cuh"),
    "tc": ("fl_tc.cu",),
    "intt_rows": ("fl_tc.cu", "fl_device.cuh"),
}
TRAFFIC = {  # (config, kernel): (bytes per step, source hash at capture)
    ("resnet18", "queue"): (3.3547e9, "748bd29df427c870"),
    ("x2x", "round1"): (1.0320e9, "809b5fd15108918d"),
    ("x2x", "round2"): (1.0677e9, "809b5fd15108918d"),
}


def kernel_source_hash(kernel):
    """SHA-256 over the named kernel's source files (name and bytes, in a
    fixed order); None for a kernel without a recorded source set."""
    import hashlib
    files = KERNEL_SOURCES.get(kernel)
    if files is None:
        return None
    h = hashlib.sha256()
    for name in files:
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_2401_16732_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_of(config, kernel):
    """ncu DRAM bytes per step for (config, kernel) if they were captured
    from the current sources, else None."""
    rec = TRAFFIC.get((config, kernel))
    if rec is None or rec[1] != kernel_source_hash(kernel):
        return None
    return rec[0]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def tensor_peak():
    """Dense fp16 tensor FLOP/s: the measured bf16 burst figure (fp16 and
    bf16 run at the same dense rate on the tensor cores), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]) * 1e12, "measured (bf16 burst; fp16 dense runs at the same rate)"
    except Exception:
        return FALLBACK_TENSOR_FLOPS, "fallback"


def layer_bytes(g, B, L, N, masked=True):
    """Algorithmic HBM bytes of the fused contraction + INTT + mask kernel for
    one layer: NTT weights, NTT inputs, output ciphertexts, masks."""
    w = L * g.Cout * g.G * N * 4
    cin = B * g.n_in * 2 * L * N * 4
    out = B * g.n_out * 2 * L * N * 4
    r = B * g.n_out * N * 4 if masked else 0
    return w + cin + out + r


def intt_butterflies(g, B, L, N):
    """Butterflies of the inverse NTTs the fused kernel runs for one layer."""
    return B * g.n_out * 2 * L * (N // 2) * (N.bit_length() - 1)


def ntt_bytes(g, B, L, N):
    return 2 * B * g.n_in * 2 * L * N * 4


def slot_macs(g, B, L, N):
    return B * g.n_out * g.G * 2 * L * N


# ---------------------------------------------------------------------------
# CPU oracle leg (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def o2_macs(wl, shape):
    """Multiply-adds Algorithm 1 (route O2) spends on one image of a layer:
    Cout * Cin * k^2 taps over 2 components, L limbs, N coefficients, bands."""
    import oracle
    geo = oracle.geometry(wl.N, *shape)
    Cin, Cout, k = shape[0], shape[1], shape[4]
    return Cout * Cin * k * k * 2 * wl.L * wl.N * geo.bands


def oracle_sample(wl, seed, budget_s):
    """Time Algorithm 1 (oracle route O2, OpenMP over output channels) on a
    bounded sample of (layer, output channel) jobs of one image: passes over
    the layers, each taking the next min(cores, Cout) output channels of every
    layer, until `budget_s` is spent; a workload that finishes well within
    the budget is run again whole.  The inner loop is the same for every
    multiply-add, so the whole workload's time follows from the measured
    multiply-add rate.  Returns (extrapolated seconds per step, seconds spent,
    sample description)."""
    import oracle
    primes = oracle.find_primes(wl.N, wl.L)
    threads = oracle.num_threads()
    spent, done, chans, rounds = 0.0, 0, 0, 0
    inputs, layers_seen = {}, set()
    while True:
        whole = True  # every job of the workload ran in this round
        for p in range(max(sh[1] for sh in wl.layers)):
            progressed = False
            for li, shape in enumerate(wl.layers):
                Cin, Cout, H, W, k, s, pd = shape
                n = min(threads, Cout)
                c0 = p * n
                if c0 >= Cout:
                    continue
                c1 = min(Cout, c0 + n)
                job = o2_macs(wl, shape) * (c1 - c0) // Cout
                if done and spent + job / (done / spent) > budget_s:
                    whole = False
                    continue
                if li not in inputs:
                    geo = oracle.geometry(wl.N, *shape)
                    inputs[li] = (geo, synth.weights(seed, (Cout, Cin, k, k), li),
                                  synth.raw_ciphertexts(seed, primes, (geo.n_in, 2, wl.L, wl.N), li))
                geo, w, ct = inputs[li]
                t0 = time.perf_counter()
                oracle.conv_alg1(ct, w, geo, primes, c0, c1)
                spent += time.perf_counter() - t0
                done += job
                chans += c1 - c0
                layers_seen.add(li)
                progressed = True
            if not progressed:
                break
        rounds += 1
        if not whole or spent * (rounds + 1) / rounds > budget_s:
            break
    rate = done / spent
    total = sum(o2_macs(wl, sh) for sh in wl.layers) * wl.B
    runs = f", the whole workload {rounds} times" if rounds > 1 else ""
    desc = (f"Algorithm 1 (oracle O2, OpenMP over output channels, {threads} threads) on {chans} output channels "
            f"from {len(layers_seen)} of {len(wl.layers)} layers of one image{runs} ({spent:.1f} s, "
            f"{rate / 1e9:.2f} G multiply-adds/s), extrapolated by multiply-add count to all channels, layers and "
            f"B={wl.B}")
    return total / rate, spent, desc


def cpu_baseline(wl, seed, budget_s=15.0):
    import oracle
    est, spent, desc = oracle_sample(wl, seed, budget_s)
    n_layers = len(wl.layers) * wl.B
    return {"value": n_layers / est, "unit": "layers/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": desc}


# ---------------------------------------------------------------------------
# x^2 + x activation protocol, server side (Sec. 5.2)
# ---------------------------------------------------------------------------
X2X_B = 16


def x2x_shapes():
    """The activation layers of ResNet-18 CIFAR: every conv input but the
    stem's (the image) is an x^2 + x output, one activation ciphertext per
    packed input ciphertext of that conv."""
    wl = WORKLOADS["resnet18"]
    return wl, wl.layers[1:]


def x2x_sample(seed, budget_s):
    """Oracle server rounds 1 and 2 (Sec. 5.2) on single ciphertexts at N=8192,
    L=3 until `budget_s` is spent.  Returns (seconds per ciphertext, sample)."""
    import oracle
    wl, _ = x2x_shapes()
    N, L = wl.N, wl.L
    primes = oracle.find_primes(N, L)
    spent, done = 0.0, 0
    while spent < budget_s or done == 0:
        ct = synth.raw_ciphertexts(seed, primes, (1, 2, L, N), done, 1)
        cy = synth.raw_ciphertexts(seed, primes, (1, 2, L, N), done, 2)
        r, v = synth.masks(seed, (1, N), T_PLAIN, done, 1), synth.masks(seed, (1, N), T_PLAIN, done, 2)
        t0 = time.perf_counter()
        oracle.x2x_server_round1(ct, r, v, primes)
        oracle.x2x_server_round2(ct, cy, r, v, primes)
        spent += time.perf_counter() - t0
        done += 1
    desc = (f"oracle rounds 1 and 2 (schoolbook PMult, O(N^2) batch encoding) on {done} activation ciphertexts "
            f"at N={N}, L={L} ({spent:.1f} s), scaled by ciphertext count")
    return spent / done, desc


def run_reference(args, wl, rank, world):
    if rank != 0:
        return 0
    if args.config == "x2x":
        return run_reference_x2x(args)
    import oracle
    threads = oracle.num_threads()
    budget = max(0.5, min(8.0, 90.0 / max(1, args.steps)))  # the whole run stays within a few minutes
    for _ in range(args.warmup):
        oracle_sample(wl, args.seed, budget / 4)
    ests, desc = [], ""
    for _ in range(args.steps):
        est, sp, desc = oracle_sample(wl, args.seed, budget)
        ests.append(est)
    n_layers = len(wl.layers) * wl.B
    est_step = sum(ests) / len(ests)
    value = n_layers / est_step
    print(json.dumps({
        "impl": "reference", "metric": "encrypted conv layers/s", "value": value, "unit": "layers/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": est_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": wl.name, "layers": len(wl.layers), "batch": wl.B, "N": wl.N, "L": wl.L,
                   "t": T_PLAIN},
        "cpu_baseline": {"value": value, "unit": "layers/s", "cores": threads, "kind": "oracle",
                         "sample": "each step: " + desc},
        "e2e": {"value": value, "unit": "layers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def run_reference_x2x(args):
    import oracle
    wl, shapes = x2x_shapes()
    geos = [oracle.geometry(wl.N, *sh) for sh in shapes]
    n = X2X_B * sum(g.n_in for g in geos)
    acts = X2X_B * sum(sh[0] * sh[2] * sh[3] for sh in shapes)
    for _ in range(args.warmup):
        x2x_sample(args.seed, 0.0)
    per_ct, desc = [], ""
    for _ in range(args.steps):
        sec, desc = x2x_sample(args.seed, 6.0)
        per_ct.append(sec)
    step_s = n * sum(per_ct) / len(per_ct)
    value = acts / step_s
    print(json.dumps({
        "impl": "reference", "metric": "x^2+x activations/s (server rounds 1+2)", "value": value,
        "unit": "activations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"x^2+x layers of ResNet-18 CIFAR, B={X2X_B}", "ciphertexts": n, "activations": acts,
                   "N": wl.N, "L": wl.L, "t": T_PLAIN},
        "cpu_baseline": {"value": value, "unit": "activations/s", "cores": 1, "kind": "oracle",
                         "sample": "each step: " + desc},
        "e2e": {"value": value, "unit": "activations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def gpu_uuid(device_index):
    """'GPU-<uuid>' of a CUDA device as NVML and nvidia-smi name it, or None."""
    try:
        import torch
        u = getattr(torch.cuda.get_device_properties(device_index), "uuid", None)
        if u is None:
            return None
        u = str(u)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


class NvmlClock:
    """SM clock and clock-event reasons of one GPU, read through NVML (the
    driver's management library; read-only queries, nothing is set)."""
    # clock-event reason bits of nvmlDeviceGetCurrentClocksEventReasons
    REASONS = ((0x4, "sw_power_cap"), (0x8, "hw_slowdown"), (0x20, "sw_thermal_slowdown"),
               (0x40, "hw_thermal_slowdown"))

    def __init__(self, index, uuid=None):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        # by UUID when known (NVML numbers every GPU of the machine, whatever
        # CUDA_VISIBLE_DEVICES selects), else by index
        if not (uuid and self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) == 0) and \
                self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        self.max_mhz = float(mx.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0 \
            else None

    def read(self):
        mhz, bits = self.ct.c_uint(), self.ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, self.ct.byref(mhz)) != 0:  # NVML_CLOCK_SM
            return None
        if self.reasons_fn(self.h, self.ct.byref(bits)) != 0:
            return None
        return float(mhz.value), int(bits.value)


class ClockSampler:
    """nvidia-smi samples every 50 ms over the whole run, plus NVML reads
    every ~0.2 ms inside the timed region (poll_until), which short timed
    regions need; the summary uses the timed-region reads when there are any."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        uuid = gpu_uuid(device_index)
        self.dev = uuid or device_index  # nvidia-smi --id takes either
        self.proc = None
        self.samples = []
        self.win = []
        try:
            self.nvml = NvmlClock(device_index, uuid)
        except Exception:
            self.nvml = None

    def poll_until(self, ev):
        """Read the clocks until CUDA event `ev` completes; the timed steps
        are already queued, so the GPU is busy meanwhile."""
        if self.nvml is None:
            return
        while True:
            r = self.nvml.read()
            if r is not None:
                self.win.append(r)
            if ev.query():
                return
            time.sleep(0.0002)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                self.samples.append({"sm": float(f[1]), "max": float(f[2]), "util": float(f[4]),
                                     "hw": f[6], "hwt": f[7], "swt": f[8], "pcap": f[9]})
            except ValueError:
                pass

    def summary(self):
        if self.win:
            reasons = [name for bit, name in NvmlClock.REASONS if any(b & bit for _, b in self.win)]
            out = {"sm_mhz": statistics.median(m for m, _ in self.win), "sm_max_mhz": self.nvml.max_mhz,
                   "reasons": reasons, "samples_timed_region": len(self.win), "source": "nvml"}
            if self.samples:
                out["nvidia_smi"] = self._smi_summary()
            return out
        return self._smi_summary()

    def _smi_summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        load = [s for s in self.samples if s["util"] > 0] or self.samples
        reasons = []
        for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                          ("pcap", "sw_power_cap")):
            if any(s[key].lower() == "active" for s in load):
                reasons.append(name)
        return {"sm_mhz": statistics.median(s["sm"] for s in load), "sm_max_mhz": max(s["max"] for s in load),
                "reasons": reasons, "samples_under_load": len(load)}


def share_tc_workspace(ctx, layers, B):
    """One tensor-core workspace, of the largest layer's size, for all the
    given layers: they run one after another on one stream, and a workspace
    larger than a layer needs is valid for it."""
    if layers:
        ws = ctx.tc_workspace(max((lay["g"] for lay in layers), key=lambda g: ctx.tc_workspace_bytes(g, B)), B)
        for lay in layers:
            lay["ws"] = ws


def run_gpu(args, wl, rank, world, local_rank, emit=True):
    import torch
    import torch.distributed as dist

    from paper_2401_16732_gb300 import flashgpu
    from paper_2401_16732_gb300.dist import max_over_ranks, whole_job_rate

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    N, L, B = wl.N, wl.L, wl.B
    ctx = flashgpu.Context(N, L, T_PLAIN)
    stream = torch.cuda.Stream(device=dev)
    seed = args.seed + 1000 * rank

    def to_dev(a, dt=torch.int32):
        a = np.ascontiguousarray(a)
        if a.dtype == np.uint32:
            a = a.view(np.int32)
        return torch.from_numpy(a).to(dt).to(dev)

    # ---- setup (untimed): weights, fresh encryptions, masks, buffers ----
    s = synth.secret_key(seed, N)
    sk = ctx.keygen(to_dev(s, torch.int8))
    layers = []
    for li, shape in enumerate(wl.layers):
        g = ctx.geom(*shape)
        w = synth.weights(seed, (g.Cout, g.Cin, g.k, g.k), li)
        x = synth.activations(seed, (B, g.Cin, g.H, g.W), li)
        a = synth.device_uniform_residues(seed, ctx.primes, (B, g.n_in, L, N), li, device=dev)
        e = synth.device_cbd_noise(seed, (B, g.n_in, N), li, device=dev)
        w_dev = to_dev(w, torch.int8)
        w_hat = ctx.encode_weights(g, w_dev) if args.form in ("ntt", "tc", "auto") else None
        if args.form == "tc":  # the tensor-core form reads the weights in slot groups of 8
            w_hat = ctx.tc_weights(g, w_hat)
        lay = {"g": g, "w": w_dev, "w_hat": w_hat,
               "ct": ctx.encrypt(sk, g, to_dev(x), a, e),
               "r": synth.device_masks(seed, (B, g.n_out, N), T_PLAIN, li, device=dev),
               "out": torch.empty((B, g.n_out, 2, L, N), dtype=torch.int32, device=dev)}
        lay["ct_in"] = lay["ct"]
        lay["form"] = "tc" if args.form == "tc" else "plain"
        del a, e
        layers.append(lay)
    tuning = {}
    if args.form == "auto":
        # per layer the faster of the plain fused form and the tensor-core
        # form (layers that choose the latter keep only their re-laid weights)
        from paper_2401_16732_gb300.autotune import tune_forms
        tuning["forms"] = tune_forms(ctx, layers, stream=stream, cache=None)
        share_tc_workspace(ctx, [lay for lay in layers if lay["form"] == "tc"], B)
    plain_layers = [lay for lay in layers if lay["form"] == "plain"]
    tc_layers = [lay for lay in layers if lay["form"] == "tc"]
    arr = ws = None
    if args.form == "ntt" or (args.form == "auto" and plain_layers):
        arr = ctx.stack_layers([{"g": lay["g"], "w_hat": lay["w_hat"], "ct_in": lay["ct"], "r": lay["r"],
                                 "out": lay["out"]} for lay in plain_layers])
        ws = ctx.stack_workspace(arr)
    torch.cuda.synchronize()
    if args.form == "auto" and arr is None:
        tuned = {"kernel": "tc", "ms": None}
    elif args.form in ("direct", "otf", "tc"):
        tuned = {"kernel": args.form, "ms": None}
        if args.form == "tc":
            share_tc_workspace(ctx, layers, B)
        elif args.form == "otf":
            for lay in layers:
                lay["ws"] = ctx.workspace(lay["g"], B)
    elif args.stack_kernel == "auto":
        from paper_2401_16732_gb300.autotune import tune_stack
        tuned = tune_stack(ctx, [{"g": lay["g"], "ct_in": lay["ct"], "r": lay["r"]} for lay in layers], arr, ws,
                           stream=stream, cache=None, graph=True)  # the timed step is one graph replay
    else:
        ctx.stack_kernel = {"per_layer": flashgpu.FL_STACK_PER_LAYER, "persistent": flashgpu.FL_STACK_PERSISTENT,
                            "queue": flashgpu.FL_STACK_QUEUE}[args.stack_kernel]
        tuned = {"kernel": args.stack_kernel, "ms": None}

    def set_tile(lay):
        # the tensor-core tile the autotuner chose for this layer (else the
        # context's): the call reads it when it launches, and a graph
        # captured from the step keeps each layer's
        if "tc_tile" in lay:
            ctx.tc_tile = lay["tc_tile"]

    def step(events=None, outs=None, arr_=None):
        # forward NTT of every layer's inputs (one launch), then the
        # contraction + inverse NTT + mask kernel(s) over all layers; `outs`
        # / `arr_` select another set of output buffers
        outs = outs or [lay["out"] for lay in layers]
        arr_ = arr if arr_ is None else arr_
        if args.form == "auto":
            # the plain layers as one stack call, then the tensor-core layers;
            # with `events` ({"stack": 3 events, "tc": 4 per layer}) the
            # stages are bracketed and called separately
            if arr_ is not None:
                if events is None:
                    ctx.he_conv2d_stack(arr_, ws, stream=stream, stage="all")
                else:
                    events["stack"][0].record(stream)
                    ctx.he_conv2d_stack(arr_, ws, stream=stream, stage="ntt")
                    events["stack"][1].record(stream)
                    ctx.he_conv2d_stack(arr_, ws, stream=stream, stage="run")
                    events["stack"][2].record(stream)
            k = 0
            for lay, o in zip(layers, outs):
                if lay["form"] != "tc":
                    continue
                set_tile(lay)
                if events is None:
                    ctx.he_conv2d_tc(lay["g"], lay["w_tc"], lay["ct"], out=o, workspace=lay["ws"], r=lay["r"],
                                     stream=stream)
                    continue
                ev = events["tc"][k]
                k += 1
                ev[0].record(stream)
                ctx.he_conv2d_ntt_inputs(lay["g"], lay["ct"], lay["ws"], stream=stream)
                ev[1].record(stream)
                ctx.he_conv2d_tc_from_ntt(lay["g"], B, lay["w_tc"], lay["ws"], stream=stream)
                ev[2].record(stream)
                ctx.intt_mask_outputs(lay["g"], lay["ws"], o, r=lay["r"], stream=stream)
                ev[3].record(stream)
            return
        if events is not None and args.form != "tc":
            events[0].record(stream)
        if args.form == "direct":
            # the paper's DRot + CMult form on the GPU: one launch per layer, no NTT
            if events is not None:
                events[1].record(stream)
            for lay, o in zip(layers, outs):
                ctx.he_conv2d_direct(lay["g"], lay["w"], lay["ct"], out=o, r=lay["r"], stream=stream)
            if events is not None:
                events[2].record(stream)
            return
        if args.form == "tc":
            # per layer: input NTT, tensor-core contraction into the
            # workspace's scratch (NTT domain, slot-tiled), inverse NTT + mask
            # of every output row into the outputs; with `events`, each stage
            # of each layer is bracketed
            # (events[k] = 4 events per layer) and the stages are separate calls
            for k, (lay, o) in enumerate(zip(layers, outs)):
                set_tile(lay)
                if events is None:
                    ctx.he_conv2d_tc(lay["g"], lay["w_hat"], lay["ct"], out=o, workspace=lay["ws"], r=lay["r"],
                                     stream=stream)
                    continue
                ev = events[k]
                ev[0].record(stream)
                ctx.he_conv2d_ntt_inputs(lay["g"], lay["ct"], lay["ws"], stream=stream)
                ev[1].record(stream)
                ctx.he_conv2d_tc_from_ntt(lay["g"], B, lay["w_hat"], lay["ws"], stream=stream)
                ev[2].record(stream)
                ctx.intt_mask_outputs(lay["g"], lay["ws"], o, r=lay["r"], stream=stream)
                ev[3].record(stream)
            return
        if args.form == "otf":
            # input NTT + on-the-fly-weight kernel per layer (the two stages are
            # not separated here: events[1] == events[0])
            if events is not None:
                events[1].record(stream)
            for lay, o in zip(layers, outs):
                ctx.he_conv2d_otf(lay["g"], lay["w"], lay["ct"], out=o, workspace=lay["ws"], r=lay["r"],
                                  stream=stream)
            if events is not None:
                events[2].record(stream)
            return
        if events is None:
            # one call: the conv kernel can follow the input NTT as a
            # programmatic dependent launch
            ctx.he_conv2d_stack(arr_, ws, stream=stream, stage="all")
            return
        ctx.he_conv2d_stack(arr_, ws, stream=stream, stage="ntt")
        events[1].record(stream)
        ctx.he_conv2d_stack(arr_, ws, stream=stream, stage="run")
        events[2].record(stream)

    if args.form in ("ntt", "tc", "auto") and not args.no_tune:
        # pass plan of the input NTTs (and of the tensor-core form's
        # inverse-NTT rows), tensor-core tile: each timed on the whole step
        from paper_2401_16732_gb300.autotune import tune_ntt_plan, tune_tc_tiles
        tuning["ntt_plan"] = tune_ntt_plan(ctx, lambda st: step(), stream=stream)
        if args.form == "tc":  # per layer (the auto form chose its layers' tiles with their forms)
            tile0 = str(ctx.tc_tile)  # the context's (default) tile
            tiles = tune_tc_tiles(ctx, layers, w_key="w_hat", stream=stream)
            tuning["tc_tile"] = {"per_layer": [t["choice"] for t in tiles],
                                 "ms_saved_vs_context_tile": round(sum(t["ms"][tile0] - t["ms"][str(t["choice"])]
                                                                       for t in tiles), 4)}

    # capture one step in a CUDA graph (40 launches for ResNet-18)
    with torch.cuda.stream(stream):
        step()
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step()
    stack_launches = {"persistent": 2, "queue": 2}.get(tuned["kernel"], 1 + len(plain_layers))
    launches_per_step = {"direct": len(layers), "otf": 2 * len(layers), "tc": 4 * len(layers)}.get(
        tuned["kernel"], stack_launches)
    if args.form == "auto":  # stack launches + input NTT, input layout, contraction, inverse NTT per TC layer
        launches_per_step = (stack_launches if plain_layers else 0) + 4 * len(tc_layers)

    def barrier():
        if world > 1:
            dist.barrier()

    def replay():
        # CUDAGraph.replay() launches on the current stream
        with torch.cuda.stream(stream):
            graph.replay()

    clocks = ClockSampler(local_rank)
    clocks.start()
    for _ in range(args.warmup):
        replay()
    stream.synchronize()
    barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        replay()
    t_end.record(stream)
    clocks.poll_until(t_end)
    t_end.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(t_start.elapsed_time(t_end), dev)

    # ---- per-kernel durations (eager launches queued behind a GPU sleep so
    # that event timestamps bracket the kernels, not host launch latency) ----
    kern = {"ntt": 0.0, "conv": 0.0, "tc": 0.0, "intt": 0.0}
    nrep = max(1, min(args.steps, 5))
    for _ in range(nrep):
        with torch.cuda.stream(stream):
            torch.cuda._sleep(2_000_000)
        if args.form in ("tc", "auto"):
            tcev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in tc_layers]
            sev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            step(tcev if args.form == "tc" else {"stack": sev, "tc": tcev})
            stream.synchronize()
            for ev in tcev:
                kern["ntt"] += ev[0].elapsed_time(ev[1]) / nrep
                kern["tc"] += ev[1].elapsed_time(ev[2]) / nrep
                kern["intt"] += ev[2].elapsed_time(ev[3]) / nrep
            if args.form == "auto" and arr is not None:
                kern["ntt"] += sev[0].elapsed_time(sev[1]) / nrep
                kern["stack"] = kern.get("stack", 0.0) + sev[1].elapsed_time(sev[2]) / nrep
            kern["conv"] = kern["tc"] + kern["intt"] + kern.get("stack", 0.0)
            continue
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        step(evs)
        stream.synchronize()
        kern["ntt"] += evs[0].elapsed_time(evs[1]) / nrep
        kern["conv"] += evs[1].elapsed_time(evs[2]) / nrep
    if args.form in ("tc", "auto") and ctx.tc_error(stream):
        raise RuntimeError("a bounded wait of the tensor-core contraction ran out")
    err_word = ctx.stack_error(ws, stream=stream) if ws is not None else 0
    if err_word:
        raise RuntimeError(f"persistent kernel reported a timed-out wait (error word {err_word})")

    # ---- end to end: pinned host inputs -> device -> path -> host outputs ----
    e2e = e2e_switched = None
    if not args.skip_e2e:
        # The copies go through the library's C-ABI (fl_copy_to_device,
        # fl_copy_to_host).  Every step copies every layer's input ciphertexts in from pinned
        # host memory and every layer's output ciphertexts back out (one
        # reused host buffer per direction, sized for the largest layer; the
        # bytes moved are those of the whole step).  When a second set of
        # output buffers fits on the device, steps are pipelined the way a
        # server runs them: step k's outputs drain on a copy stream while step
        # k+1's inputs arrive and its kernels run.
        in_words = max(lay["ct"].numel() for lay in layers)
        out_words = max(lay["out"].numel() for lay in layers)
        h_in = torch.empty(in_words, dtype=torch.int32, pin_memory=True)
        h_out = torch.empty(out_words, dtype=torch.int32, pin_memory=True)
        h_in.copy_(max(layers, key=lambda lay: lay["ct"].numel())["ct"].view(-1).cpu())
        h2d = sum(lay["ct"].numel() * 4 for lay in layers)
        d2h = sum(lay["out"].numel() * 4 for lay in layers)
        n_e2e = max(2, min(args.steps, 6 if d2h < 8e9 else 2))
        free, _ = torch.cuda.mem_get_info(dev)
        sets = [([lay["out"] for lay in layers], arr, graph)]
        if free > 1.25 * d2h + (2 << 30):
            outs2 = [torch.empty_like(lay["out"]) for lay in layers]
            arr2 = None
            if arr is not None:
                arr2 = ctx.stack_layers([{"g": lay["g"], "w_hat": lay["w_hat"], "ct_in": lay["ct"], "r": lay["r"],
                                          "out": o} for lay, o in zip(layers, outs2) if lay["form"] == "plain"])
            with torch.cuda.stream(stream):
                step(outs=outs2, arr_=arr2)
            stream.synchronize()
            graph2 = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph2, stream=stream):
                step(outs=outs2, arr_=arr2)
            sets.append((outs2, arr2, graph2))
        copy_stream = torch.cuda.Stream(device=dev)

        def run_e2e(L_out=None):
            # L_out: switch every output to its first L_out primes on the
            # device (BFV modulus switching) before it leaves
            nb = 2 if len(sets) == 2 else 1
            drain = None
            if L_out:
                need = d2h * L_out // L
                free_now, _ = torch.cuda.mem_get_info(dev)
                nb = 2 if free_now > 2 * need + (2 << 30) else 1 if free_now > need + (1 << 30) else 0
                if nb == 0:
                    return None
                drain = [[torch.empty(tuple(o.shape[:-2]) + (L_out, N), dtype=o.dtype, device=dev) for o in sets[0][0]]
                         for _ in range(nb)]
            ev_comp = [torch.cuda.Event() for _ in range(nb)]
            ev_done = [torch.cuda.Event() for _ in range(nb)]
            for e in ev_done:
                e.record(copy_stream)

            def e2e_step(k):
                outs, _, g_ = sets[k % len(sets)]
                di = k % nb
                with torch.cuda.stream(stream):
                    for lay in layers:
                        ctx.copy_to_device(h_in[:lay["ct"].numel()], lay["ct"].view(-1), stream=stream)
                    if not L_out:
                        stream.wait_event(ev_done[di])  # this output set has drained
                    g_.replay()
                    if L_out:
                        stream.wait_event(ev_done[di])
                        for o, d in zip(outs, drain[di]):
                            ctx.mod_switch(o, L_out, out=d, stream=stream)
                    ev_comp[di].record(stream)
                with torch.cuda.stream(copy_stream):
                    copy_stream.wait_event(ev_comp[di])
                    for o in (drain[di] if L_out else outs):
                        ctx.copy_to_host(o.view(-1), h_out[:o.numel()], stream=copy_stream)
                    ev_done[di].record(copy_stream)

            for k in range(2):
                e2e_step(k)
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            for k in range(n_e2e):
                e2e_step(k)
            copy_stream.synchronize()
            stream.synchronize()
            rate, _ = whole_job_rate(B * len(layers) * n_e2e, time.perf_counter() - t0, dev)
            out_bytes = d2h if not L_out else d2h * L_out // L
            return {"value": rate, "unit": "layers/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": out_bytes,
                    "steps": n_e2e, "pipelined": nb == 2, "copies": "fl_copy_to_device / fl_copy_to_host (C-ABI)"}

        e2e = run_e2e()
        if L > 2:
            e2e_switched = run_e2e(2)
        if e2e_switched is not None:
            e2e_switched["note"] = ("outputs switched to their first 2 RNS primes on the device before the copy "
                                    "(BFV modulus switching, an addition to the paper's protocol)")
    clocks.stop()

    if rank != 0:
        return 0
    geoms = [lay["g"] for lay in layers]
    conv_bytes = sum(layer_bytes(g, B, L, N) for g in geoms)
    step_bytes = conv_bytes + sum(ntt_bytes(g, B, L, N) for g in geoms)
    macs = sum(slot_macs(g, B, L, N) for g in geoms)
    hbm, peak_kind = peaks()
    bfly = sum(intt_butterflies(g, B, L, N) for g in geoms)
    kern_s = kern["conv"] * 1e-3
    achieved = conv_bytes / kern_s / 1e9
    achieved_bfly = bfly / kern_s
    ALU_BFLY_PEAK, alu_src = alu_peak()
    hbm_floor, alu_floor = conv_bytes / (hbm * 1e9), bfly / ALU_BFLY_PEAK
    value = world * B * len(layers) * args.steps / (ms * 1e-3)
    kname = {"persistent": "k_stack (persistent, warp-specialised, all layers)",
             "queue": "k_conv_queue (resident CTAs over one queue of all layers' items)"}.get(
        tuned["kernel"], "k_conv_intt (one launch per layer)") + ": contraction + inverse NTT + mask"
    traffic = traffic_of(args.config, tuned["kernel"])
    hbm_line = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": peak_kind, "traffic": traffic,
                "kernel_source_sha256_16": kernel_source_hash(tuned["kernel"])}
    # traffic is the kernel's DRAM bytes, reported whichever roofline binds
    alu_line = {"bound": "alu", "achieved": achieved_bfly / 1e12, "peak": ALU_BFLY_PEAK / 1e12,
                "unit": "T butterflies/s", "frac": achieved_bfly / ALU_BFLY_PEAK, "peak_source": alu_src,
                "traffic": traffic, "kernel_source_sha256_16": kernel_source_hash(tuned["kernel"])}
    main, other = (hbm_line, alu_line) if hbm_floor >= alu_floor else (alu_line, hbm_line)
    roof = dict(main)
    roof.update({"kernel": kname, "kernel_ms_per_step": kern["conv"], "algorithmic_bytes_per_step": conv_bytes,
                 "algorithmic_butterflies_per_step": bfly, "hbm_floor_ms": hbm_floor * 1e3,
                 "alu_floor_ms": alu_floor * 1e3, "other_roofline": other,
                 "ntt_inputs_ms_per_step": kern["ntt"]})
    if tuned["kernel"] == "direct":
        # Cin*k^2 signed 32x32->64-bit multiply-adds per output coefficient,
        # against one such multiply-add per lane per clock on the 16-lane
        # integer multiply pipe of each SM sub-partition
        dmacs = sum(B * g.n_out * 2 * L * N * g.Cin * g.k * g.k for g in geoms)
        rate = dmacs / kern_s
        roof = {"bound": "alu", "achieved": rate / 1e12, "peak": DIRECT_MAC_PEAK / 1e12, "unit": "T MAC/s",
                "frac": rate / DIRECT_MAC_PEAK, "traffic": None,
                "peak_source": "derived: 152 SMs x 4 x 16 integer-multiply lanes x 2.07 GHz, one MAC per lane-clock",
                "kernel": "k_direct (one launch per layer): DRot + CMult, no NTT", "kernel_ms_per_step": kern["conv"],
                "algorithmic_macs_per_step": dmacs}
        kname = roof["kernel"]
    if tuned["kernel"] == "otf":
        # forward NTTs of the rebuilt weight polynomials + the output INTTs;
        # HBM traffic without the weight stream
        wbfly = sum(B * g.bands * g.Cout * L * g.G * (N // 2) * (N.bit_length() - 1) for g in geoms)
        rate = (bfly + wbfly) / kern_s
        obytes = sum(layer_bytes(g, B, L, N) - L * g.Cout * g.G * N * 4 + ntt_bytes(g, B, L, N) for g in geoms)
        roof = {"bound": "alu", "achieved": rate / 1e12, "peak": ALU_BFLY_PEAK / 1e12, "unit": "T butterflies/s",
                "frac": rate / ALU_BFLY_PEAK, "traffic": None, "peak_source": alu_src,
                "kernel": "k_ntt_fwd + k_conv_otf per layer: weight polynomials rebuilt and transformed in shared memory",
                "kernel_ms_per_step": kern["conv"], "algorithmic_butterflies_per_step": bfly + wbfly,
                "weight_ntt_butterflies_per_step": wbfly, "hbm_bytes_per_step": obytes,
                "encoded_weight_bytes_avoided": sum(L * g.Cout * g.G * N * 4 for g in geoms)}
        kname = roof["kernel"]
    if tuned["kernel"] == "tc":
        # two kernels per layer after the input NTT: the tensor-core
        # contraction (NTT-domain outputs to the scratch in HBM) and the inverse NTT +
        # mask of every output row; each is timed with its own events
        tpk, tpk_src = tensor_peak()
        digit_flops = 2 * 16 * macs  # 16 fp16 digit products per modular multiply-add
        tc_bytes = sum(L * g.Cout * g.G * N * 4 + B * g.n_in * 2 * L * N * 4 + B * g.n_out * 2 * L * N * 4
                       for g in geoms)  # weights + NTT inputs read, NTT-domain outputs written
        intt_bytes = sum(2 * B * g.n_out * 2 * L * N * 4 + B * g.n_out * N * 4 for g in geoms)
        tc_s, intt_s = kern["tc"] * 1e-3, kern["intt"] * 1e-3
        tc_hbm = {"bound": "hbm", "achieved": tc_bytes / tc_s / 1e9, "peak": hbm, "unit": "GB/s",
                  "frac": tc_bytes / tc_s / 1e9 / hbm, "peak_source": peak_kind}
        tc_tensor = {"bound": "tensor", "achieved": digit_flops / tc_s / 1e12, "peak": tpk / 1e12, "unit": "TFLOP/s",
                     "frac": digit_flops / tc_s / tpk, "peak_source": tpk_src}
        tc_main, tc_other = (tc_hbm, tc_tensor) if tc_bytes / (hbm * 1e9) >= digit_flops / tpk else (tc_tensor, tc_hbm)
        tc_line = dict(tc_main, kernel="k_conv_tc (tcgen05 kind::f16 digit products, tensor-memory accumulators)",
                       kernel_ms_per_step=kern["tc"], algorithmic_bytes_per_step=tc_bytes,
                       algorithmic_digit_flops_per_step=digit_flops, other_roofline=tc_other,
                       traffic=traffic_of(args.config, "tc"), kernel_source_sha256_16=kernel_source_hash("tc"))
        intt_hbm = {"bound": "hbm", "achieved": intt_bytes / intt_s / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": intt_bytes / intt_s / 1e9 / hbm, "peak_source": peak_kind}
        intt_alu = dict(alu_line, achieved=bfly / intt_s / 1e12, frac=bfly / intt_s / ALU_BFLY_PEAK)
        i_main, i_other = (intt_hbm, intt_alu) if intt_bytes / (hbm * 1e9) >= bfly / ALU_BFLY_PEAK else (intt_alu, intt_hbm)
        intt_line = dict(i_main, kernel="k_intt_mask_rows (inverse NTT + mask of every output row, gathered from the scratch)",
                         kernel_ms_per_step=kern["intt"], algorithmic_bytes_per_step=intt_bytes,
                         algorithmic_butterflies_per_step=bfly, other_roofline=i_other,
                         traffic=traffic_of(args.config, "intt_rows"),
                         kernel_source_sha256_16=kernel_source_hash("intt_rows"))
        roof, other_k = (tc_line, intt_line) if kern["tc"] >= kern["intt"] else (intt_line, tc_line)
        roof = dict(roof, other_kernels=[other_k], ntt_inputs_ms_per_step=kern["ntt"])
        kname = roof["kernel"]
    if args.form == "auto":
        # the step's kernels: the plain layers' stack (contraction + INTT +
        # mask, fused) and the tensor-core layers' contraction and
        # inverse-NTT rows; against the ALU bound on every output INTT
        ks = (kern.get("stack", 0.0) + kern["tc"] + kern["intt"]) * 1e-3
        roof = dict(alu_line, achieved=bfly / ks / 1e12, frac=bfly / ks / ALU_BFLY_PEAK,
                    kernel=f"{len(plain_layers)} layers plain (stack kernel {tuned['kernel']}), "
                           f"{len(tc_layers)} layers tensor-core (k_conv_tc + k_intt_mask_rows)",
                    kernel_ms_per_step={"plain_stack": kern.get("stack", 0.0), "k_conv_tc": kern["tc"],
                                        "k_intt_mask_rows": kern["intt"], "input_ntt": kern["ntt"]},
                    algorithmic_butterflies_per_step=bfly, other_roofline=dict(hbm_line, achieved=conv_bytes / ks / 1e9,
                                                                             frac=conv_bytes / ks / 1e9 / hbm))
        kname = roof["kernel"]
    line = {
        "metric": "encrypted conv layers/s", "value": value, "unit": "layers/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": wl.name, "layers": len(layers), "batch": B, "N": N, "L": L, "t": T_PLAIN,
                   "l2": f"no flush: {step_bytes / 1e9:.2f} GB of algorithmic traffic per step > {L2_BYTES / 1e6:.0f} MB L2",
                   "graph": "one CUDA graph per step: input NTT of all layers + the contraction/INTT/mask kernel(s)",
                   "stack_kernel": tuned["kernel"], "autotune_ms": tuned["ms"], "form": args.form,
                   "ntt_plan": ctx.ntt_plan,
                   "tc_tile": [lay["tc_tile"] for lay in tc_layers if "tc_tile" in lay] or ctx.tc_tile,
                   "tuning": tuning},
        "slot_mac_per_s": world * macs * args.steps / (ms * 1e-3),
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
        "clocks": clocks.summary(),
    }
    if e2e is not None:
        line["e2e"] = e2e
    if e2e_switched is not None:
        line["e2e_switched"] = e2e_switched
    if world == 1 and not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline(wl, args.seed)
    if not emit:
        return line
    if world == 1 and args.config == "resnet18" and args.form == "ntt" and not args.no_batched:
        del layers, graph, arr, ws
        line["batched"] = run_batched(args, local_rank, {args.config: line["value"]})
    print(json.dumps(line), flush=True)
    return 0


# (the default workload's tensor-core form too, beside the line's plain form)
BATCHED = (("resnet18", "tc"),
           ("resnet18-b64", "ntt"), ("resnet18-b64", "tc"), ("resnet18-b64", "auto"),
           ("resnet50-b8", "ntt"), ("resnet50-b8", "tc"), ("resnet50-b8", "auto"))


def run_batched(args, local_rank, plain_values=None):
    """The batched stacks (ResNet-18 CIFAR B=64, ResNet-50 ImageNet B=8) in the
    plain form, the tensor-core form and the autotuned per-layer mix, and the
    default workload (ResNet-18 CIFAR B=1) in the tensor-core form, each
    measured as the default line is (one CUDA graph per step, device-side
    events, clocks during the timed region), at up to 5 timed steps, without
    the end-to-end and CPU legs; plain_values gives the plain form's value of
    a config measured elsewhere (the default line's own workload).  Returns
    {config: {form: summary}}."""
    import argparse as _ap
    import gc

    import torch
    out = {}
    for cfg, form in BATCHED:
        a = _ap.Namespace(**vars(args))
        a.config, a.form, a.steps, a.skip_e2e, a.skip_cpu, a.no_batched = cfg, form, min(args.steps, 5), True, True, True
        gc.collect()  # the previous workload's buffers (also after a failed one)
        torch.cuda.empty_cache()
        try:
            ln = run_gpu(a, WORKLOADS[cfg], 0, 1, local_rank, emit=False)
        except Exception as exc:  # report, keep the headline line
            out.setdefault(cfg, {})[form] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            continue
        r = ln["roofline"]
        summ = {"value": ln["value"], "unit": ln["unit"], "ms_per_step": ln["ms_per_step"], "steps": ln["steps"],
                "gpu_launches": ln["gpu_launches"], "stack_kernel": ln["config"]["stack_kernel"],
                "ntt_plan": ln["config"]["ntt_plan"], "tc_tile": ln["config"]["tc_tile"], "clocks": ln["clocks"],
                "roofline": {k: r[k] for k in ("bound", "achieved", "peak", "unit", "frac", "kernel",
                                               "kernel_ms_per_step", "traffic", "peak_source") if k in r}}
        if "other_roofline" in r:
            summ["roofline"]["other_roofline"] = {k: r["other_roofline"][k] for k in ("bound", "achieved", "unit",
                                                                                      "frac")}
        if "other_kernels" in r:
            summ["roofline"]["other_kernels"] = [{k: o[k] for k in ("kernel", "bound", "achieved", "unit", "frac",
                                                                  "kernel_ms_per_step") if k in o}
                                                 for o in r["other_kernels"]]
        tun = ln["config"].get("tuning") or {}
        if "forms" in tun:
            summ["forms"] = [f["form"] for f in tun["forms"]]
            summ["form_ms"] = [f["ms"] for f in tun["forms"]]
        if "forms" in tun:
            summ["form_tiles"] = [f.get("tc_tile") for f in tun["forms"]]
        # whole-step choices carry their timings under "ms"; the per-layer
        # tile choice of the tensor-core form is summarised as it is
        summ["tuning_ms"] = {k: v.get("ms", v) for k, v in tun.items() if k != "forms"}
        out.setdefault(cfg, {})[form] = summ
        del ln
    torch.cuda.empty_cache()
    for cfg, forms in out.items():
        plain = forms["ntt"].get("value") if "ntt" in forms else (plain_values or {}).get(cfg)
        if plain:
            for f, summ in forms.items():
                if f != "ntt" and "value" in summ:
                    summ["speedup_over_plain"] = summ["value"] / plain
    return out


def run_x2x(args, rank, world, local_rank):
    """Server rounds 1 and 2 of the x^2 + x protocol over every activation
    ciphertext of ResNet-18 CIFAR, B=16 (N=8192, L=3).  The offline step (r, v
    and their encodings) is untimed, as in Sec. 6.3."""
    import torch

    from paper_2401_16732_gb300 import flashgpu
    from paper_2401_16732_gb300.dist import max_over_ranks, whole_job_rate
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl, shapes = x2x_shapes()
    N, L, B = wl.N, wl.L, X2X_B
    ctx = flashgpu.Context(N, L, T_PLAIN)
    geoms = [ctx.geom(*sh) for sh in shapes]
    n = B * sum(g.n_in for g in geoms)
    acts = B * sum(sh[0] * sh[2] * sh[3] for sh in shapes)
    seed = args.seed + 1000 * rank
    stream = torch.cuda.Stream(device=dev)
    prep = ctx.x2x_prepare(synth.device_masks(seed, (n, N), T_PLAIN, 1, device=dev),
                           synth.device_masks(seed, (n, N), T_PLAIN, 2, device=dev))
    ct_z, ct_x, ct_y = (synth.device_uniform_residues(seed, ctx.primes, (n, 2, L, N), k, device=dev)
                        for k in (3, 4, 5))
    out1, out2 = torch.empty_like(ct_z), torch.empty_like(ct_z)
    torch.cuda.synchronize()

    def step(ev=None, o1=None):
        o1 = out1 if o1 is None else o1
        if ev is not None:
            ev[0].record(stream)
        ctx.x2x_round1(prep, ct_z, o1, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        ctx.x2x_round2(prep, ct_x, ct_y, out2, stream=stream)
        if ev is not None:
            ev[2].record(stream)

    clocks = ClockSampler(local_rank)
    clocks.start()
    for _ in range(args.warmup):
        step()
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    clocks.poll_until(t1)
    t1.synchronize()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(t0.elapsed_time(t1), dev)
    k1 = k2 = 0.0
    nrep = max(1, min(args.steps, 5))
    for _ in range(nrep):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        with torch.cuda.stream(stream):
            torch.cuda._sleep(2_000_000)
        step(evs)
        stream.synchronize()
        k1 += evs[0].elapsed_time(evs[1]) / nrep
        k2 += evs[1].elapsed_time(evs[2]) / nrep

    e2e = None
    if not args.skip_e2e:
        # client -> server: <z> (batch), <X>, <Y>; server -> client: round 1's
        # <2rz + v>.  Steps are pipelined: round 1's output of step k drains on
        # a copy stream (two output buffers) while step k+1's inputs arrive.
        h_in = [torch.empty(ct_z.numel(), dtype=torch.int32, pin_memory=True) for _ in range(3)]
        for h, d in zip(h_in, (ct_z, ct_x, ct_y)):
            h.copy_(d.view(-1).cpu())
        h_out = torch.empty(ct_z.numel(), dtype=torch.int32, pin_memory=True)
        o1s = [out1, torch.empty_like(out1)]
        copy_stream = torch.cuda.Stream(device=dev)
        ev_comp = [torch.cuda.Event() for _ in o1s]
        ev_done = [torch.cuda.Event() for _ in o1s]
        for e in ev_done:
            e.record(copy_stream)
        n_e2e = max(2, min(args.steps, 6))

        def e2e_step(k):
            si = k % 2
            with torch.cuda.stream(stream):
                for h, d in zip(h_in, (ct_z, ct_x, ct_y)):
                    ctx.copy_to_device(h, d.view(-1), stream=stream)
                stream.wait_event(ev_done[si])
                step(o1=o1s[si])
                ev_comp[si].record(stream)
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(ev_comp[si])
                ctx.copy_to_host(o1s[si].view(-1), h_out, stream=copy_stream)
                ev_done[si].record(copy_stream)

        e2e_step(0)
        e2e_step(1)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        for k in range(n_e2e):
            e2e_step(k)
        copy_stream.synchronize()
        stream.synchronize()
        rate, _ = whole_job_rate(acts * n_e2e, time.perf_counter() - ts, dev)
        e2e = {"value": rate, "unit": "activations/s", "h2d_bytes_per_step": 3 * ct_z.numel() * 4,
               "d2h_bytes_per_step": out1.numel() * 4, "steps": n_e2e, "pipelined": True}
    clocks.stop()
    if rank != 0:
        return 0
    hbm, peak_kind = peaks()
    logn = N.bit_length() - 1
    bfly1 = n * L * 4 * (N // 2) * logn  # two forward and two inverse NTTs per (ciphertext, limb)
    bytes1 = n * (5 * L + 1) * N * 4     # <z>, NTT(2r), encode(v) in; result out
    bytes2 = n * (6 * L + 1) * N * 4     # <X>, <Y>, r^2 - r + v in; result out
    alu1 = bfly1 / (k1 * 1e-3)
    hbm1, hbm2 = bytes1 / (k1 * 1e-3) / 1e9, bytes2 / (k2 * 1e-3) / 1e9
    ALU_BFLY_PEAK, alu_src = alu_peak()
    roof = {"bound": "alu", "achieved": alu1 / 1e12, "peak": ALU_BFLY_PEAK / 1e12, "unit": "T butterflies/s",
            "frac": alu1 / ALU_BFLY_PEAK, "peak_source": alu_src,
            "traffic": traffic_of("x2x", "round1"),
            "kernel": "k_x2x_round1: forward NTT x2, NTT-domain PMult, inverse NTT x2, + encode(v)",
            "kernel_ms_per_step": k1, "algorithmic_butterflies_per_step": bfly1,
            "hbm_view": {"achieved": hbm1, "peak": hbm, "frac": hbm1 / hbm, "algorithmic_bytes_per_step": bytes1},
            "other_kernels": [{"kernel": "k_x2x_round2: <X> - <Y> + Delta*(r^2 - r + v)", "bound": "hbm",
                               "kernel_ms_per_step": k2, "achieved": hbm2, "peak": hbm, "unit": "GB/s",
                               "frac": hbm2 / hbm, "peak_source": peak_kind, "algorithmic_bytes_per_step": bytes2,
                               "traffic": traffic_of("x2x", "round2")}]}
    line = {
        "metric": "x^2+x activations/s (server rounds 1+2)", "value": world * acts * args.steps / (ms * 1e-3),
        "unit": "activations/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"x^2+x layers of ResNet-18 CIFAR, B={B}", "ciphertexts": n, "activations": acts,
                   "N": N, "L": L, "t": T_PLAIN,
                   "l2": f"no flush: {(bytes1 + bytes2) / 1e9:.2f} GB per step > {L2_BYTES / 1e6:.0f} MB L2"},
        "gpu_launches": 2 * args.steps, "roofline": roof, "clocks": clocks.summary(),
    }
    if e2e is not None:
        line["e2e"] = e2e
    if world == 1 and not args.skip_cpu:
        sec, desc = x2x_sample(args.seed, 10.0)
        line["cpu_baseline"] = {"value": acts / (n * sec), "unit": "activations/s", "cores": 1, "kind": "oracle",
                                "sample": desc}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args, rank, world, local_rank):
    """Serving loop (continuous batching) on ResNet-18 (N=8192) and ResNet-50
    (N=16384) requests: Poisson arrivals at 200 requests/s, 70% / 30%, batch
    size uniform in 1..8.  Reports served layers/s and per-request p50/p99,
    and the same loop at 12 requests/s, below one GPU's capacity."""
    import torch

    from paper_2401_16732_gb300 import serve
    from paper_2401_16732_gb300.workloads import resnet18_cifar, resnet50_imagenet
    torch.cuda.set_device(local_rank)
    models = {"resnet18": serve.ModelSpec("resnet18", 8192, 3, resnet18_cifar()),
              "resnet50": serve.ModelSpec("resnet50", 16384, 4, resnet50_imagenet())}
    from paper_2401_16732_gb300 import flashgpu
    kernel = {"per_layer": flashgpu.FL_STACK_PER_LAYER, "persistent": flashgpu.FL_STACK_PERSISTENT,
              "queue": flashgpu.FL_STACK_QUEUE}["queue" if args.stack_kernel == "auto" else args.stack_kernel]
    srv = serve.Server(models, stack_kernel=kernel)
    mix = {"resnet18": 0.7, "resnet50": 0.3}
    warm = serve.poisson_requests(max(args.warmup, 3), 200.0, mix, seed=args.seed + 100)
    srv.run(warm, realtime=False)
    n = 12 * args.steps
    reqs = serve.poisson_requests(n, 200.0, mix, seed=args.seed)
    keep = {(q.rid, 0) for q in reqs[:4]}
    srv.keep = keep
    srv.layer_images = 0
    torch.cuda.synchronize()
    finished, wall = srv.run(reqs, realtime=True)
    # the same loop below capacity (about half of what one GPU serves), where
    # the latencies are service times rather than queueing
    low_rate = 12.0
    low = serve.poisson_requests(40, low_rate, mix, seed=args.seed + 200)
    for q in low:
        q.rid += 10_000
    srv.keep = set()
    low_done, low_wall = srv.run(low, realtime=True)
    low_stats = serve.latency_stats(low_done)
    low_li = sum(q.B * len(models[q.model].layers) for q in low_done)
    if rank != 0:
        return 0
    stats = serve.latency_stats(finished)
    li = sum(q.B * len(models[q.model].layers) for q in finished)
    offered = sum(q.B * len(models[q.model].layers) for q in reqs) / reqs[-1].arrival
    print(json.dumps({
        "metric": "served encrypted conv layers/s", "value": li / wall, "unit": "layers/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "serving: Poisson 200 req/s, 70% ResNet-18 CIFAR (N=8192, L=3), 30% ResNet-50 "
                               "ImageNet (N=16384, L=4), batch U{1..8}, continuous batching by layer rounds",
                   "requests": n, "admission": "peak live bytes of the request's largest layer",
                   "weights_resident_gib": sum(r.weight_bytes for r in srv.res.values()) / 2 ** 30,
                   "stack_kernel": "queue" if args.stack_kernel == "auto" else args.stack_kernel},
        "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"], "mean_ms": stats.get("mean_ms"),
        "wall_s": wall, "rounds": srv.rounds, "peak_active_requests": srv.peak_active,
        "offered_layers_per_s": offered, "offered_over_served": offered / (li / wall),
        "below_capacity": {"rate_req_s": low_rate, "requests": len(low), "served": len(low_done),
                           "p50_ms": low_stats["p50_ms"], "p99_ms": low_stats["p99_ms"],
                           "mean_ms": low_stats.get("mean_ms"), "layers_per_s": low_li / low_wall},
    }), flush=True)
    return 0


def run_peaks():
    """The measured ceilings (libflpeaks): lazy Gentleman-Sande butterflies/s
    and tcgen05.mma kind::f16 flops/s at M128 K16 and N = 64, 128, 256."""
    import ctypes

    import torch
    torch.cuda.init()
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2401_16732_gb300", "libflpeaks.so"))
    dbl = ctypes.POINTER(ctypes.c_double)
    lib.fl_measure_butterfly_rate.argtypes = [ctypes.c_int, dbl]
    lib.fl_measure_tc_f16_rate.argtypes = [ctypes.c_int, ctypes.c_int, dbl, dbl]
    out = {"device": torch.cuda.get_device_name(0)}
    v = ctypes.c_double()
    rc = lib.fl_measure_butterfly_rate(20000, ctypes.byref(v))
    out["butterflies_per_s"] = v.value if rc == 0 else {"error": rc}
    tc = {}
    for n in (64, 128, 256):
        f, c = ctypes.c_double(), ctypes.c_double()
        rc = lib.fl_measure_tc_f16_rate(n, 20000, ctypes.byref(f), ctypes.byref(c))
        tc[f"M128 N{n} K16"] = ({"tflops": f.value / 1e12, "cycles_per_mma": c.value,
                                 "flop_per_clk_per_sm": 2 * 128 * n * 16 / c.value} if rc == 0 else {"error": rc})
    out["tcgen05_f16"] = tc
    try:  # the SM clock right after the measurements, and its maximum
        nv = NvmlClock(0, gpu_uuid(0))
        out["sm_mhz_after"], out["sm_max_mhz"] = nv.read()[0], nv.max_mhz
    except Exception:
        pass
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="resnet18", choices=sorted(WORKLOADS) + ["serve", "x2x"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--form", default="ntt", choices=["ntt", "direct", "otf", "tc", "auto"],
                    help="ntt: the NTT route with encoded weights (default); direct: the paper's DRot + CMult form "
                         "on the GPU; otf: the NTT route with weights rebuilt on the fly (no encoded weights); "
                         "tc: the NTT route with the tensor-core contraction (tcgen05, not fused with the INTT); "
                         "auto: per layer the faster of the plain and tensor-core forms (autotuned)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default NTT pass plan and tensor-core tile (no autotuning of them)")
    ap.add_argument("--no-batched", action="store_true",
                    help="default workload only: skip the batched-stack measurements added to its line")
    ap.add_argument("--stack-kernel", default="auto", choices=["auto", "per_layer", "persistent", "queue"],
                    help="kernel for the contraction/INTT/mask stage (auto: time both, keep the faster)")
    ap.add_argument("--layers", default=None,
                    help="comma-separated layer indices: run only these layers of the chosen stack (a smaller "
                         "workload, e.g. for a profiler capture)")
    ap.add_argument("--peaks", action="store_true",
                    help="print the measured roofline ceilings of this GPU (butterfly rate, tcgen05 kind::f16 "
                         "MMA rates) as one JSON line and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.peaks:
        return run_peaks()
    if args.config == "serve":
        return run_serve(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
                         int(os.environ.get("LOCAL_RANK", "0")))
    wl = WORKLOADS[args.config] if args.config != "x2x" else None
    if args.layers:
        if wl is None:
            ap.error("--layers selects layers of a convolution stack")
        idx = [int(v) for v in args.layers.split(",")]
        if not idx or any(not 0 <= i < len(wl.layers) for i in idx):
            ap.error(f"--layers: indices in 0..{len(wl.layers) - 1}")
        wl = Workload(f"{wl.name}: layers {args.layers} only", wl.N, wl.L, wl.B, tuple(wl.layers[i] for i in idx))
        args.no_batched = True
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, wl, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        if args.config == "x2x":
            return run_x2x(args, rank, world, local_rank)
        return run_gpu(args, wl, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
