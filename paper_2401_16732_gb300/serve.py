"""Serving loop: continuous batching of encrypted inference requests.

Each request is one image batch (B images) through one model's conv stack.
The server keeps every model's encoded weights resident on the device and
runs in rounds: a round takes the next layer of every admitted request and
runs all of them in one stack launch per model (fl_he_conv2d_stack: one NTT
launch over all inputs, then the contraction / inverse NTT / mask kernels),
the models on separate CUDA streams so their work overlaps.  A request that
arrives while others are running joins at the next round as soon as device
memory allows (admission by the request's peak live set: the largest layer's
inputs, NTT workspace, masks and outputs).  Latency is arrival to the round
in which the request's last layer is done (outputs resident, ready to send).

Host-side failure handling (no device fault is involved): a request whose
peak live set exceeds the whole memory budget is rejected at admission
instead of being admitted alone; `cancel(rid)` withdraws a request, pending
or active, before the next round and releases its reservation; a stack
kernel that reports a timed-out wait raises before any later round runs.

Inputs of every (request, layer) are fresh synthetic encryptions drawn on the
device from a seed (request id, layer), so any (request, layer) can be
recomputed by the oracle and results do not depend on which other requests
share a round.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import flashgpu, synth

T_PLAIN = 65537


@dataclass(frozen=True)
class ModelSpec:
    name: str
    N: int
    L: int
    layers: tuple  # (Cin, Cout, H, W, k, stride, pad)
    weight_seed: int = 7


@dataclass
class Request:
    rid: int
    model: str
    B: int
    arrival: float  # seconds after the start of the run
    seed: int = 1
    next_layer: int = 0
    admitted: float | None = None
    done: float | None = None
    error: str | None = None
    outputs: dict = field(default_factory=dict)  # layer -> output tensor, when kept


class _Resident:
    """A model on the device: context, geometries, encoded weights, stream."""

    def __init__(self, spec: ModelSpec, device):
        self.spec = spec
        self.ctx = flashgpu.Context(spec.N, spec.L, T_PLAIN)
        self.geoms = [self.ctx.geom(*sh) for sh in spec.layers]
        self.w = []
        self.w_hat = []
        for li, g in enumerate(self.geoms):
            w = synth.weights(spec.weight_seed, (g.Cout, g.Cin, g.k, g.k), li)
            self.w.append(w)
            self.w_hat.append(self.ctx.encode_weights(g, torch.from_numpy(w).to(device)))
        self.stream = torch.cuda.Stream(device=device)
        self.weight_bytes = sum(t.numel() * 4 for t in self.w_hat)

    def layer_bytes(self, li: int, B: int) -> int:
        g, N, L = self.geoms[li], self.spec.N, self.spec.L
        return 4 * B * N * (g.n_in * 2 * L * 2 + g.n_out * 2 * L + g.n_out)  # inputs, NTT inputs, outputs, masks

    def peak_bytes(self, B: int) -> int:
        return max(self.layer_bytes(li, B) for li in range(len(self.geoms)))


def layer_inputs(req: Request, r: _Resident, li: int, device):
    """The fresh encryption (uniform residues) and masks of one (request, layer)."""
    g, N, L = r.geoms[li], r.spec.N, r.spec.L
    ct = synth.device_uniform_residues(req.seed, r.ctx.primes, (req.B, g.n_in, 2, L, N), req.rid, li,
                                       device=device)
    m = synth.device_masks(req.seed, (req.B, g.n_out, N), T_PLAIN, req.rid, li, device=device)
    return ct, m


class Server:
    def __init__(self, models: dict, device=None, mem_budget: int | None = None, keep_outputs=(),
                 stack_kernel: int | None = None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.res = {name: _Resident(spec, self.device) for name, spec in models.items()}
        if stack_kernel is not None:
            for r in self.res.values():
                r.ctx.stack_kernel = stack_kernel
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            mem_budget = int(free * 0.85)
        self.mem_budget = mem_budget
        self.keep = set(keep_outputs)  # (rid, layer) pairs whose outputs are kept
        self.rounds = 0
        self.layer_images = 0
        self.peak_reserved = 0
        self.peak_active = 0
        self.rejected = []    # requests refused at admission (q.error says why)
        self.cancelled = []   # requests withdrawn by cancel()
        self._cancel = set()

    def cancel(self, rid: int):
        """Withdraw request `rid` before the next round (pending or active)."""
        self._cancel.add(rid)

    # -- one round: the next layer of every active request ----------------
    def _round(self, active):
        launched = []
        for name, r in self.res.items():
            reqs = [q for q in active if q.model == name]
            if not reqs:
                continue
            specs = []
            with torch.cuda.stream(r.stream):
                for q in reqs:
                    li = q.next_layer
                    ct, m = layer_inputs(q, r, li, self.device)
                    g = r.geoms[li]
                    out = torch.empty((q.B, g.n_out, 2, r.spec.L, r.spec.N), dtype=torch.int32, device=self.device)
                    specs.append({"g": g, "w_hat": r.w_hat[li], "ct_in": ct, "r": m, "out": out, "q": q, "li": li})
                for c0 in range(0, len(specs), flashgpu.FL_STACK_MAX_LAYERS):  # at most 64 layers per launch
                    chunk = specs[c0:c0 + flashgpu.FL_STACK_MAX_LAYERS]
                    arr = r.ctx.stack_layers(chunk)
                    ws = r.ctx.stack_workspace(arr)
                    r.ctx.he_conv2d_stack(arr, ws, stream=r.stream)
                    launched.append((r, chunk, arr, ws))
        now_done = []
        for r, specs, arr, ws in launched:
            r.stream.synchronize()
            err = r.ctx.stack_error(ws, stream=r.stream)
            if err:
                raise RuntimeError(f"stack kernel reported error word {err}")
            for sp in specs:
                q, li = sp["q"], sp["li"]
                if (q.rid, li) in self.keep:
                    q.outputs[li] = sp["out"]
                self.layer_images += q.B
                q.next_layer += 1
                if q.next_layer == len(r.geoms):
                    now_done.append(q)
        self.rounds += 1
        return now_done

    def run(self, requests: list[Request], realtime: bool = True, t0: float | None = None, on_round=None):
        """Serve `requests` (sorted by arrival).  With realtime, a request can
        only be admitted once the wall clock has passed its arrival time.
        `on_round(server, finished_so_far)` runs after every round."""
        pending = sorted(requests, key=lambda q: q.arrival)
        active, finished = [], []
        reserved = 0
        start = time.perf_counter() if t0 is None else t0

        def drop_cancelled():
            nonlocal reserved
            for q in [q for q in pending + active if q.rid in self._cancel]:
                if q in active:
                    active.remove(q)
                    reserved -= q.reserved
                else:
                    pending.remove(q)
                q.error = "cancelled"
                self.cancelled.append(q)
            self._cancel.clear()

        while pending or active:
            drop_cancelled()
            now = time.perf_counter() - start
            # admit in arrival order while the memory budget allows
            while pending and (not realtime or pending[0].arrival <= now):
                q = pending[0]
                need = self.res[q.model].peak_bytes(q.B)
                if need > self.mem_budget:
                    pending.pop(0)
                    q.error = f"needs {need} bytes of device memory, above the budget of {self.mem_budget}"
                    self.rejected.append(q)
                    continue
                if reserved + need > self.mem_budget and active:
                    break
                pending.pop(0)
                q.admitted = now
                q.reserved = need
                reserved += need
                active.append(q)
                self.peak_reserved = max(self.peak_reserved, reserved)
                self.peak_active = max(self.peak_active, len(active))
            if not active:
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 0.01)))
                continue
            done = self._round(active)
            now = time.perf_counter() - start
            for q in done:
                q.done = now
                reserved -= q.reserved
                active.remove(q)
                finished.append(q)
            if on_round is not None:
                on_round(self, finished)
        wall = time.perf_counter() - start
        return finished, wall


def poisson_requests(n: int, rate: float, mix: dict, bmax: int = 8, seed: int = 3) -> list[Request]:
    """n requests with exponential inter-arrival times (mean 1/rate), model
    drawn from `mix` (name -> probability), batch size uniform in 1..bmax."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 77])))
    names = list(mix)
    probs = np.array([mix[k] for k in names], dtype=np.float64)
    t, out = 0.0, []
    for rid in range(n):
        t += g.exponential(1.0 / rate)
        out.append(Request(rid=rid, model=names[g.choice(len(names), p=probs / probs.sum())],
                           B=int(g.integers(1, bmax + 1)), arrival=t, seed=seed))
    return out


def latency_stats(finished: list[Request]) -> dict:
    lat = sorted((q.done - q.arrival) * 1e3 for q in finished)
    if not lat:
        return {"p50_ms": None, "p99_ms": None}

    def pct(p):
        k = min(len(lat) - 1, max(0, math.ceil(p / 100 * len(lat)) - 1))
        return lat[k]
    return {"p50_ms": pct(50), "p99_ms": pct(99), "mean_ms": sum(lat) / len(lat), "max_ms": lat[-1]}
