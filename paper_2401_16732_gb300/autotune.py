"""Pick the fastest stack kernel for a workload by timing each on the device.

The choice depends only on the stack's shapes (ring degree, limbs, layer
geometries, batch sizes), so it is cached in a JSON file keyed by them.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import flashgpu

KERNELS = ((flashgpu.FL_STACK_PER_LAYER, "per_layer"), (flashgpu.FL_STACK_PERSISTENT, "persistent"),
           (flashgpu.FL_STACK_QUEUE, "queue"))
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "flashgpu_autotune.json")


def _key(ctx, specs, graph) -> str:
    shapes = [(sp["g"].Cin, sp["g"].Cout, sp["g"].H, sp["g"].W, sp["g"].k, sp["g"].stride, sp["g"].pad,
               int(sp["ct_in"].shape[0]), sp.get("r") is not None) for sp in specs]
    dev = torch.cuda.get_device_name(ctx.device)
    raw = json.dumps([dev, ctx.N, ctx.L, shapes, "graph replays" if graph else "whole stack call"])
    return hashlib.sha256(raw.encode()).hexdigest()[:24]


def _time(ctx, arr, ws, stream, reps, graph):
    """Best of reps+1 timed stack calls (eager), or the mean of 4*reps
    back-to-back replays of the call captured as a CUDA graph."""
    torch.cuda.synchronize()
    if graph:
        # graphs are captured on a side stream (never the default stream)
        st = stream if stream != torch.cuda.default_stream(stream.device) else torch.cuda.Stream(stream.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            ctx.he_conv2d_stack(arr, ws, stream=st, stage="all")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            for _ in range(2):
                g.replay()
            e0.record(st)
            for _ in range(4 * reps):
                g.replay()
            e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / (4 * reps)
    best = None
    for _ in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.he_conv2d_stack(arr, ws, stream=stream, stage="all")
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best


def tune_stack(ctx: flashgpu.Context, specs, arr, ws, stream=None, reps: int = 3, cache: str | None = DEFAULT_CACHE,
               graph: bool = False):
    """Time every stack kernel on the stack `arr` (inputs already in place),
    set the fastest on `ctx` and return {"kernel": name, "ms": {...}}.  Each
    timing covers the whole stack call, input NTT included: how the fused
    kernel follows the NTT (programmatic dependent launch) is part of what
    differs between the kernels.  graph=True times the call the way a caller
    that captures it in a CUDA graph runs it (replays back to back), where
    host launch latency no longer adds to small stacks."""
    stream = stream or torch.cuda.current_stream()
    key = _key(ctx, specs, graph)
    table = {}
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if key in table:
        ctx.stack_kernel = table[key]["kernel_id"]
        return {"kernel": table[key]["kernel"], "ms": table[key]["ms"], "cached": True}
    ctx.he_conv2d_stack(arr, ws, stream=stream, stage="ntt")
    ms = {}
    for kid, name in KERNELS:
        ctx.stack_kernel = kid
        ms[name] = _time(ctx, arr, ws, stream, reps, graph)
        if ctx.stack_error(ws, stream=stream):
            ms[name] = float("inf")
    best = min(ms, key=ms.get)
    kid = dict((n, k) for k, n in KERNELS)[best]
    ctx.stack_kernel = kid
    table[key] = {"kernel": best, "kernel_id": kid, "ms": ms}
    if cache:
        try:
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            with open(cache, "w") as f:
                json.dump(table, f, indent=1)
        except OSError:
            pass
    return {"kernel": best, "ms": ms, "cached": False}
