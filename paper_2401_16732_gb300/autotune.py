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


# ---------------------------------------------------------------------------
# NTT pass plan, tensor-core tile and per-layer form
# ---------------------------------------------------------------------------
def time_call(fn, stream, reps: int = 3, graph: bool = True) -> float:
    """Mean milliseconds of `fn(stream)`: 4*reps back-to-back replays of it
    captured as a CUDA graph (graph=True, after two warm-up replays), else
    the best of reps+1 eager calls."""
    torch.cuda.synchronize()
    st = stream if stream != torch.cuda.default_stream(stream.device) else torch.cuda.Stream(stream.device)
    if graph:
        with torch.cuda.stream(st):
            fn(st)
        st.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            fn(st)
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
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn(st)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best


def _choose(ctx, attr: str, options, fn, stream, reps, graph):
    """Time fn with ctx.<attr> set to every option; keep the fastest set."""
    ms = {}
    for opt in options:
        setattr(ctx, attr, opt)
        ms[str(opt)] = time_call(fn, stream, reps, graph)
    best = min(ms, key=ms.get)
    setattr(ctx, attr, int(best))
    return {"choice": int(best), "ms": ms}


def tune_ntt_plan(ctx: flashgpu.Context, fn, stream=None, reps: int = 3, graph: bool = True):
    """Pick the NTT pass plan (first row pass radix 2^r1) for a workload: fn
    runs the workload's step (its input NTTs, and the inverse-NTT-rows kernel
    of the tensor-core form, use the context's plan)."""
    stream = stream or torch.cuda.current_stream()
    return _choose(ctx, "ntt_plan", flashgpu.NTT_PLANS[ctx.N.bit_length() - 1], fn, stream, reps, graph)


def tune_tc_tile(ctx: flashgpu.Context, fn, stream=None, reps: int = 3, graph: bool = True):
    """Pick the tensor-core tile (slot groups of 4 per CTA) for a workload."""
    stream = stream or torch.cuda.current_stream()
    return _choose(ctx, "tc_tile", flashgpu.TC_TILES, fn, stream, reps, graph)


def _time_tc_tiles(ctx, g, w_tc, lay, workspace, stream, reps, graph, tiles=None):
    """Milliseconds of one layer's he_conv2d_tc under every tensor-core tile
    (the context's tile is restored afterwards): ({tile: ms}, fastest tile)."""
    saved = ctx.tc_tile
    ms = {}
    try:
        for tile in tiles or flashgpu.TC_TILES:
            ctx.tc_tile = tile
            ms[str(tile)] = time_call(lambda st: ctx.he_conv2d_tc(g, w_tc, lay["ct_in"], out=lay["out"],
                                                                  workspace=workspace, r=lay["r"], stream=st),
                                      stream, reps, graph)
    finally:
        ctx.tc_tile = saved
    return ms, int(min(ms, key=ms.get))


def tune_tc_tiles(ctx: flashgpu.Context, layers, w_key: str = "w_tc", stream=None, reps: int = 3,
                  graph: bool = True):
    """Per tensor-core layer, time he_conv2d_tc under every tile and record
    the fastest as the layer's "tc_tile" (a caller sets ctx.tc_tile to it
    before that layer's call).  The best tile depends on the layer: a long
    tile halves the per-CTA set-up, but leaves few CTAs (a partial last wave)
    on layers with few output-channel and column tiles.  `layers` holds dicts
    with g, ct_in, r, out, the weight tiles under `w_key` and optionally
    "ws" (a tensor-core workspace).  Returns [{"choice", "ms"}] per layer."""
    stream = stream or torch.cuda.current_stream()
    out = []
    for lay in layers:
        g, B = lay["g"], int(lay["ct_in"].shape[0])
        wst = lay.get("ws")
        if wst is None:
            wst = ctx.tc_workspace(g, B)
        ms, best = _time_tc_tiles(ctx, g, lay[w_key], lay, wst, stream, reps, graph)
        lay["tc_tile"] = best
        out.append({"choice": best, "ms": ms})
        del wst
    return out


def tune_forms(ctx: flashgpu.Context, layers, stream=None, reps: int = 3, graph: bool = True,
               cache: str | None = DEFAULT_CACHE):
    """Per layer, time the plain fused form (he_conv2d with the mask) against
    the tensor-core form (he_conv2d_tc, under every tensor-core tile) and keep
    the faster.  `layers` holds dicts with g, w_hat, ct_in, r, out; the
    tensor-core weights are built for the timing and kept (as "w_tc") only for
    layers that choose that form, and "w_hat" is dropped from those, so at most
    one extra weight copy is live at a time.  Layers with G above FL_TC_MAX_G
    stay plain.  Returns the list of {"form", "ms": {"plain", "tc"}, "tc_tile"}
    per layer; each layer dict gets "form", and a tensor-core layer its fastest
    tile as "tc_tile"."""
    stream = stream or torch.cuda.current_stream()
    table = {}
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    dev = torch.cuda.get_device_name(ctx.device)
    out = []
    for lay in layers:
        g, B = lay["g"], int(lay["ct_in"].shape[0])
        key = hashlib.sha256(json.dumps([dev, "form, tile per layer", ctx.N, ctx.L, ctx.ntt_plan, B,
                                         (g.Cin, g.Cout, g.H, g.W, g.k, g.stride, g.pad)]).encode()).hexdigest()[:24]
        if g.G > flashgpu.FL_TC_MAX_G:
            res = {"form": "plain", "ms": {"plain": None, "tc": None}, "tc_tile": None}
        elif key in table:
            res = dict(table[key], cached=True)
        else:
            ws = ctx.workspace(g, B)
            wst = ctx.tc_workspace(g, B)
            w_tc = ctx.tc_weights(g, lay["w_hat"])
            tile_ms, tile = _time_tc_tiles(ctx, g, w_tc, lay, wst, stream, reps, graph)
            ms = {"plain": time_call(lambda st: ctx.he_conv2d(g, lay["w_hat"], lay["ct_in"], out=lay["out"],
                                                              workspace=ws, r=lay["r"], stream=st),
                                     stream, reps, graph),
                  "tc": tile_ms[str(tile)]}
            res = {"form": min(ms, key=ms.get), "ms": ms, "tc_tile": tile}
            table[key] = res
            del ws, wst, w_tc
        lay["form"] = res["form"]
        if res["form"] == "tc":
            lay["w_tc"] = ctx.tc_weights(g, lay["w_hat"])
            if res.get("tc_tile"):
                lay["tc_tile"] = res["tc_tile"]
            del lay["w_hat"]
        out.append(res)
    if cache:
        try:
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            with open(cache, "w") as f:
                json.dump(table, f, indent=1)
        except OSError:
            pass
    return out
