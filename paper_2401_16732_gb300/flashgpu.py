"""Thin Python binding of the flashgpu C-ABI (include/flashgpu.h).

Argument marshalling only: every step of the HE convolution runs in the CUDA
kernels of libflashgpu.so.  Device buffers are torch tensors (ciphertexts as
int32 tensors holding residues below 2^30, i.e. the same bits as uint32);
streams are torch CUDA streams.  There is no CPU path: if the shared library
is missing the import of this module fails.
"""
from __future__ import annotations

import ctypes
import math
import os
import re

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libflashgpu.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "flashgpu.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2401_16732_gb300.build` "
                      "(there is no CPU fallback)")
_lib = ctypes.CDLL(LIB_PATH)

FL_OK, FL_ERR_ARG, FL_ERR_SHAPE, FL_ERR_CUDA, FL_ERR_OOM, FL_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
FL_STACK_PER_LAYER, FL_STACK_PERSISTENT, FL_STACK_QUEUE = 0, 1, 2
FL_NOALLOC_SCRATCH_BYTES = 16 << 20
FL_TC_MAX_G = 64
NTT_PLANS = {11: (3,), 12: (3, 4), 13: (3, 4, 5), 14: (4, 5)}  # available first-pass radix exponents
TC_TILES = (4, 8, 16, 32, 64)
FL_STACK_MAX_LAYERS = 64


class ConvGeom(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "N", "Cin", "Cout", "H", "W", "k", "stride", "pad", "Hp", "Wp", "Ho", "Wo",
        "Rin", "Rout", "bands", "P", "c_n", "G", "n_in", "n_out")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class StackLayer(ctypes.Structure):
    _fields_ = [("geom", ctypes.POINTER(ConvGeom)), ("B", ctypes.c_int32), ("w_hat_dev", ctypes.c_void_p),
                ("ct_in_dev", ctypes.c_void_p), ("r_dev", ctypes.c_void_p), ("ct_out_dev", ctypes.c_void_p)]


_vp, _i, _u32, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_size_t
_gp = ctypes.POINTER(ConvGeom)
_SIGS = {
    "fl_last_error": ([], ctypes.c_char_p),
    "fl_conv_geom_make": ([_i] * 8 + [_gp], _i),
    "fl_ctx_create": ([_i, _i, _u32, ctypes.POINTER(_vp)], _i),
    "fl_ctx_destroy": ([_vp], None),
    "fl_ctx_params": ([_vp, _vp, _vp, _vp], _i),
    "fl_keygen": ([_vp, _vp, _vp, _vp], _i),
    "fl_encrypt": ([_vp, _vp, _gp, _i, _vp, _vp, _vp, _vp, _vp], _i),
    "fl_encrypt_online": ([_vp, _gp, _i, _vp, _vp, _vp, _vp], _i),
    "fl_decrypt_workspace_bytes": ([_vp, _i], _sz),
    "fl_decrypt": ([_vp, _vp, _i, _vp, _vp, _vp, _sz, _vp], _i),
    "fl_extract_outputs": ([_gp, _i, _vp, _vp, _vp], _i),
    "fl_weights_bytes": ([_vp, _gp], _sz),
    "fl_encode_weights": ([_vp, _gp, _vp, _vp, _vp], _i),
    "fl_he_conv2d_workspace_bytes": ([_vp, _gp, _i], _sz),
    "fl_he_conv2d": ([_vp, _gp, _i, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "fl_mask_to_share": ([_vp, _i, _vp, _vp, _vp], _i),
    "fl_he_conv2d_direct": ([_vp, _gp, _i, _vp, _vp, _vp, _vp, _vp], _i),
    "fl_he_conv2d_tc": ([_vp, _gp, _i, _vp, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "fl_ctx_set_ntt_plan": ([_vp, _i], _i),
    "fl_ctx_get_ntt_plan": ([_vp], _i),
    "fl_ctx_set_tc_tile": ([_vp, _i], _i),
    "fl_ctx_get_tc_tile": ([_vp], _i),
    "fl_noise_workspace_bytes": ([_vp, _i], _sz),
    "fl_noise_inf": ([_vp, _vp, _i, _vp, _vp, _vp, _sz, _vp, ctypes.POINTER(ctypes.c_double)], _i),
    "fl_copy_to_device": ([_vp, _vp, _vp, _sz, _vp], _i),
    "fl_copy_to_host": ([_vp, _vp, _vp, _sz, _vp], _i),
    "fl_tc_weights_bytes": ([_vp, _gp], _sz),
    "fl_tc_weights": ([_vp, _gp, _vp, _vp, _vp], _i),
    "fl_he_conv2d_tc_workspace_bytes": ([_vp, _gp, _i], _sz),
    "fl_he_conv2d_tc_from_ntt": ([_vp, _gp, _i, _vp, _vp, _sz, _vp], _i),
    "fl_intt_mask_outputs": ([_vp, _gp, _i, _vp, _sz, _vp, _vp, _vp], _i),
    "fl_mod_switch": ([_vp, _i, _vp, _i, _vp, _vp], _i),
    "fl_he_conv2d_otf": ([_vp, _gp, _i, _vp, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "fl_he_conv2d_mask": ([_vp, _gp, _i, _vp, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "fl_he_conv2d_ntt_inputs": ([_vp, _gp, _i, _vp, _vp, _sz, _vp], _i),
    "fl_he_conv2d_from_ntt": ([_vp, _gp, _i, _vp, _vp, _sz, _vp, _vp, _vp], _i),
    "fl_stack_workspace_bytes": ([_vp, ctypes.POINTER(StackLayer), _i], _sz),
    "fl_he_conv2d_stack": ([_vp, ctypes.POINTER(StackLayer), _i, _vp, _sz, _vp], _i),
    "fl_he_conv2d_stack_ntt": ([_vp, ctypes.POINTER(StackLayer), _i, _vp, _sz, _vp], _i),
    "fl_he_conv2d_stack_run": ([_vp, ctypes.POINTER(StackLayer), _i, _vp, _sz, _vp], _i),
    "fl_stack_error": ([_vp, _vp, ctypes.POINTER(ctypes.c_uint64)], _i),
    "fl_tc_error": ([_vp, _vp, ctypes.POINTER(ctypes.c_uint64)], _i),
    "fl_he_conv2d_mask_noalloc": ([_vp, _gp, _i, _vp, _vp, _vp, _vp, _vp], _i),
    "fl_ctx_set_stack_kernel": ([_vp, _i], _i),
    "fl_ctx_get_stack_kernel": ([_vp], _i),
    "fl_batch_encode": ([_vp, _i, _vp, _vp, _vp], _i),
    "fl_batch_decode": ([_vp, _i, _vp, _vp, _vp], _i),
    "fl_x2x_prep_bytes": ([_vp, _i], _sz),
    "fl_x2x_prepare": ([_vp, _i, _vp, _vp, _vp, _vp], _i),
    "fl_x2x_round1": ([_vp, _i, _vp, _vp, _vp, _vp], _i),
    "fl_x2x_round2": ([_vp, _i, _vp, _vp, _vp, _vp, _vp], _i),
    "fl_repack_outputs": ([_gp, _gp, _i, _vp, _vp, _vp], _i),
    "fl_selftest_wait_timeout": ([_vp, ctypes.POINTER(ctypes.c_uint64)], _i),
    "fl_ntt_forward": ([_vp, _i, _vp, _vp], _i),
    "fl_ntt_inverse": ([_vp, _i, _vp, _vp], _i),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes, _f.restype = _args, _res


def header_symbols() -> list[str]:
    """Every entry point include/flashgpu.h declares."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(fl_[a-z0-9_]+)\s*\(", text)))


class FlashError(RuntimeError):
    pass


def _check(rc: int):
    if rc != FL_OK:
        raise FlashError(f"flashgpu error {rc}: {_lib.fl_last_error().decode()}")


def fl_last_error() -> str:
    return _lib.fl_last_error().decode()


def fl_conv_geom_make(N, Cin, Cout, H, W, k, stride=1, pad=0) -> ConvGeom:
    g = ConvGeom()
    _check(_lib.fl_conv_geom_make(N, Cin, Cout, H, W, k, stride, pad, ctypes.byref(g)))
    return g


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


_KINDS = {"u32": ((torch.int32, torch.uint32), "32-bit"), "i16": ((torch.int16, torch.uint16), "16-bit"),
          "i8": ((torch.int8,), "int8"), "any": (None, "")}


def _dev(t, kind, shape, name, device=None):
    """The C entry points take raw device pointers and cannot check what they
    point to: every tensor handed to one is checked here first -- a CUDA
    tensor (on `device` when given), contiguous, of the element kind and (when
    `shape` is not None) the shape the call reads or writes."""
    dtypes, what = _KINDS[kind]
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous() or \
            (dtypes is not None and t.dtype not in dtypes):
        raise FlashError(f"{name}: expected a contiguous {what + ' ' if what else ''}CUDA tensor")
    if device is not None and t.device.index != device:
        raise FlashError(f"{name}: on cuda:{t.device.index}, the context is on cuda:{device}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise FlashError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")
    return t


def _dev_u32(t: torch.Tensor, shape, name, device=None):
    return _dev(t, "u32", shape, name, device)


def _dev_i16(t: torch.Tensor, shape, name, device=None):
    return _dev(t, "i16", shape, name, device)


def selftest_wait_timeout(stream=None) -> tuple[int, int]:
    """Run the bounded-wait self-test; returns (status, error word)."""
    v = ctypes.c_uint64()
    rc = _lib.fl_selftest_wait_timeout(_stream(stream), ctypes.byref(v))
    return rc, v.value


def repack_outputs(prev: ConvGeom, nxt: ConvGeom, src, out=None, stream=None) -> torch.Tensor:
    """Plain vectors [B][prev.n_out][N] in prev's output layout -> [B][nxt.n_in][N]
    in nxt's zero-padded input layout."""
    B = src.shape[0]
    _dev_u32(src, (B, prev.n_out, prev.N), "src")
    if out is None:
        out = torch.empty((B, nxt.n_in, nxt.N), dtype=src.dtype, device=src.device)
    _dev_u32(out, (B, nxt.n_in, nxt.N), "out", src.device.index)
    _check(_lib.fl_repack_outputs(ctypes.byref(prev), ctypes.byref(nxt), B, _ptr(src), _ptr(out), _stream(stream)))
    return out


class Context:
    """fl_ctx on the current CUDA device (ring degree N, L limbs, plaintext t)."""

    def __init__(self, N: int, L: int, t: int = 65537):
        h = ctypes.c_void_p()
        _check(_lib.fl_ctx_create(N, L, t, ctypes.byref(h)))
        self.h, self.N, self.L, self.t = h, N, L, t
        q = (ctypes.c_uint32 * L)()
        d = (ctypes.c_uint32 * L)()
        p = (ctypes.c_uint32 * L)()
        _check(_lib.fl_ctx_params(h, q, d, p))
        self.primes, self.delta, self.psi = list(q), list(d), list(p)
        self.device = torch.cuda.current_device()

    def __del__(self):
        if getattr(self, "h", None):
            _lib.fl_ctx_destroy(self.h)
            self.h = None

    def geom(self, Cin, Cout, H, W, k, stride=1, pad=0) -> ConvGeom:
        return fl_conv_geom_make(self.N, Cin, Cout, H, W, k, stride, pad)

    def _new(self, *shape):
        return torch.empty(shape, dtype=torch.int32, device=f"cuda:{self.device}")

    def _u32(self, t, shape, name):
        return _dev(t, "u32", shape, name, self.device)

    def _ct(self, t, name):
        """Ciphertexts [..., 2, L, N]; returns how many."""
        _dev(t, "u32", None, name, self.device)
        if t.dim() < 3 or tuple(t.shape[-3:]) != (2, self.L, self.N):
            raise FlashError(f"{name}: expected [..., 2, {self.L}, {self.N}], got {tuple(t.shape)}")
        return t.numel() // (2 * self.L * self.N)

    def _ws(self, t, name="workspace"):
        """A workspace: any contiguous tensor on the context's device; the
        library checks its size in bytes."""
        return _dev(t, "any", None, name, self.device)

    def _out(self, out, shape, name="out"):
        return self._new(*shape) if out is None else self._u32(out, shape, name)

    # -- client side -----------------------------------------------------
    def keygen(self, s: torch.Tensor, stream=None) -> torch.Tensor:
        _dev(s, "i8", (self.N,), "s", self.device)
        sk = self._new(self.L, self.N)
        _check(_lib.fl_keygen(self.h, _ptr(s), _ptr(sk), _stream(stream)))
        return sk

    def encrypt(self, sk, g: ConvGeom, x, a, e, out=None, stream=None) -> torch.Tensor:
        B = x.shape[0]
        self._u32(sk, (self.L, self.N), "sk")
        self._u32(x, (B, g.Cin, g.H, g.W), "x")
        self._u32(a, (B, g.n_in, self.L, self.N), "a")
        self._u32(e, (B, g.n_in, self.N), "e")
        out = self._out(out, (B, g.n_in, 2, self.L, self.N))
        _check(_lib.fl_encrypt(self.h, _ptr(sk), ctypes.byref(g), B, _ptr(x), _ptr(a), _ptr(e), _ptr(out),
                               _stream(stream)))
        return out

    def encrypt_online(self, g: ConvGeom, x, enc0, out=None, stream=None) -> torch.Tensor:
        B = x.shape[0]
        self._u32(x, (B, g.Cin, g.H, g.W), "x")
        self._u32(enc0, (B, g.n_in, 2, self.L, self.N), "enc0")
        out = torch.empty_like(enc0) if out is None else self._u32(out, tuple(enc0.shape), "out")
        _check(_lib.fl_encrypt_online(self.h, ctypes.byref(g), B, _ptr(x), _ptr(enc0), _ptr(out), _stream(stream)))
        return out

    def decrypt(self, sk, ct, stream=None) -> torch.Tensor:
        """ct [..., 2, L, N] -> m [..., N] (values in [0, t))."""
        self._u32(sk, (self.L, self.N), "sk")
        n = self._ct(ct, "ct")
        lead = ct.shape[:-3]
        ws = torch.empty(_lib.fl_decrypt_workspace_bytes(self.h, n) // 4 + 4, dtype=torch.int32, device=ct.device)
        m = self._new(*lead, self.N)
        _check(_lib.fl_decrypt(self.h, _ptr(sk), n, _ptr(ct), _ptr(m), _ptr(ws), ws.numel() * 4, _stream(stream)))
        return m

    def extract_outputs(self, g: ConvGeom, m, stream=None) -> torch.Tensor:
        B = m.shape[0]
        self._u32(m, (B, g.n_out, self.N), "m")
        y = self._new(B, g.Cout, g.Ho, g.Wo)
        _check(_lib.fl_extract_outputs(ctypes.byref(g), B, _ptr(m), _ptr(y), _stream(stream)))
        return y

    # -- server side -----------------------------------------------------
    def weights_bytes(self, g: ConvGeom) -> int:
        return _lib.fl_weights_bytes(self.h, ctypes.byref(g))

    def encode_weights(self, g: ConvGeom, w, out=None, stream=None) -> torch.Tensor:
        _dev(w, "i8", (g.Cout, g.Cin, g.k, g.k), "w", self.device)
        out = self._out(out, (self.L, g.Cout, g.G, self.N))
        _check(_lib.fl_encode_weights(self.h, ctypes.byref(g), _ptr(w), _ptr(out), _stream(stream)))
        return out

    def workspace_bytes(self, g: ConvGeom, B: int) -> int:
        return _lib.fl_he_conv2d_workspace_bytes(self.h, ctypes.byref(g), B)

    def workspace(self, g: ConvGeom, B: int) -> torch.Tensor:
        return torch.empty(max(self.workspace_bytes(g, B), 16) // 4, dtype=torch.int32,
                           device=f"cuda:{self.device}")

    def he_conv2d(self, g, w_hat, ct_in, out=None, workspace=None, r=None, stream=None) -> torch.Tensor:
        """Homomorphic convolution of ct_in [B][n_in][2][L][N]; with r
        ([B][n_out][N]) the mask addition is fused (fl_he_conv2d_mask)."""
        B = ct_in.shape[0]
        self._u32(ct_in, (B, g.n_in, 2, self.L, self.N), "ct_in")
        self._u32(w_hat, (self.L, g.Cout, g.G, self.N), "w_hat")
        out = self._out(out, (B, g.n_out, 2, self.L, self.N))
        ws = self.workspace(g, B) if workspace is None else self._ws(workspace)
        if r is None:
            _check(_lib.fl_he_conv2d(self.h, ctypes.byref(g), B, _ptr(w_hat), _ptr(ct_in), _ptr(out), _ptr(ws),
                                     ws.numel() * ws.element_size(), _stream(stream)))
        else:
            self._u32(r, (B, g.n_out, self.N), "r")
            _check(_lib.fl_he_conv2d_mask(self.h, ctypes.byref(g), B, _ptr(w_hat), _ptr(ct_in), _ptr(r), _ptr(out),
                                          _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))
        return out

    def he_conv2d_ntt_inputs(self, g, ct_in, workspace, stream=None):
        """Stage a3 of he_conv2d: forward NTT of ct_in into the workspace."""
        self._u32(ct_in, (ct_in.shape[0], g.n_in, 2, self.L, self.N), "ct_in")
        self._ws(workspace)
        _check(_lib.fl_he_conv2d_ntt_inputs(self.h, ctypes.byref(g), ct_in.shape[0], _ptr(ct_in), _ptr(workspace),
                                            workspace.numel() * workspace.element_size(), _stream(stream)))

    def he_conv2d_from_ntt(self, g, B, w_hat, workspace, out, r=None, stream=None):
        """Stages a4-a6 of he_conv2d from a workspace filled by he_conv2d_ntt_inputs."""
        self._u32(w_hat, (self.L, g.Cout, g.G, self.N), "w_hat")
        self._ws(workspace)
        self._u32(out, (B, g.n_out, 2, self.L, self.N), "out")
        if r is not None:
            self._u32(r, (B, g.n_out, self.N), "r")
        _check(_lib.fl_he_conv2d_from_ntt(self.h, ctypes.byref(g), B, _ptr(w_hat), _ptr(workspace),
                                          workspace.numel() * workspace.element_size(), _ptr(r), _ptr(out),
                                          _stream(stream)))
        return out

    # -- many layers in one launch ------------------------------------------
    def stack_layers(self, specs):
        """specs: list of dicts with keys g, w_hat, ct_in, out and optional r.
        Returns the ctypes array fl_he_conv2d_stack takes.  The array holds
        raw device pointers, so it keeps every geometry and tensor it points
        to alive through its `_keep` list: a tensor built inline in `specs`
        is not freed (and its memory reused) while the array exists."""
        arr = (StackLayer * len(specs))()
        keep = []
        for k, sp in enumerate(specs):
            g = sp["g"]
            B = sp["ct_in"].shape[0]
            self._u32(sp["w_hat"], (self.L, g.Cout, g.G, self.N), f"layer {k}: w_hat")
            self._u32(sp["ct_in"], (B, g.n_in, 2, self.L, self.N), f"layer {k}: ct_in")
            self._u32(sp["out"], (B, g.n_out, 2, self.L, self.N), f"layer {k}: out")
            if sp.get("r") is not None:
                self._u32(sp["r"], (B, g.n_out, self.N), f"layer {k}: r")
            keep.extend([g, sp["w_hat"], sp["ct_in"], sp["out"], sp.get("r")])
            arr[k].geom = ctypes.pointer(g)
            arr[k].B = sp["ct_in"].shape[0]
            arr[k].w_hat_dev = sp["w_hat"].data_ptr()
            arr[k].ct_in_dev = sp["ct_in"].data_ptr()
            arr[k].r_dev = sp["r"].data_ptr() if sp.get("r") is not None else None
            arr[k].ct_out_dev = sp["out"].data_ptr()
        arr._keep = keep
        return arr

    def stack_workspace(self, arr) -> torch.Tensor:
        nbytes = _lib.fl_stack_workspace_bytes(self.h, arr, len(arr))
        return torch.empty(max(nbytes, 256) // 4, dtype=torch.int32, device=f"cuda:{self.device}")

    def he_conv2d_stack(self, arr, workspace, stream=None, stage="all"):
        fn = {"all": _lib.fl_he_conv2d_stack, "ntt": _lib.fl_he_conv2d_stack_ntt,
              "run": _lib.fl_he_conv2d_stack_run}[stage]
        self._ws(workspace)
        _check(fn(self.h, arr, len(arr), _ptr(workspace), workspace.numel() * workspace.element_size(),
                  _stream(stream)))

    @property
    def stack_kernel(self) -> int:
        return _lib.fl_ctx_get_stack_kernel(self.h)

    @stack_kernel.setter
    def stack_kernel(self, k: int):
        _check(_lib.fl_ctx_set_stack_kernel(self.h, k))

    @property
    def ntt_plan(self) -> int:
        """First row-pass radix exponent r1 of the input NTT and the
        inverse-NTT-rows kernel (fl_ctx_set_ntt_plan); 0 sets the default."""
        return _lib.fl_ctx_get_ntt_plan(self.h)

    @ntt_plan.setter
    def ntt_plan(self, r1: int):
        _check(_lib.fl_ctx_set_ntt_plan(self.h, r1))

    @property
    def tc_tile(self) -> int:
        """Slot groups of 4 per CTA of the tensor-core contraction (4, 8, 16)."""
        return _lib.fl_ctx_get_tc_tile(self.h)

    @tc_tile.setter
    def tc_tile(self, groups: int):
        _check(_lib.fl_ctx_set_tc_tile(self.h, groups))

    def stack_error(self, workspace, stream=None) -> int:
        self._ws(workspace)
        v = ctypes.c_uint64()
        rc = _lib.fl_stack_error(_ptr(workspace), _stream(stream), ctypes.byref(v))
        if rc not in (FL_OK, FL_ERR_TIMEOUT):
            _check(rc)
        return v.value

    def he_conv2d_mask_noalloc(self, g, w_hat, ct_in, r, out, stream=None) -> torch.Tensor:
        """fl_he_conv2d_mask without a workspace: the library's fixed scratch
        array is used instead (FL_NOALLOC_SCRATCH_BYTES; calls must not
        overlap on the GPU).  Allocates nothing on the device; `out` is the
        caller's [B][n_out][2][L][N] buffer.  Every buffer's dtype, device,
        contiguity and shape is checked before the call."""
        B = ct_in.shape[0]
        self._u32(ct_in, (B, g.n_in, 2, self.L, self.N), "ct_in")
        self._u32(w_hat, (self.L, g.Cout, g.G, self.N), "w_hat")
        self._u32(r, (B, g.n_out, self.N), "r")
        self._u32(out, (B, g.n_out, 2, self.L, self.N), "out")
        _check(_lib.fl_he_conv2d_mask_noalloc(self.h, ctypes.byref(g), ct_in.shape[0], _ptr(w_hat), _ptr(ct_in),
                                              _ptr(r), _ptr(out), _stream(stream)))
        return out

    def he_conv2d_otf(self, g, w, ct_in, out=None, workspace=None, r=None, stream=None) -> torch.Tensor:
        """On-the-fly weights: the same ciphertexts as he_conv2d (plus the mask
        when r is given) from int8 filters w [Cout][Cin][k][k], with no
        encoded weights."""
        B = ct_in.shape[0]
        _dev(w, "i8", (g.Cout, g.Cin, g.k, g.k), "w", self.device)
        self._u32(ct_in, (B, g.n_in, 2, self.L, self.N), "ct_in")
        if r is not None:
            self._u32(r, (B, g.n_out, self.N), "r")
        out = self._out(out, (B, g.n_out, 2, self.L, self.N))
        workspace = self.workspace(g, B) if workspace is None else self._ws(workspace)
        _check(_lib.fl_he_conv2d_otf(self.h, ctypes.byref(g), B, _ptr(w), _ptr(ct_in), _ptr(r), _ptr(out),
                                     _ptr(workspace), workspace.numel() * workspace.element_size(),
                                     _stream(stream)))
        return out

    def he_conv2d_direct(self, g, w, ct_in, out=None, r=None, stream=None) -> torch.Tensor:
        """Direct form (DRot + CMult, no NTT) from int8 filters w [Cout][Cin][k][k];
        the same ciphertexts as he_conv2d (plus the mask when r is given)."""
        B = ct_in.shape[0]
        _dev(w, "i8", (g.Cout, g.Cin, g.k, g.k), "w", self.device)
        self._u32(ct_in, (B, g.n_in, 2, self.L, self.N), "ct_in")
        if r is not None:
            self._u32(r, (B, g.n_out, self.N), "r")
        out = self._out(out, (B, g.n_out, 2, self.L, self.N))
        _check(_lib.fl_he_conv2d_direct(self.h, ctypes.byref(g), B, _ptr(w), _ptr(ct_in), _ptr(r), _ptr(out),
                                        _stream(stream)))
        return out

    def tc_workspace_bytes(self, g, B: int) -> int:
        return _lib.fl_he_conv2d_tc_workspace_bytes(self.h, ctypes.byref(g), B)

    def tc_workspace(self, g, B: int) -> torch.Tensor:
        """Workspace of he_conv2d_tc: the inputs' NTT images, their
        slot-tiled copy and the slot-tiled NTT-domain outputs."""
        nbytes = self.tc_workspace_bytes(g, B)
        return torch.empty(max(nbytes, 16) // 4, dtype=torch.int32, device=f"cuda:{self.device}")

    def tc_weight_shape(self, g):
        """Shape of tc_weights' result: [L][ceil(Cout/128)][N/4][ceil(G/4)][8192]
        fp16 digits (one 16 KB weight tile per (limb, 128 output channels,
        4-slot group, K step))."""
        return (self.L, (g.Cout + 127) // 128, self.N // 4, (g.G + 3) // 4, 8192)

    def tc_weights(self, g, w_hat, out=None, stream=None) -> torch.Tensor:
        """The encoded weights [L][Cout][G][N] as he_conv2d_tc's weight tiles:
        balanced base-256 digits in fp16, in the MMA's shared-memory layout
        (int16 tensor of tc_weight_shape(g); see fl_tc_weights)."""
        self._u32(w_hat, (self.L, g.Cout, g.G, self.N), "w_hat")
        if g.G > FL_TC_MAX_G:
            raise FlashError(f"G={g.G} above {FL_TC_MAX_G}: the tensor-core form is not exact")
        shape = self.tc_weight_shape(g)
        if 2 * math.prod(shape) != _lib.fl_tc_weights_bytes(self.h, ctypes.byref(g)):
            raise FlashError("tensor-core weight tiles: the library's size differs from the binding's shape")
        out = torch.empty(shape, dtype=torch.int16, device=w_hat.device) if out is None else out
        _dev_i16(out, shape, "out", self.device)
        _check(_lib.fl_tc_weights(self.h, ctypes.byref(g), _ptr(w_hat), _ptr(out), _stream(stream)))
        return out

    def he_conv2d_tc(self, g, w_tc, ct_in, out=None, workspace=None, r=None, stream=None) -> torch.Tensor:
        """Tensor-core form (tcgen05, fp16 digits, fp32 accumulation): the
        same ciphertexts as he_conv2d (plus the mask when r is given) from
        the weight tiles of tc_weights.  G <= FL_TC_MAX_G."""
        B = ct_in.shape[0]
        self._u32(ct_in, (B, g.n_in, 2, self.L, self.N), "ct_in")
        _dev_i16(w_tc, self.tc_weight_shape(g), "w_tc", self.device)
        if r is not None:
            self._u32(r, (B, g.n_out, self.N), "r")
        out = self._new(B, g.n_out, 2, self.L, self.N) if out is None else out
        self._u32(out, (B, g.n_out, 2, self.L, self.N), "out")
        workspace = self.tc_workspace(g, B) if workspace is None else self._ws(workspace)
        _check(_lib.fl_he_conv2d_tc(self.h, ctypes.byref(g), B, _ptr(w_tc), _ptr(ct_in), _ptr(r), _ptr(out),
                                    _ptr(workspace), workspace.numel() * workspace.element_size(),
                                    _stream(stream)))
        return out

    def he_conv2d_tc_from_ntt(self, g, B, w_tc, workspace, stream=None):
        """Stage of he_conv2d_tc: the tensor-core contraction from a workspace
        filled by he_conv2d_ntt_inputs; the NTT-domain outputs (values in
        [0, 2q), slot-tiled) stay in the workspace for intt_mask_outputs."""
        _dev_i16(w_tc, self.tc_weight_shape(g), "w_tc", self.device)
        self._ws(workspace)
        _check(_lib.fl_he_conv2d_tc_from_ntt(self.h, ctypes.byref(g), B, _ptr(w_tc), _ptr(workspace),
                                             workspace.numel() * workspace.element_size(), _stream(stream)))

    def intt_mask_outputs(self, g, workspace, out, r=None, stream=None):
        """Stage of he_conv2d_tc: the inverse NTT of the NTT-domain outputs
        he_conv2d_tc_from_ntt left in the workspace, plus the mask when r is
        given, into out."""
        B = out.shape[0]
        self._u32(out, (B, g.n_out, 2, self.L, self.N), "out")
        if r is not None:
            self._u32(r, (B, g.n_out, self.N), "r")
        self._ws(workspace)
        _check(_lib.fl_intt_mask_outputs(self.h, ctypes.byref(g), B, _ptr(workspace),
                                         workspace.numel() * workspace.element_size(), _ptr(r), _ptr(out),
                                         _stream(stream)))
        return out

    def noise_inf(self, sk, ct, m, stream=None) -> float:
        """Largest |v| of the decryption noise (Appendix A) of ct [..., 2, L, N]
        against the expected messages m [..., N] (values in [0, t))."""
        self._u32(sk, (self.L, self.N), "sk")
        n = self._ct(ct, "ct")
        _dev(m, "u32", None, "m", self.device)
        if m.numel() != n * self.N:
            raise FlashError(f"m: {m.numel()} values for {n} ciphertexts of {self.N} coefficients")
        ws = torch.empty(max(_lib.fl_noise_workspace_bytes(self.h, n), 16) // 4, dtype=torch.int32, device=ct.device)
        v = ctypes.c_double()
        _check(_lib.fl_noise_inf(self.h, _ptr(sk), n, _ptr(ct), _ptr(m), _ptr(ws), ws.numel() * 4, _stream(stream),
                                 ctypes.byref(v)))
        return v.value

    def copy_to_device(self, host, dev, stream=None):
        """Copy the host tensor's 32-bit words into the device tensor through
        the library (fl_copy_to_device); asynchronous for pinned host memory."""
        if not isinstance(host, torch.Tensor) or host.is_cuda or not host.is_contiguous() or \
                host.numel() != dev.numel() or host.element_size() != 4:
            raise FlashError("copy_to_device: a contiguous 32-bit host tensor and a device tensor of the same size")
        self._u32(dev, dev.shape, "dev")
        _check(_lib.fl_copy_to_device(self.h, _ptr(host), _ptr(dev), host.numel(), _stream(stream)))
        return dev

    def copy_to_host(self, dev, host, stream=None):
        """Copy the device tensor's 32-bit words into the host tensor through
        the library (fl_copy_to_host); asynchronous for pinned host memory."""
        self._u32(dev, dev.shape, "dev")
        if not isinstance(host, torch.Tensor) or host.is_cuda or not host.is_contiguous() or \
                host.numel() != dev.numel() or host.element_size() != 4:
            raise FlashError("copy_to_host: a device tensor and a contiguous 32-bit host tensor of the same size")
        _check(_lib.fl_copy_to_host(self.h, _ptr(dev), _ptr(host), dev.numel(), _stream(stream)))
        return host

    def tc_error(self, stream=None) -> int:
        """Synchronise and read (and clear) the tensor-core form's error word:
        0, or bit 0 when a bounded wait inside he_conv2d_tc ran out."""
        v = ctypes.c_uint64()
        rc = _lib.fl_tc_error(self.h, _stream(stream), ctypes.byref(v))
        if rc not in (FL_OK, FL_ERR_TIMEOUT):
            _check(rc)
        return v.value

    def mod_switch(self, ct, L_out: int, out=None, stream=None) -> torch.Tensor:
        """Ciphertexts [..., 2, L, N] -> [..., 2, L_out, N] under the first L_out primes."""
        n = self._ct(ct, "ct")
        shape = tuple(ct.shape[:-2]) + (L_out, self.N)
        if out is None:
            out = torch.empty(shape, dtype=ct.dtype, device=ct.device)
        self._u32(out, shape, "out")
        _check(_lib.fl_mod_switch(self.h, n, _ptr(ct), L_out, _ptr(out), _stream(stream)))
        return out

    def mask_to_share(self, ct, r, stream=None) -> torch.Tensor:
        """In place: c0 += Delta*r for ct [..., 2, L, N], r [..., N]."""
        n = self._ct(ct, "ct")
        self._u32(r, tuple(ct.shape[:-3]) + (self.N,), "r")
        _check(_lib.fl_mask_to_share(self.h, n, _ptr(ct), _ptr(r), _stream(stream)))
        return ct

    # -- x^2 + x protocol, server side (Sec. 5.2) and batch encoding ---------
    def _n_vec(self, t, name):
        if t.numel() % self.N:
            raise FlashError(f"{name}: size {t.numel()} is not a multiple of N={self.N}")
        return self._u32(t, t.shape, name).numel() // self.N

    def batch_encode(self, slots, out=None, stream=None) -> torch.Tensor:
        """slots [..., N] -> plaintext polynomials [..., N] in [0, t)."""
        n = self._n_vec(slots, "slots")
        out = torch.empty_like(slots) if out is None else self._u32(out, tuple(slots.shape), "out")
        _check(_lib.fl_batch_encode(self.h, n, _ptr(slots), _ptr(out), _stream(stream)))
        return out

    def batch_decode(self, m, out=None, stream=None) -> torch.Tensor:
        """plaintext polynomials [..., N] (values in [0, t)) -> slots [..., N]."""
        n = self._n_vec(m, "m")
        out = torch.empty_like(m) if out is None else self._u32(out, tuple(m.shape), "out")
        _check(_lib.fl_batch_decode(self.h, n, _ptr(m), _ptr(out), _stream(stream)))
        return out

    def x2x_prepare(self, r, v, out=None, stream=None) -> torch.Tensor:
        """Offline step: masks r, v [..., N] -> prep [n][L+2][N]."""
        n = self._n_vec(r, "r")
        self._u32(v, r.shape, "v")
        out = self._out(out, (n, self.L + 2, self.N), "prep")
        _check(_lib.fl_x2x_prepare(self.h, n, _ptr(r), _ptr(v), _ptr(out), _stream(stream)))
        return out

    def x2x_round1(self, prep, ct_z, out=None, stream=None) -> torch.Tensor:
        """<2rz + v> (batch encoded) from <z> (batch encoded) [n][2][L][N]."""
        n = prep.shape[0]
        self._u32(prep, (n, self.L + 2, self.N), "prep")
        self._u32(ct_z, (n, 2, self.L, self.N), "ct_z")
        out = self._out(out, (n, 2, self.L, self.N))
        _check(_lib.fl_x2x_round1(self.h, n, _ptr(prep), _ptr(ct_z), _ptr(out), _stream(stream)))
        return out

    def x2x_round2(self, prep, ct_x, ct_y, out=None, stream=None) -> torch.Tensor:
        """<a^2 + a> = <X> - <Y> + (r^2 - r + v), direct encoded [n][2][L][N]."""
        n = prep.shape[0]
        self._u32(prep, (n, self.L + 2, self.N), "prep")
        self._u32(ct_x, (n, 2, self.L, self.N), "ct_x")
        self._u32(ct_y, (n, 2, self.L, self.N), "ct_y")
        out = self._out(out, (n, 2, self.L, self.N))
        _check(_lib.fl_x2x_round2(self.h, n, _ptr(prep), _ptr(ct_x), _ptr(ct_y), _ptr(out), _stream(stream)))
        return out

    def _polys(self, data, name="data"):
        """Polynomials [..., L, N] in place; returns how many L-limb groups."""
        self._u32(data, data.shape, name)
        if data.dim() < 2 or tuple(data.shape[-2:]) != (self.L, self.N):
            raise FlashError(f"{name}: expected [..., {self.L}, {self.N}], got {tuple(data.shape)}")
        return data.numel() // (self.L * self.N)

    def ntt_forward(self, data, stream=None):
        self._polys(data)
        _check(_lib.fl_ntt_forward(self.h, data.numel() // (self.L * self.N), _ptr(data), _stream(stream)))
        return data

    def ntt_inverse(self, data, stream=None):
        self._polys(data)
        _check(_lib.fl_ntt_inverse(self.h, data.numel() // (self.L * self.N), _ptr(data), _stream(stream)))
        return data
