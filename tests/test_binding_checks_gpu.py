"""The Python binding checks every tensor before it hands a raw pointer to
the C entry points: a tensor of the wrong shape, element type or device, or
a non-contiguous view, is refused with FlashError and no call is made (the
library itself cannot see what a device pointer points to).

On the CPU: the checking helper, and a reading of flashgpu.py's source that
every tensor whose pointer a method passes on has gone through a check (or
was allocated by the method).  On the GPU: each refusal, on a small context.
The misfits keep their storage at least as large as the valid tensor's, so
that even a missing check could not make a kernel reach past an allocation;
the host-memory misfit is refused by the same check that the source reading
shows every pointer goes through."""
import ast
import pathlib

import pytest

torch = pytest.importorskip("torch")

N, L, T = 2048, 1, 65537
SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2401_16732_gb300" / "flashgpu.py"


def test_helper_refuses_host_and_misshaped_tensors():
    from paper_2401_16732_gb300 import flashgpu as fg
    with pytest.raises(fg.FlashError, match="CUDA tensor"):
        fg._dev(torch.zeros(4, dtype=torch.int32), "u32", (4,), "x")
    with pytest.raises(fg.FlashError, match="CUDA tensor"):
        fg._dev([0, 1], "any", None, "x")


def test_every_pointer_the_binding_passes_on_is_checked_first():
    """Every `_ptr(x)` in a function of flashgpu.py names a tensor that the
    same function checks (_dev, _u32, _ws, _ct, ...) or allocates itself.
    The host buffers of the two copy calls are checked by hand (host memory,
    contiguous, 32-bit, same size): they are listed here."""
    checks = {"_u32", "_dev", "_dev_u32", "_dev_i16", "_ws", "_ct", "_n_vec", "_polys", "_out"}
    allocs = {"_new", "empty", "empty_like", "workspace", "tc_workspace", "stack_workspace"}
    by_hand = {("copy_to_device", "host"), ("copy_to_host", "host")}

    def name(call):
        f = call.func
        return f.attr if isinstance(f, ast.Attribute) else getattr(f, "id", None)

    missing = []
    for fn in ast.walk(ast.parse(SRC.read_text())):
        if not isinstance(fn, ast.FunctionDef):
            continue
        checked, ptrs = set(), []
        for node in ast.walk(fn):
            if isinstance(node, ast.Call) and node.args:
                if name(node) in checks:
                    checked.add(ast.unparse(node.args[0]))
                if name(node) == "_ptr":
                    ptrs.append(ast.unparse(node.args[0]))
            if isinstance(node, ast.Assign) and any(
                    isinstance(c, ast.Call) and name(c) in checks | allocs for c in ast.walk(node.value)):
                checked.update(ast.unparse(t) for t in node.targets)
        missing += [(fn.name, p) for p in ptrs if p not in checked and (fn.name, p) not in by_hand]
    assert not missing, missing


def _misfits(t):
    """Misfits of a valid CUDA tensor t, each on storage at least as large as
    t's: one element short (a 1-D view of a longer buffer), a wider element
    type, a non-contiguous view of the right shape, and a host copy."""
    longer = torch.zeros(t.numel() + 1024, dtype=t.dtype, device=t.device)
    wider = torch.int64 if t.dtype != torch.int64 else torch.int32
    return {"short": longer[:t.numel() - 1],
            "dtype": torch.zeros(t.shape, dtype=wider, device=t.device),
            "strided": torch.zeros(t.shape + (2,), dtype=t.dtype, device=t.device)[..., 0],
            "host": t.cpu()}


@pytest.fixture(scope="module")
def setup():
    from paper_2401_16732_gb300 import flashgpu as fg
    c = fg.Context(N, L, T)
    g = c.geom(8, 4, 8, 8, 3, 1, 1)
    B = 2

    def z(*shape, dtype=torch.int32):
        return torch.zeros(shape, dtype=dtype, device="cuda")

    t = {"w": z(g.Cout, g.Cin, g.k, g.k, dtype=torch.int8), "w_hat": z(L, g.Cout, g.G, N),
         "ct_in": z(B, g.n_in, 2, L, N), "r": z(B, g.n_out, N), "conv_out": z(B, g.n_out, 2, L, N),
         "sk": z(L, N), "x": z(B, g.Cin, g.H, g.W), "a": z(B, g.n_in, L, N), "e": z(B, g.n_in, N),
         "m": z(B, g.n_out, N), "prep": z(B, L + 2, N), "ct": z(B, 2, L, N), "ct_r": z(B, N),
         "enc_out": z(B, g.n_in, 2, L, N), "w_out": z(L, g.Cout, g.G, N)}
    return fg, c, g, B, t


def _call(c, g, B, a, name):
    if name == "he_conv2d":
        c.he_conv2d(g, a["w_hat"], a["ct_in"], out=a["conv_out"], r=a["r"])
    elif name == "from_ntt":
        c.he_conv2d_from_ntt(g, B, a["w_hat"], c.workspace(g, B), a["conv_out"], r=a["r"])
    elif name == "otf":
        c.he_conv2d_otf(g, a["w"], a["ct_in"], out=a["conv_out"], r=a["r"])
    elif name == "direct":
        c.he_conv2d_direct(g, a["w"], a["ct_in"], out=a["conv_out"], r=a["r"])
    elif name == "encrypt":
        c.encrypt(a["sk"], g, a["x"], a["a"], a["e"], out=a["enc_out"])
    elif name == "encode_weights":
        c.encode_weights(g, a["w"], out=a["w_out"])
    elif name == "extract_outputs":
        c.extract_outputs(g, a["m"])
    elif name == "x2x_round1":
        c.x2x_round1(a["prep"], a["ct"], out=a["x2x_out"])
    elif name == "mask_to_share":
        c.mask_to_share(a["ct"], a["ct_r"])
    elif name == "ntt_forward":
        c.ntt_forward(a["ct"])
    elif name == "stack":
        arr = c.stack_layers([{"g": g, "w_hat": a["w_hat"], "ct_in": a["ct_in"], "out": a["conv_out"],
                               "r": a["r"]}])
        c.he_conv2d_stack(arr, c.stack_workspace(arr))


# (call, the argument replaced by each misfit in turn)
CASES = [("he_conv2d", "w_hat"), ("he_conv2d", "ct_in"), ("he_conv2d", "conv_out"), ("he_conv2d", "r"),
         ("from_ntt", "w_hat"), ("from_ntt", "conv_out"), ("from_ntt", "r"),
         ("otf", "w"), ("otf", "conv_out"), ("otf", "r"), ("direct", "w"), ("direct", "r"),
         ("encrypt", "sk"), ("encrypt", "x"), ("encrypt", "e"), ("encrypt", "enc_out"),
         ("encode_weights", "w"), ("encode_weights", "w_out"), ("extract_outputs", "m"),
         ("x2x_round1", "prep"), ("x2x_round1", "x2x_out"), ("mask_to_share", "ct_r"), ("ntt_forward", "ct"),
         ("stack", "conv_out"), ("stack", "w_hat")]


@pytest.mark.gpu
@pytest.mark.parametrize("call,arg", CASES)
def test_misfit_arguments_are_refused_before_the_call(setup, call, arg):
    fg, c, g, B, t = setup
    good = dict(t, x2x_out=torch.zeros((B, 2, L, N), dtype=torch.int32, device="cuda"))
    _call(c, g, B, good, call)  # the valid arguments go through
    torch.cuda.synchronize()
    for kind, bad in _misfits(good[arg]).items():
        with pytest.raises(fg.FlashError):
            _call(c, g, B, dict(good, **{arg: bad}), call)
    torch.cuda.synchronize()
