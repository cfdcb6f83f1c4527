"""The allocation-free entry point, fl_he_conv2d_mask_noalloc, against the
workspace-taking fl_he_conv2d_mask.

fl_he_conv2d_mask_noalloc exists for callers that may not allocate device
memory (a plugin whose host framework owns all device memory, or a request
loop that must not allocate on its hot path); it keeps its scratch in a
fixed array inside the library instead of a caller workspace.  This file is
collected last so that a failure here never hides the other tests."""
import numpy as np
import pytest

from paper_2401_16732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
T = 65537


def _dev(a, dtype=torch.int32):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(dtype).cuda()


@pytest.mark.parametrize("N,L,shape,B", [(4096, 2, (16, 16, 16, 16, 3, 1, 1), 1),
                                         (8192, 3, (64, 24, 32, 32, 3, 1, 1), 2)])
def test_noalloc_equals_workspace_entry_point_on_two_calls(N, L, shape, B):
    from paper_2401_16732_gb300 import flashgpu as fg
    c = fg.Context(N, L, T)
    g = c.geom(*shape)
    for call in range(2):  # the second call reuses the scratch the first one left behind
        seed = 900 + call
        w = synth.weights(seed, (g.Cout, g.Cin, g.k, g.k))
        ct = _dev(synth.raw_ciphertexts(seed, c.primes, (B, g.n_in, 2, L, N)))
        r = _dev(synth.masks(seed, (B, g.n_out, N), T))
        wh = c.encode_weights(g, _dev(w, torch.int8))
        want = c.he_conv2d(g, wh, ct, r=r)  # fl_he_conv2d_mask with a workspace
        out = torch.full_like(want, -1)
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        free_before, _ = torch.cuda.mem_get_info()  # the CUDA driver's count of free memory: it sees a cudaMalloc inside the library too
        c.he_conv2d_mask_noalloc(g, wh, ct, r, out)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
        if call == 1:
            # the first call may load the library's device code (the scratch
            # array comes with it); from then on the device's free memory
            # must not move
            assert torch.cuda.mem_get_info()[0] == free_before
        assert torch.equal(out, want), f"call {call}"


def test_noalloc_checks_buffer_shapes_before_the_call():
    from paper_2401_16732_gb300 import flashgpu as fg
    c = fg.Context(4096, 2, T)
    g = c.geom(16, 16, 16, 16, 3, 1, 1)
    wh = torch.zeros((2, g.Cout, g.G, 4096), dtype=torch.int32, device="cuda")
    ct = torch.zeros((1, g.n_in, 2, 2, 4096), dtype=torch.int32, device="cuda")
    r = torch.zeros((1, g.n_out, 4096), dtype=torch.int32, device="cuda")
    out = torch.zeros((1, g.n_out, 2, 2, 4096), dtype=torch.int32, device="cuda")
    with pytest.raises(fg.FlashError, match="^out:"):
        c.he_conv2d_mask_noalloc(g, wh, ct, r, out[:, :-1])  # one output ciphertext short
    with pytest.raises(fg.FlashError, match="^r:"):
        c.he_conv2d_mask_noalloc(g, wh, ct, r.cpu(), out)  # mask on the host
    with pytest.raises(fg.FlashError, match="^w_hat:"):
        c.he_conv2d_mask_noalloc(g, wh[:, :, :, :2048], ct, r, out)


def test_noalloc_rejects_calls_beyond_its_scratch():
    from paper_2401_16732_gb300 import flashgpu as fg
    c = fg.Context(8192, 3, T)
    g = c.geom(64, 64, 32, 32, 3, 1, 1)  # 1.97 MB of scratch per image
    B = fg.FL_NOALLOC_SCRATCH_BYTES // c.workspace_bytes(g, 1) + 1
    wh = torch.zeros((3, 64, g.G, 8192), dtype=torch.int32, device="cuda")
    ct = torch.zeros((B, g.n_in, 2, 3, 8192), dtype=torch.int32, device="cuda")
    r = torch.zeros((B, g.n_out, 8192), dtype=torch.int32, device="cuda")
    out = torch.zeros((B, g.n_out, 2, 3, 8192), dtype=torch.int32, device="cuda")
    with pytest.raises(fg.FlashError, match="scratch"):
        c.he_conv2d_mask_noalloc(g, wh, ct, r, out)
