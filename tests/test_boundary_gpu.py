"""The client-side boundary calls: the decryption-noise hook (Appendix A)
against the oracle's exact noise norm, and the host <-> device copies that
the end-to-end measurement routes through the library."""
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


@pytest.mark.parametrize("N,L", [(4096, 2), (8192, 3), (16384, 4)])
def test_noise_of_fresh_and_convolved_ciphertexts_matches_the_oracle(fg, oracle, N, L):
    """Fresh encryptions have noise -e, so the hook gives max |e| (at most 21
    for CBD eta = 21); after a convolution and the mask, the hook equals the
    oracle's exact noise norm against the decrypted messages, below the
    derived bound."""
    c = fg.Context(N, L, T)
    g = c.geom(16, 8, 16, 16, 3, 1, 1)
    B = 2
    s = synth.secret_key(31, N)
    x = synth.activations(31, (B, g.Cin, g.H, g.W))
    a = synth.uniform_residues(31, c.primes, (B, g.n_in, L, N))
    e = synth.cbd_noise(31, (B, g.n_in, N))
    sk = c.keygen(dev(s, torch.int8))
    ct = c.encrypt(sk, g, dev(x), dev(a), dev(e))
    geo = oracle.geometry(N, *(16, 8, 16, 16, 3, 1, 1))
    m_in = np.stack([oracle.pack_inputs(x[b], geo) for b in range(B)]).astype(np.uint32)
    fresh = c.noise_inf(sk, ct.view(-1, 2, L, N), dev(m_in))
    assert fresh == np.abs(e).max()
    assert fresh == max(oracle.noise_inf(s, u32(ct)[b], m_in[b], c.primes) for b in range(B))
    w = synth.weights(31, (g.Cout, g.Cin, g.k, g.k))
    r = dev(synth.masks(31, (B, g.n_out, N), T))
    y = c.he_conv2d(g, c.encode_weights(g, dev(w, torch.int8)), ct, r=r)
    m_out = c.decrypt(sk, y)
    got = c.noise_inf(sk, y.view(-1, 2, L, N), m_out)
    want = max(oracle.noise_inf(s, u32(y)[b], u32(m_out)[b], c.primes) for b in range(B))
    assert got == want
    assert 0 < got <= oracle.noise_bound(w, c.primes, T, masked=True)


def test_noise_hook_rejects_short_workspace_and_bad_arguments(fg):
    c = fg.Context(2048, 1, T)
    with pytest.raises(fg.FlashError):
        c.noise_inf(torch.zeros((1, 2048), dtype=torch.int32, device="cuda"),
                    torch.zeros((1, 2, 1, 2048), dtype=torch.int32, device="cuda"),
                    torch.zeros(100, dtype=torch.int32, device="cuda"))


def test_copies_through_the_library_round_trip(fg):
    """fl_copy_to_device / fl_copy_to_host move ciphertext words between
    pinned (and pageable) host memory and the device bit for bit, and refuse
    a host pointer in the device slot."""
    c = fg.Context(4096, 2, T)
    host = torch.from_numpy(synth.raw_ciphertexts(32, c.primes, (3, 2, 2, 4096)).view(np.int32)).pin_memory()
    d = torch.empty(host.shape, dtype=torch.int32, device="cuda")
    c.copy_to_device(host, d)
    back = torch.empty_like(host).pin_memory()
    c.copy_to_host(d, back)
    torch.cuda.synchronize()
    assert torch.equal(back, host)
    pageable = torch.zeros_like(host)
    c.copy_to_host(d, pageable)
    torch.cuda.synchronize()
    assert torch.equal(pageable, host)
    with pytest.raises(fg.FlashError):
        c.copy_to_device(host, host.clone())
    import ctypes
    # the C entry point itself refuses device memory in the host slot
    rc = fg._lib.fl_copy_to_device(c.h, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()), d.numel(), None)
    assert rc == fg.FL_ERR_ARG
