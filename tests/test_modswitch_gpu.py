"""Parity of GPU modulus switching with the oracle, and decryption of
switched convolution outputs under the smaller context."""
import numpy as np
import pytest

from paper_2401_16732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
T = 65537


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def dev(a, dtype=torch.int32):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda()
    return torch.from_numpy(a).to(dtype).cuda()


@pytest.fixture(scope="module")
def fg():
    from paper_2401_16732_gb300 import flashgpu
    return flashgpu


_ctx = {}


def ctx(fg, N, L):
    if (N, L) not in _ctx:
        _ctx[(N, L)] = fg.Context(N, L)
    return _ctx[(N, L)]


@pytest.mark.parametrize("N,L,L_out,n", [(2048, 2, 1, 3), (4096, 3, 2, 2), (8192, 3, 2, 2), (16384, 4, 2, 1),
                                         (16384, 4, 3, 1), (2048, 3, 3, 2)])
def test_mod_switch_matches_oracle(fg, oracle, N, L, L_out, n):
    c = ctx(fg, N, L)
    ct = synth.raw_ciphertexts(80, c.primes, (n, 2, L, N))
    # the ends of every residue range, where the centred rounding flips
    ct[0, 0, :, :4] = np.array([[0, 1, q // 2, q - 1] for q in c.primes], np.uint32)
    ct[0, 0, -1, 4:8] = [c.primes[-1] // 2 + 1, c.primes[-1] // 2 - 1, 2, c.primes[-1] - 2]
    got = u32(c.mod_switch(dev(ct), L_out))
    assert got.shape == (n, 2, L_out, N)
    assert (got == oracle.mod_switch(ct, c.primes, L_out)).all()


def test_switched_conv_outputs_decrypt_under_the_small_context(fg, oracle):
    """Encrypt, convolve, mask, switch from 3 to 2 limbs, decrypt with a
    2-limb context: the shares still reconstruct conv2d mod t."""
    N, L, B = 8192, 3, 2
    c, c2 = ctx(fg, N, L), ctx(fg, N, 2)
    assert c2.primes == c.primes[:2]
    g = c.geom(16, 8, 16, 16, 3, 1, 1)
    geo = oracle.geometry(N, 16, 8, 16, 16, 3, 1, 1)
    s = synth.secret_key(81, N)
    sk, sk2 = c.keygen(dev(s, torch.int8)), c2.keygen(dev(s, torch.int8))
    x = synth.activations(81, (B, 16, 16, 16))
    w = synth.weights(81, (8, 16, 3, 3))
    ct = c.encrypt(sk, g, dev(x), dev(synth.uniform_residues(81, c.primes, (B, g.n_in, L, N))),
                   dev(synth.cbd_noise(81, (B, g.n_in, N))))
    r = synth.masks(81, (B, g.n_out, N), T)
    y = c.he_conv2d(g, c.encode_weights(g, dev(w, torch.int8)), ct, r=dev(r))
    ys = c.mod_switch(y, 2)
    assert (u32(ys)[0] == oracle.mod_switch(u32(y)[0], c.primes, 2)).all()
    m = u32(c2.decrypt(sk2, ys)).astype(np.int64)
    for b in range(B):
        share_sum = (m[b] + (T - r[b].astype(np.int64))) % T
        assert (oracle.extract_outputs(share_sum, geo) == oracle.conv2d_int(x[b], w, 1, 1) % T).all()


def test_mod_switch_arguments(fg):
    c = ctx(fg, 2048, 2)
    ct = torch.zeros((1, 2, 2, 2048), dtype=torch.int32, device="cuda")
    with pytest.raises(fg.FlashError, match="L_out"):
        c.mod_switch(ct, 3)
    with pytest.raises(fg.FlashError, match="overlap"):
        c.mod_switch(ct, 1, out=ct.view(-1)[:2 * 2048].view(1, 2, 1, 2048))
    assert c.mod_switch(torch.zeros((0, 2, 2, 2048), dtype=torch.int32, device="cuda"), 1).shape[0] == 0
