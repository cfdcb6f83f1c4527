"""Seeded synthetic inputs for the HE convolution path.

This module holds none of the method's arithmetic: it only draws random
integers.  Both the CUDA path and the CPU oracle take what it returns as
plain inputs, so the randomness the protocol draws (secret key, encryption
randomness and noise, server masks) is identical on both sides by
construction.

Distributions (Flash, arXiv 2401.16732, leaves them to SEAL; these are the
workload's stated choices):
* activations: uniform integers in [0, 255] (an 8-bit image / activation map)
* weights:     uniform integers in [-8, 7] (filters below 8 bits, Sec. 6.1)
* secret key:  uniform ternary {-1, 0, 1}
* noise e:     centred binomial, eta = 21 (difference of two Binomial(21, 1/2))
* a:           uniform residues in [0, q_l) for every RNS limb
* masks r:     uniform in [0, t)

Every array is drawn from its own stream, keyed by (seed, purpose, index), so
that adding a draw never changes another.
"""
from __future__ import annotations

import numpy as np

ACT, WEIGHT, SECRET, NOISE, UNIFORM_A, MASK, RAW = range(1, 8)


def rng(seed: int, purpose: int, *index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, purpose, *index])))


def activations(seed: int, shape, *index) -> np.ndarray:
    return rng(seed, ACT, *index).integers(0, 256, size=shape, dtype=np.int64).astype(np.int32)


def weights(seed: int, shape, *index) -> np.ndarray:
    return rng(seed, WEIGHT, *index).integers(-8, 8, size=shape, dtype=np.int64).astype(np.int8)


def secret_key(seed: int, N: int) -> np.ndarray:
    return rng(seed, SECRET).integers(-1, 2, size=N, dtype=np.int64).astype(np.int8)


def cbd_noise(seed: int, shape, *index, eta: int = 21) -> np.ndarray:
    g = rng(seed, NOISE, *index)
    return (g.binomial(eta, 0.5, size=shape) - g.binomial(eta, 0.5, size=shape)).astype(np.int32)


def uniform_residues(seed: int, primes, shape, *index) -> np.ndarray:
    """[*shape][L][N]-shaped draw where the last two axes are (limb, coeff):
    shape = (..., L, N) and limb l is uniform in [0, primes[l])."""
    g = rng(seed, UNIFORM_A, *index)
    out = np.empty(shape, np.uint32)
    for l, ql in enumerate(primes):
        out[..., l, :] = g.integers(0, ql, size=shape[:-2] + shape[-1:], dtype=np.int64)
    return out


def masks(seed: int, shape, t: int, *index) -> np.ndarray:
    return rng(seed, MASK, *index).integers(0, t, size=shape, dtype=np.int64).astype(np.uint32)


def raw_ciphertexts(seed: int, primes, shape, *index) -> np.ndarray:
    """Uniform residues shaped like ciphertexts [..., 2, L, N]; the homomorphic
    convolution is a linear map on polynomials, so uniform inputs exercise it
    over the full 30-bit residue range."""
    g = rng(seed, RAW, *index)
    out = np.empty(shape, np.uint32)
    for l, ql in enumerate(primes):
        out[..., l, :] = g.integers(0, ql, size=shape[:-2] + shape[-1:], dtype=np.int64)
    return out


# ---------------------------------------------------------------------------
# Device-side draws for large benchmark inputs (same distributions; a seeded
# torch generator on the device instead of numpy on the host).
# ---------------------------------------------------------------------------
def _torch_gen(seed: int, purpose: int, *index: int, device="cuda"):
    import torch
    ss = np.random.SeedSequence([seed, purpose, *index]).generate_state(2, np.uint32)
    g = torch.Generator(device=device)
    g.manual_seed(int(ss[0]) << 32 | int(ss[1]))
    return g


def device_uniform_residues(seed: int, primes, shape, *index, device="cuda"):
    """int32 tensor [..., L, N] on `device`, limb l uniform in [0, primes[l])."""
    import torch
    g = _torch_gen(seed, UNIFORM_A, *index, device=device)
    out = torch.empty(shape, dtype=torch.int32, device=device)
    for l, ql in enumerate(primes):
        out[..., l, :] = torch.randint(0, int(ql), shape[:-2] + shape[-1:], generator=g, device=device,
                                       dtype=torch.int64).to(torch.int32)
    return out


def device_masks(seed: int, shape, t: int, *index, device="cuda"):
    import torch
    g = _torch_gen(seed, MASK, *index, device=device)
    return torch.randint(0, t, shape, generator=g, device=device, dtype=torch.int32)


def device_cbd_noise(seed: int, shape, *index, eta: int = 21, device="cuda"):
    import torch
    g = _torch_gen(seed, NOISE, *index, device=device)
    n = torch.full(shape, float(eta), device=device)
    p = torch.full(shape, 0.5, device=device)
    return (torch.binomial(n, p, generator=g) - torch.binomial(n, p, generator=g)).to(torch.int32)
