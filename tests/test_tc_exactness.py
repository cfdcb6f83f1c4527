"""The integer arithmetic of the tensor-core form, emulated on the CPU with
fp32 rounding (numpy float32), so that the exactness argument of
fl_he_conv2d_tc is checked without a GPU: balanced base-256 digits sum back
to the residue; fp32 sums of digit products stay exact up to G = 64 input
ciphertexts (the bias 3 * 2^22 keeps every partial sum in [2^23, 2^24]); and
the recombination of the four digit sums gives a value congruent to Y mod q
in [0, 2q) for every prime a context can hold, at the extremes of the sums
and on random ones."""
import numpy as np

import oracle

FP_BIAS = 0x4B400000        # bits of 3 * 2^22 in fp32
BIAS = 3 * (1 << 22)


def digits(v):
    """Balanced base-256 digits d_a(v) = byte_a(v + 0x80808080) - 128."""
    y = (v.astype(np.uint64) + 0x80808080) & 0xFFFFFFFF
    return np.stack([((y >> (8 * a)) & 255).astype(np.int64) - 128 for a in range(4)], axis=-1)


def f32_fma(a, b, c):
    """fmaf on float32 operands: a * b + c exact in float64 here (< 2^53),
    rounded once to float32."""
    return (a.astype(np.float64) * b + c.astype(np.float64)).astype(np.float32)


def recombine(P, q):
    """The kernel's recombination of the digit sums P[..., e] (e = 0..3),
    from the accumulators' fp32 values (3 * 2^22 + P) and bit patterns."""
    val = (P + BIAS).astype(np.float32)
    bits = (P + FP_BIAS).astype(np.int64)
    assert (val.view(np.uint32).astype(np.int64) == bits).all()  # the bias puts every sum in [2^23, 2^24]
    k123 = np.float32(12582912.0 * 16843008.0)
    assert float(k123) == 12582912.0 * 16843008.0
    y = f32_fma(val[..., 3], 16777216.0, np.full(P.shape[:-1], -k123, np.float32))
    y = f32_fma(val[..., 2], 65536.0, y)
    y = f32_fma(val[..., 1], 256.0, y)
    kb = f32_fma(y, np.float64(np.float32(1.0 / q)), np.full(y.shape, 12582912.0, np.float32))
    kb = kb.view(np.uint32).astype(np.int64)
    lo = (bits[..., 0] + (bits[..., 1] << 8) + (bits[..., 2] << 16) + (bits[..., 3] << 24)) & 0xFFFFFFFF
    c = (FP_BIAS * q + q - FP_BIAS * 0x01010101) & 0xFFFFFFFF
    return (kb * ((-q) & 0xFFFFFFFF) + lo + c) & 0xFFFFFFFF


def shoup(x, w, q):
    """Shoup's product as the kernel computes it: x w - floor(x w' / 2^32) q
    with w' = floor(w 2^32 / q)."""
    wsh = (w << 32) // q
    return x * w - ((x * wsh) >> 32) * q


def test_digits_sum_back_below_the_wrap_and_every_split_value_is_below_it():
    """The split is exact for v < 0x7F7F7F80 (v + 0x80808080 below 2^32) and
    wraps from there on; the values the kernel splits, residues below q and
    Shoup products of them (X'_a), stay below 1.25 q < 0x7F7F7F80 for every
    prime a context can hold."""
    rng = np.random.default_rng(1)
    lim = 0x7F7F7F80
    v = np.concatenate([rng.integers(0, lim, 100000), [0, 1, 0x7F7F7F7F, lim - 1]])
    d = digits(v)
    assert d.min() >= -128 and d.max() <= 127
    assert (sum(d[:, a] << (8 * a) for a in range(4)) == v).all()
    assert sum(int(x) << (8 * a) for a, x in enumerate(digits(np.array([lim]))[0])) != lim  # the wrap
    for N, L in ((2048, 1), (16384, 4)):
        for q in oracle.find_primes(N, L):
            assert 5 * q // 4 < lim
            x = [int(xi) for xi in rng.integers(0, q, 20000)] + [0, 1, q - 1]
            for a in (1, 2, 3):
                r = [shoup(xi, 256 ** a, q) for xi in x]
                assert all(0 <= ri < 5 * q // 4 for ri in r)
                assert all((ri - xi * 256 ** a) % q == 0 for ri, xi in zip(r, x))


def test_fp32_digit_sums_are_exact_up_to_64_ciphertexts():
    """K = 4G digit products per sum: at G = 64 the extreme sums reach
    +-2^22, and 3 * 2^22 + P stays an exact fp32 integer whatever the order
    of the additions (every partial sum lies in [2^23, 2^24])."""
    G = 64
    rng = np.random.default_rng(2)
    for w, x in ((-128, -128), (127, -128), (-128, 127), (127, 127)):
        prods = np.full(4 * G, w * x, dtype=np.int64)
        acc = np.float32(BIAS)
        for p in prods:  # one order; all partial sums are integers below 2^24
            acc = np.float32(acc + np.float32(p))
            assert 1 << 23 <= acc <= 1 << 24 and acc == np.round(acc)
        assert int(acc) - BIAS == int(prods.sum())
    for _ in range(50):
        prods = rng.integers(-128, 128, 4 * G) * rng.integers(-128, 128, 4 * G)
        order = rng.permutation(4 * G)
        acc = np.float32(BIAS)
        for p in prods[order]:
            acc = np.float32(acc + np.float32(p))
        assert int(acc) - BIAS == int(prods.sum())


def test_recombination_is_exact_mod_q_in_0_2q():
    lim = 1 << 22
    ext = np.array(np.meshgrid(*[[-lim, -lim + 1, 0, lim - 1, lim]] * 4)).reshape(4, -1).T
    rng = np.random.default_rng(3)
    rnd = rng.integers(-lim, lim + 1, size=(100000, 4))
    for N, L in ((2048, 1), (8192, 3), (16384, 4)):
        for q in oracle.find_primes(N, L):
            for P in (ext, rnd):
                r = recombine(P, q)
                Y = P[:, 0] + (P[:, 1] << 8) + (P[:, 2] << 16) + (P[:, 3] << 24)
                assert (r < 2 * q).all()
                assert ((r - Y) % q == 0).all()


def test_recombination_of_real_products_gives_the_modular_product_sum():
    """End to end on digits: W, X residues mod q, X'_a = 256^a X mod q, the
    digit sums P_e = sum_(g,a) d_a(W_g) d_e(X'_a,g), recombined, equal
    sum_g W_g X_g mod q (up to one q)."""
    rng = np.random.default_rng(4)
    q = oracle.find_primes(16384, 4)[3]
    G = 64
    W = rng.integers(0, q, size=(500, G))
    X = rng.integers(0, q, size=(500, G))
    W[0], X[0] = q - 1, q - 1
    Xp = np.stack([(X * pow(256, a, q)) % q for a in range(4)], axis=-1)  # [n][g][a]
    dW = digits(W)                                                        # [n][g][a]
    dX = digits(Xp.reshape(-1)).reshape(500, G, 4, 4)                     # [n][g][a][e]
    P = np.einsum("nga,ngae->ne", dW, dX)
    assert np.abs(P).max() <= G << 16
    r = recombine(P, q)
    want = (W.astype(object) * X.astype(object)).sum(axis=1) % q
    assert all(int(a) % q == int(b) for a, b in zip(r, want))
    assert (r < 2 * q).all()
