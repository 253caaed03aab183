"""The byte arithmetic the point test runs on 16-bit lanes, checked on the CPU.

The engines take the per-byte maximum (alpha^-, the largest lower
neighbour), the per-byte saturated c - lambda and c + lambda, and their
16-bit-lane forms for u16 pixels, through 16-bit lane minima and maxima:
a word's even bytes (mask 0x00ff00ff) and odd bytes (0xff00ff00), each left
in place, are two pairs of 16-bit lanes whose order is the bytes' order.
These are identities of integer arithmetic; this test restates each one with
plain lane operations and checks it against per-byte arithmetic on random
words and on the edge values (0, 255, lambda >= 255).  The GPU parity tests
check the compiled kernels themselves."""
import numpy as np

E8, O8 = 0x00FF00FF, 0xFF00FF00
M32 = 0xFFFFFFFF


def lanes(x):
    return x & 0xFFFF, (x >> 16) & 0xFFFF


def vmin2(a, b):
    (a0, a1), (b0, b1) = lanes(a), lanes(b)
    return np.minimum(a0, b0) | (np.minimum(a1, b1) << 16)


def vmax2(a, b):
    (a0, a1), (b0, b1) = lanes(a), lanes(b)
    return np.maximum(a0, b0) | (np.maximum(a1, b1) << 16)


def subus8(c, l):
    ce, co = c & E8, c & O8
    return ((ce - vmin2(ce, l & E8)) & M32) | ((co - vmin2(co, l & O8)) & M32)


def addus8(c, l):
    nc = ~c & M32
    return (((c & E8) + vmin2(l & E8, nc & E8)) & M32) | (((c & O8) + vmin2(l & O8, nc & O8)) & M32)


def alpha4(nb, M):
    e = o = np.zeros_like(M)
    for d in range(8):
        v = nb[d] & ((((M >> d) & 0x01010101) * 0xFF) & M32)
        e = vmax2(e, v & E8)
        o = vmax2(o, v & O8)
    return e | o


def bytes_of(x):
    return [(x >> (8 * k)) & 0xFF for k in range(4)]


def word(bs):
    return sum(b.astype(np.uint64) << np.uint64(8 * k) for k, b in enumerate(bs))


def test_saturated_byte_offsets():
    rng = np.random.default_rng(5)
    c = rng.integers(0, 1 << 32, 50000, dtype=np.uint64)
    c[:4] = [0, M32, 0x00FF00FF, 0xFF00FF00]
    for lam in (0, 1, 5, 20, 127, 128, 254, 255):
        l = np.uint64(lam * 0x01010101)
        sub = word([np.maximum(b.astype(np.int64) - lam, 0).astype(np.uint64) for b in bytes_of(c)])
        add = word([np.minimum(b + np.uint64(lam), np.uint64(255)) for b in bytes_of(c)])
        assert np.array_equal(subus8(c, l), sub)
        assert np.array_equal(addus8(c, l), add)


def test_largest_lower_neighbour():
    rng = np.random.default_rng(6)
    n = 20000
    nb = [rng.integers(0, 1 << 32, n, dtype=np.uint64) for _ in range(8)]
    M = rng.integers(0, 1 << 32, n, dtype=np.uint64)
    M[:2] = [0, M32]  # no lower neighbour; all eight lower
    got = alpha4(nb, M)
    ref = word([np.max(np.stack([np.where((M >> np.uint64(8 * k + d)) & np.uint64(1), (nb[d] >> np.uint64(8 * k)) & np.uint64(255), 0)
                                 for d in range(8)]), axis=0).astype(np.uint64) for k in range(4)])
    assert np.array_equal(got, ref)


def test_u16_lane_offsets():
    rng = np.random.default_rng(7)
    c = rng.integers(0, 1 << 32, 50000, dtype=np.uint64)
    c[:3] = [0, M32, 0x0000FFFF]
    for lam in (0, 1, 80, 320, 4095, 65535):
        l = np.uint64(lam * 0x00010001)
        lo, hi = lanes(c)
        sub = (c - vmin2(c, l)) & M32  # c - min(c, lambda) per lane
        add = (c + vmin2(l, ~c & M32)) & M32  # c + min(lambda, 65535 - c) per lane
        assert np.array_equal(sub, np.maximum(lo.astype(np.int64) - lam, 0).astype(np.uint64)
                              | (np.maximum(hi.astype(np.int64) - lam, 0).astype(np.uint64) << np.uint64(16)))
        assert np.array_equal(add, np.minimum(lo + np.uint64(lam), np.uint64(65535))
                              | (np.minimum(hi + np.uint64(lam), np.uint64(65535)) << np.uint64(16)))
