"""Philox4x64-10 counter-based generator, written from its published definition.

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py; the product path never imports anything under oracle/.

Definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11, Sec. 3.2): a 4-word counter (c0, c1, c2, c3) and a 2-word key
(k0, k1) of 64-bit words go through 10 rounds.  One round multiplies c0 and c2
by the constants M0 and M1 into 128-bit products (hi, lo) and outputs
    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0));
between rounds the key is bumped by the Weyl constants (W0, W1) modulo 2^64.

RBRP draws one uniform per (row, block): counter = (row, block, 0, 0), key =
(seed, problem), and the uniform is u = ((w0 >> 11) + 1/2) * 2^-53, which lies
in the open interval (0, 1) so that -log(u) is finite and positive.

Pin: numpy.random.Philox is the same generator; its random_raw() advances the
counter by one before producing each 4-word block, so
philox4x64_10(c, k) == Philox(counter=c - 1, key=k).random_raw(4)
(tests/test_oracle_philox.py).
"""
import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
ROUNDS = 10
_MASK64 = (1 << 64) - 1


def philox4x64_10_scalar(ctr, key):
    """One 4-word Philox4x64-10 output block with Python integers (slow, tiny cases)."""
    c = [int(x) & _MASK64 for x in ctr]
    k = [int(x) & _MASK64 for x in key]
    for _ in range(ROUNDS):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [(p1 >> 64) ^ c[1] ^ k[0], p1 & _MASK64, (p0 >> 64) ^ c[3] ^ k[1], p0 & _MASK64]
        k = [(k[0] + W0) & _MASK64, (k[1] + W1) & _MASK64]
    return c


def _mulhilo(a_const, b):
    """128-bit product of a 64-bit constant and a uint64 array, as (hi, lo) uint64 arrays.

    Built from 32-bit limbs so that every partial product fits in 64 bits.
    """
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    aL = np.uint64(a_const & 0xFFFFFFFF)
    aH = np.uint64(a_const >> 32)
    bL = b & m32
    bH = b >> s32
    p0 = aL * bL
    p1 = aL * bH
    p2 = aH * bL
    p3 = aH * bH
    mid = (p0 >> s32) + (p1 & m32) + (p2 & m32)
    hi = p3 + (p1 >> s32) + (p2 >> s32) + (mid >> s32)
    lo = (mid << s32) | (p0 & m32)
    return hi, lo


def philox4x64_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x64-10 over broadcastable uint64 arrays; returns (w0, w1, w2, w3)."""
    with np.errstate(over="ignore"):
        c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(*(np.asarray(x, dtype=np.uint64) for x in (c0, c1, c2, c3, k0, k1)))
        c0, c1, c2, c3, k0, k1 = (np.array(x, dtype=np.uint64) for x in (c0, c1, c2, c3, k0, k1))
        w0c, w1c = np.uint64(W0), np.uint64(W1)
        for _ in range(ROUNDS):
            hi0, lo0 = _mulhilo(M0, c0)
            hi1, lo1 = _mulhilo(M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            k0 = k0 + w0c
            k1 = k1 + w1c
    return c0, c1, c2, c3


def uniforms(rows, block, seed, problem=0):
    """u(row, block) in (0, 1) for RBRP's sampler: counter (row, block, 0, 0), key (seed, problem)."""
    rows = np.asarray(rows, dtype=np.uint64)
    w0, _, _, _ = philox4x64_10(rows, np.uint64(block), np.uint64(0), np.uint64(0),
                                np.uint64(seed), np.uint64(problem))
    return ((w0 >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
