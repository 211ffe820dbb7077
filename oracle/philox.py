"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).

Written from the published definition: a 128-bit counter (four 32-bit words)
and a 64-bit key (two words) go through 10 rounds.  Each round multiplies
words 0 and 2 by the two Philox multipliers, keeps the 64-bit products split
into high/low halves, and permutes/XORs them with words 1, 3 and the key; the
key is bumped by the two Weyl constants between rounds.

Stream layout used by both sides of the sketch (a text specification, not
shared code):  key = (seed & 0xffffffff, seed >> 32),
counter = (index & 0xffffffff, index >> 32, stream, 0).

Streams:  3 = CountSketch/SJLT bucket and sign, 5 = Gaussian sketch entries,
6 = SRHT diagonal signs, 7 = SRHT row-selection keys.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)

STREAM_COUNTSKETCH = 3
STREAM_GAUSSIAN = 5
STREAM_SRHT_SIGN = 6
STREAM_SRHT_KEY = 7


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  Inputs are uint32-valued arrays/scalars; returns 4 uint32 arrays."""
    c0 = np.asarray(c0, dtype=np.uint64)
    c1 = np.asarray(c1, dtype=np.uint64)
    c2 = np.asarray(c2, dtype=np.uint64)
    c3 = np.asarray(c3, dtype=np.uint64)
    k0 = np.uint64(k0)
    k1 = np.uint64(k1)
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0            # < 2^64: exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return (c0.astype(np.uint32), c1.astype(np.uint32), c2.astype(np.uint32),
            c3.astype(np.uint32))


def draw(seed: int, stream: int, index):
    """Four 32-bit words for each 64-bit `index` on `stream` under `seed`."""
    idx = np.asarray(index, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return philox4x32_10(idx & MASK, idx >> np.uint64(32), np.full(idx.shape, stream, np.uint64),
                         np.zeros(idx.shape, np.uint64), seed & 0xFFFFFFFF, seed >> 32)


def uniform_open(w):
    """Map a 32-bit word to the open interval (0, 1): (w + 1/2) * 2^-32."""
    return (np.asarray(w, dtype=np.float64) + 0.5) * (2.0 ** -32)
