"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), vectorised in numpy.

Each call maps a 128-bit counter and a 64-bit key to four 32-bit words. A
round multiplies counter words 0 and 2 by two fixed odd constants (keeping
the high and low halves), mixes the high halves with the other two words
and the key, and the key is advanced by two Weyl constants between rounds.
The CUDA twin in csrc/qldscene.cu implements the same definition.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)
ROUNDS = 10


def philox4x32(c0, c1, c2, c3, k0, k1, rounds=ROUNDS):
    """Vectorised Philox4x32-R. Counter words are uint32-valued arrays (any
    shape, broadcast); key words are Python ints. Returns four uint32 arrays."""
    c0 = np.asarray(c0, np.uint64) & MASK32
    c1 = np.asarray(c1, np.uint64) & MASK32
    c2 = np.asarray(c2, np.uint64) & MASK32
    c3 = np.asarray(c3, np.uint64) & MASK32
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for r in range(rounds):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
        k0 = (k0 + W0) & 0xFFFFFFFF
        k1 = (k1 + W1) & 0xFFFFFFFF
    return (c0.astype(np.uint32), c1.astype(np.uint32), c2.astype(np.uint32), c3.astype(np.uint32))
