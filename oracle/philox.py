"""Counter-based random numbers for the seeing (PSF) displacement (oracle;
test infrastructure only).

Philox4x32 with 10 rounds as published by Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): a 128-bit counter
(four 32-bit words) and a 64-bit key (two words); each round multiplies
counter words 0 and 2 by the two round constants of that publication,
takes the high and low halves of the 64-bit products, mixes the high
halves with the other counter words and the key, and then advances the
key by the two Weyl constants.  The GPU path implements the same published
definition independently; the two agree bit for bit on every draw.
"""
import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57          # round multipliers
W0, W1 = 0x9E3779B9, 0xBB67AE85          # key increments (Weyl sequence)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Four uint32 arrays (broadcast together) of the counter, two uint32
    key words; returns the four output words as uint32 arrays."""
    c = [np.asarray(v, dtype=np.uint64) & _MASK for v in np.broadcast_arrays(c0, c1, c2, c3)]
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = np.uint64(M0) * c[0]          # < 2^64: exact in uint64
        p1 = np.uint64(M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        k0 = (k0 + np.uint64(W0)) & _MASK
        k1 = (k1 + np.uint64(W1)) & _MASK
    return [v.astype(np.uint32) for v in c]
