"""Philox4x32-10 counter-based generator, vectorised over numpy arrays.

Written from the published definition (Salmon et al., SC'11, Section 4.2):
a 4x32-bit counter and a 2x32-bit key; each of the 10 rounds multiplies
counter words 0 and 2 by two fixed 32-bit constants, XORs the high halves
into the opposite words together with the round key, and permutes the words;
the key is advanced by two Weyl constants between rounds.
"""
import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def _mulhilo(a, x):
    """(hi, lo) 32-bit halves of the 64-bit product a*x, a a Python int."""
    p = np.uint64(a) * x.astype(np.uint64)
    return (p >> np.uint64(32)).astype(np.uint32), (p & _MASK).astype(np.uint32)


def philox4x32_10(c0, c1, c2, c3, k0, k1, rounds=10):
    """Apply Philox4x32 with ``rounds`` rounds to counters (c0..c3), key (k0, k1).

    All counter arguments are broadcastable uint32 arrays (or ints); the key
    words are ints.  Returns four uint32 arrays (x0, x1, x2, x3).
    """
    x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64).astype(np.uint32) for c in (c0, c1, c2, c3))
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    ka, kb = int(k0) & 0xFFFFFFFF, int(k1) & 0xFFFFFFFF
    for _ in range(rounds):
        hi0, lo0 = _mulhilo(PHILOX_M0, x0)
        hi1, lo1 = _mulhilo(PHILOX_M1, x2)
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint32(ka), lo1,
                          hi0 ^ x3 ^ np.uint32(kb), lo0)
        ka = (ka + PHILOX_W0) & 0xFFFFFFFF
        kb = (kb + PHILOX_W1) & 0xFFFFFFFF
    return x0, x1, x2, x3
