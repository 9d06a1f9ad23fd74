"""Philox4x32-10 counter-based RNG, written from Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11), Sec. 4.

State: a 128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1).  One
round multiplies c0 and c2 by two fixed odd constants, keeps the high and low
32-bit halves and mixes them with c1, c3 and the key; the key is advanced by
the Weyl constants between rounds.  Ten rounds give one 4x32-bit output.

Every random draw of the method is one output word of this function at a
counter that names what it is for (pixel or sample id, iteration, stream tag,
block), so the CUDA path and this oracle draw identical numbers.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = np.uint64(0xFFFFFFFF)

# stream tags (third counter word)
TAG_DEPTH = 0
TAG_POSE = 1
TAG_INIT = 2
# iteration word used by the bootstrap steps (before iteration 0)
ITER_BOOT = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words for the given counters and key.

    All arguments broadcast; results are uint32 arrays."""
    c0 = np.asarray(c0, np.uint64) & MASK
    c1 = np.asarray(c1, np.uint64) & MASK
    c2 = np.asarray(c2, np.uint64) & MASK
    c3 = np.asarray(c3, np.uint64) & MASK
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    for _ in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
        k0 = (k0 + W0) & 0xFFFFFFFF
        k1 = (k1 + W1) & 0xFFFFFFFF
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def seed_key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def u24_float(x):
    """Map a 32-bit word to a float32 in [0, 1): (x >> 8) * 2^-24 (exact)."""
    x = np.asarray(x, np.uint32)
    return (x >> np.uint32(8)).astype(np.float32) * np.float32(2.0 ** -24)


def index_pick(x, n):
    """Map a 32-bit word to an integer in [0, n): (x * n) >> 32 (exact)."""
    return (np.asarray(x, np.uint64) * np.uint64(n)) >> np.uint64(32)
