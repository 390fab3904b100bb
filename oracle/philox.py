"""Philox4x32-10 counter-based block function, numpy reference.

Definition: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11 (Philox-4x32, 10 rounds).

A round maps the counter (c0, c1, c2, c3) under key (k0, k1) to

    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))

with 32x32->64 bit products, and the key is bumped by the Weyl constants
between rounds.  Pins (tests/test_oracle_philox.py): cuRAND's own
PHILOX4_32_10 host generator (run, not read) and the all-zero known answer.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF
ROUNDS = 10


def philox4x32(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.

    All arguments are integers or numpy integer arrays holding values in
    [0, 2^32); they broadcast together.  Returns four uint64 arrays whose
    values are the four 32-bit output words.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & np.uint64(MASK32)
    c1 = np.asarray(c1, dtype=np.uint64) & np.uint64(MASK32)
    c2 = np.asarray(c2, dtype=np.uint64) & np.uint64(MASK32)
    c3 = np.asarray(c3, dtype=np.uint64) & np.uint64(MASK32)
    k0 = np.asarray(k0, dtype=np.uint64) & np.uint64(MASK32)
    k1 = np.asarray(k1, dtype=np.uint64) & np.uint64(MASK32)
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    c0, c1, c2, c3 = c0.copy(), c1.copy(), c2.copy(), c3.copy()
    k0, k1 = k0.copy(), k1.copy()
    m32 = np.uint64(MASK32)
    s32 = np.uint64(32)
    for r in range(ROUNDS):
        if r > 0:
            k0 = (k0 + np.uint64(W0)) & m32
            k1 = (k1 + np.uint64(W1)) & m32
        p0 = np.uint64(M0) * c0          # < 2^64: no overflow
        p1 = np.uint64(M1) * c2
        n0 = (p1 >> s32) ^ c1 ^ k0
        n1 = p1 & m32
        n2 = (p0 >> s32) ^ c3 ^ k1
        n3 = p0 & m32
        c0, c1, c2, c3 = n0, n1, n2, n3
    return c0, c1, c2, c3


def philox_scalar(ctr, key):
    """Scalar convenience form: ctr = 4 ints, key = 2 ints -> tuple of 4 ints."""
    out = philox4x32(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1])
    return tuple(int(o) for o in out)


def seed_key(seed: int):
    """64-bit seed -> Philox key words (low, high)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & MASK32, seed >> 32
