"""Shared random-stream specification, oracle side (test infrastructure only).

The paper samples its independent symbols (noise choices s and random
measurement bits m1, Sec. 5, symbol classes; Sec. 6, sampling of
independent symbols) but fixes no generator, seed layout or stream order.
To compare samplers shot by shot, every sampler here (state vector, tableau,
plain SymFT, CUDA) draws from one counter-based specification, written out
independently on each side:

Key      Philox key = (seed & 0xffffffff, seed >> 32).

Noise    Channel ordinal c (circuit order, after REPEAT unrolling), shot block
         b = shot >> 9 (NOISE_BLOCK = 512 shots, lanes 0..511).
         head draw          = Philox(c >> 2, b, 0, TAG_HEAD)[c & 3]
         tail draw i (>= 0) = Philox(c, b, i >> 2, TAG_TAIL)[i & 3]
         Block-geometric process: L = 0, u = head draw;
           j* = min{ j in [0, 511 - L] : u < THETA_j }, stop if none;
           the channel fires on lane L + j*; if it has more than one Pauli
           cell the next tail draw v picks cell min{ k : v < PHI_k };
           L = L + j* + 1 (stop at 512); u = next tail draw; repeat.
         The block length is a choice of this specification (the paper
         samples sparse noise by geometric gaps, Sec. 6, and fixes no block):
         512 lanes make one head draw cover ~0.5 expected fires at q = 1e-3.
         THETA_j = min(floor((1 - r^(j+1)) * 2^32), 2^32 - 1), r = 1 - q,
         r^(j+1) by repeated multiplication in FP64; q = the channel's total
         error probability.  PHI_k = min(floor(W_k / W * 2^32), 2^32 - 1)
         with W_k the running FP64 sum of cell weights 0..k in order and W
         their total; the last cell takes every v >= PHI_{K-2}.
         This is i.i.d. Bernoulli(q) per shot up to the 2^-32 quantisation.

Measure  Measurement ordinal t (every measurement event in circuit order,
         recorded or hidden), shot r:
           MBIT word (t, w)  = Philox(t, (w >> 1), w >> 33, TAG_MBIT),
                               words (o0 | o1 << 32) for even w,
                               (o2 | o3 << 32) for odd w;  w = r >> 6
           F(t, r)           = 52 high bits of the 64-bit word
                               Philox(t, (r >> 1), r >> 33, TAG_MFRAC)
                               [(o0 | o1 << 32) even r, (o2 | o3 << 32) odd r]
           u(t, r)           = (bit_{r & 63}(MBIT(t, r >> 6)) * 2^52 + F) * 2^-53
         Rule: the recorded bit is 0 iff u(t, r) < Pr(m_t = 0).  With
         Pr = 1/2 this is the MBIT bit itself, so a uniformly random
         measurement needs only the packed MBIT word.

Pins: tests/test_oracle_streams.py checks the first-fire law against brute
force enumeration of the thresholds, lane marginals against Bernoulli(q),
pairwise lane independence, and the u construction against its definition
at the boundary cases (Pr = 1/2, 0, 1).
"""
from __future__ import annotations

from bisect import bisect_right

import numpy as np

from .philox import philox4x32, seed_key

NOISE_BLOCK = 512
TAG_HEAD = 1
TAG_TAIL = 2
TAG_MBIT = 3
TAG_MFRAC = 4
TWO32 = 4294967296.0


def theta_table(q: float) -> list[int]:
    """THETA_j, j = 0..NOISE_BLOCK-1, for a channel with total error probability q."""
    r = 1.0 - float(q)
    out = []
    rp = r
    for _ in range(NOISE_BLOCK):
        v = (1.0 - rp) * TWO32
        iv = int(np.floor(v))
        out.append(min(iv, 0xFFFFFFFF))
        rp = rp * r
    return out


def phi_table(weights) -> list[int]:
    """PHI_k for k = 0..K-2 from the cell weights (empty for K = 1)."""
    w = [float(x) for x in weights]
    total = 0.0
    for x in w:
        total = total + x
    out = []
    run = 0.0
    for k in range(len(w) - 1):
        run = run + w[k]
        v = run / total * TWO32
        out.append(min(int(np.floor(v)), 0xFFFFFFFF))
    return out


def _word(o_a, o_b):
    return int(o_a) | (int(o_b) << 32)


def head_draw(seed: int, c: int, b: int) -> int:
    k0, k1 = seed_key(seed)
    o = philox4x32(c >> 2, b & 0xFFFFFFFF, 0, TAG_HEAD, k0, k1)
    return int(o[c & 3])


def tail_draw(seed: int, c: int, b: int, i: int) -> int:
    k0, k1 = seed_key(seed)
    o = philox4x32(c & 0xFFFFFFFF, b & 0xFFFFFFFF, i >> 2, TAG_TAIL, k0, k1)
    return int(o[i & 3])


def channel_block_fires(seed: int, c: int, b: int, theta, phi):
    """Run the block-geometric process for channel c on shot block b.

    Returns a list of (lane, cell) pairs in increasing lane order.  The first
    index j with u < THETA_j is found by bisection: THETA is non-decreasing,
    so it is the number of entries <= u (the linear scan of the definition
    gives the same index).
    """
    fires = []
    if theta[NOISE_BLOCK - 1] == 0:
        return fires
    L = 0
    u = head_draw(seed, c, b)
    i = 0
    while True:
        jstar = bisect_right(theta, u)
        if jstar > NOISE_BLOCK - 1 - L:
            break
        lane = L + jstar
        cell = 0
        if len(phi) > 0:
            v = tail_draw(seed, c, b, i)
            i += 1
            cell = len(phi)
            for k in range(len(phi)):
                if v < phi[k]:
                    cell = k
                    break
        fires.append((lane, cell))
        L = lane + 1
        if L >= NOISE_BLOCK:
            break
        u = tail_draw(seed, c, b, i)
        i += 1
    return fires


def mbit_word(seed: int, t: int, w: int) -> int:
    k0, k1 = seed_key(seed)
    o = philox4x32(t & 0xFFFFFFFF, (w >> 1) & 0xFFFFFFFF, w >> 33, TAG_MBIT, k0, k1)
    if w & 1:
        return _word(o[2], o[3])
    return _word(o[0], o[1])


def mbit_words(seed: int, t: int, w_lo: int, n_words: int) -> np.ndarray:
    """Vectorised MBIT words for w in [w_lo, w_lo + n_words)."""
    k0, k1 = seed_key(seed)
    w = np.arange(w_lo, w_lo + n_words, dtype=np.uint64)
    o = philox4x32(np.uint64(t & 0xFFFFFFFF), (w >> np.uint64(1)) & np.uint64(0xFFFFFFFF),
                   w >> np.uint64(33), TAG_MBIT, k0, k1)
    even = o[0] | (o[1] << np.uint64(32))
    odd = o[2] | (o[3] << np.uint64(32))
    return np.where((w & np.uint64(1)) == 1, odd, even).astype(np.uint64)


def mfrac(seed: int, t: int, r: int) -> int:
    k0, k1 = seed_key(seed)
    o = philox4x32(t & 0xFFFFFFFF, (r >> 1) & 0xFFFFFFFF, r >> 33, TAG_MFRAC, k0, k1)
    word = _word(o[2], o[3]) if (r & 1) else _word(o[0], o[1])
    return word >> 12


def meas_uniform(seed: int, t: int, r: int) -> float:
    """u(t, r) in [0, 1) exactly as specified (a multiple of 2^-53)."""
    bit = (mbit_word(seed, t, r >> 6) >> (r & 63)) & 1
    f = mfrac(seed, t, r)
    return float(bit * (1 << 52) + f) * 2.0 ** -53


def outcome_from(p0: float, u: float) -> int:
    """The recorded bit: 0 iff u < Pr(m = 0)."""
    return 0 if u < p0 else 1
