"""Per-shot Pauli noise drawn from the shared stream specification (oracle side).

Test infrastructure only.  For each noise channel of a parsed circuit and each
512-shot block, the block-geometric process of ``oracle.streams`` yields the
(lane, cell) fire list; this module turns it into "shot r applies Pauli cell k
of channel c".  The Pauli noise channel itself is the one of Sec. 2
(N(rho) = sum_j p_j N_j rho N_j): a fired cell k applies N_k, no fire applies I.
"""
from __future__ import annotations

from functools import lru_cache

from .streams import NOISE_BLOCK, channel_block_fires, phi_table, theta_table


class NoiseSampler:
    def __init__(self, circuit, seed: int):
        self.seed = int(seed)
        self.channels = [op for op in circuit.ops if op.kind == "noise"]
        self._tables = {}
        for op in self.channels:
            key = (op.q, op.weights)
            if key not in self._tables:
                self._tables[key] = (theta_table(op.q), phi_table(op.weights))
        self._cache = {}

    def block(self, b: int):
        """{channel ordinal: {lane: cell}} for shot block b (cached)."""
        if b in self._cache:
            return self._cache[b]
        out = {}
        for op in self.channels:
            th, ph = self._tables[(op.q, op.weights)]
            fires = channel_block_fires(self.seed, op.c, b, th, ph)
            if fires:
                out[op.c] = dict(fires)
        if len(self._cache) > 64:
            self._cache.clear()
        self._cache[b] = out
        return out

    def shot(self, r: int):
        """{channel ordinal: cell} of the channels that fire on shot r."""
        blk = self.block(r // NOISE_BLOCK)
        lane = r % NOISE_BLOCK
        return {c: lanes[lane] for c, lanes in blk.items() if lane in lanes}
