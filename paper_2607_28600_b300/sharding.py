"""Shot-range sharding across ranks (host logic only).

Shots are independent and every random draw is keyed by the absolute shot
index (counter-based streams), so a sample set splits into contiguous shot
ranges that separate calls -- on one GPU or on several -- produce bit for bit
as one call would.  Ranges start on multiples of SHOT_ALIGN (the noise block
of the stream specification), the alignment every sampling call requires.
"""
from __future__ import annotations

from . import SHOT_ALIGN


def shard_range(total: int, rank: int, world: int) -> tuple[int, int]:
    """(shot_offset, shots) of `rank` when `world` ranks share shots [0, total).

    Whole noise blocks are dealt out as evenly as possible; the last rank
    also takes the ragged tail.  A rank may get zero shots when there are
    fewer blocks than ranks.
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    if total < 0:
        raise ValueError("total must be >= 0")
    blocks = total // SHOT_ALIGN
    lo = rank * blocks // world
    hi = (rank + 1) * blocks // world
    start = lo * SHOT_ALIGN
    end = total if rank == world - 1 else hi * SHOT_ALIGN
    return start, end - start


def weak_offset(shots_per_rank: int, rank: int) -> int:
    """First shot of `rank` when every rank samples `shots_per_rank` shots of
    one common sample set (weak scaling): disjoint ranges on aligned starts."""
    if shots_per_rank < 0 or rank < 0:
        raise ValueError("need shots_per_rank >= 0 and rank >= 0")
    per = -(-shots_per_rank // SHOT_ALIGN) * SHOT_ALIGN
    return rank * per
