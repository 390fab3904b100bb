"""Records, detectors, observables and the postselection rule (oracle side).

Test infrastructure only.  Detectors and observables are parities of recorded
measurement outcomes (DETECTOR / OBSERVABLE_INCLUDE annotations of the
Stim-style input, Sec. 7).  Postselection (Sec. 6, detector postselection)
rejects a shot at the first postselected detector, in annotation order, whose
parity is 1; rejected shots keep every bit produced up to and including that
detector and report zeros afterwards:

  * record bits whose record index is >= the number of records that existed
    when the rejecting DETECTOR line was reached are 0,
  * detector bits with a larger detector index are 0 (the rejecting detector
    itself reads 1),
  * all observable bits are 0, and the discard flag is 1.

Modes: POSTSELECT_NONE (0) never rejects, POSTSELECT_ALL (1) postselects every
detector, POSTSELECT_LISTED (2) postselects the detectors whose indices are
given; the others are still reported (and zeroed after a rejection) but never
reject.
"""
from __future__ import annotations

import numpy as np

POSTSELECT_NONE = 0
POSTSELECT_ALL = 1
POSTSELECT_LISTED = 2


def finalize(circuit, outcomes, postselect: int = POSTSELECT_NONE, post_dets=None):
    """outcomes: sequence over measurement ordinals of one shot's bits.

    post_dets: detector indices that reject (POSTSELECT_LISTED only).
    Returns (records, dets, obs, discard) as numpy uint8 arrays / int.
    """
    listed = set(int(i) for i in post_dets) if post_dets is not None else set()
    rec = np.zeros(circuit.num_records, dtype=np.uint8)
    det = np.zeros(circuit.num_dets, dtype=np.uint8)
    obs = np.zeros(circuit.num_obs, dtype=np.uint8)
    discarded = False
    for op in circuit.ops:
        if op.kind == "meas" and op.rec >= 0:
            if not discarded:
                rec[op.rec] = outcomes[op.t]
        elif op.kind == "det":
            if discarded:
                continue
            v = 0
            for t in op.conds:
                v ^= int(outcomes[t])
            det[op.index] = v
            rejects = (postselect == POSTSELECT_ALL
                       or (postselect == POSTSELECT_LISTED and op.index in listed))
            if rejects and v == 1:
                discarded = True
        elif op.kind == "obs":
            if discarded:
                continue
            v = 0
            for t in op.conds:
                v ^= int(outcomes[t])
            obs[op.index] ^= v
    if discarded:
        obs[:] = 0
    return rec, det, obs, int(discarded)


def pack_columns(bits_by_shot: np.ndarray, n_words: int) -> np.ndarray:
    """(S, ncol) uint8 bits -> (ncol, n_words) uint64 packed columns.

    Bit (r & 63) of word r >> 6 of column j holds shot r's bit j; padding is 0.
    """
    S, ncol = bits_by_shot.shape
    out = np.zeros((ncol, n_words), dtype=np.uint64)
    for r in range(S):
        row = bits_by_shot[r]
        nz = np.nonzero(row)[0]
        if len(nz):
            out[nz, r >> 6] |= np.uint64(1) << np.uint64(r & 63)
    return out
