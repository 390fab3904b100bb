"""Pins of the oracle's postselection rule (Sec. 6, detector postselection),
including the listed-detector mode, on hand-worked outcomes.

The circuit measures three qubits, each followed by a detector on its record,
and closes with an observable on the last two records.  For the outcomes
(1, 0, 1) the bits are worked out by hand for every mode below.
"""
import random

import numpy as np

from oracle.circuit import parse
from oracle.records import POSTSELECT_ALL, POSTSELECT_LISTED, POSTSELECT_NONE, finalize

TEXT = """M 0
DETECTOR rec[-1]
M 1
DETECTOR rec[-1]
M 2
DETECTOR rec[-1]
OBSERVABLE_INCLUDE(0) rec[-1] rec[-2]
"""
OUT = [1, 0, 1]


def _fin(mode, listed=None):
    rec, det, obs, d = finalize(parse(TEXT), OUT, mode, listed)
    return rec.tolist(), det.tolist(), obs.tolist(), d


def test_none_keeps_everything():
    assert _fin(POSTSELECT_NONE) == ([1, 0, 1], [1, 0, 1], [1], 0)


def test_all_rejects_at_first_fired_detector():
    # detector 0 fires: records 1, 2 and detectors 1, 2 come later and read 0
    assert _fin(POSTSELECT_ALL) == ([1, 0, 0], [1, 0, 0], [0], 1)


def test_listed_quiet_detector_never_rejects():
    assert _fin(POSTSELECT_LISTED, [1]) == ([1, 0, 1], [1, 0, 1], [1], 0)


def test_listed_late_detector_rejects_and_clears_only_the_observable():
    assert _fin(POSTSELECT_LISTED, [2]) == ([1, 0, 1], [1, 0, 1], [0], 1)
    assert _fin(POSTSELECT_LISTED, [1, 2]) == ([1, 0, 1], [1, 0, 1], [0], 1)


def test_listed_special_cases_reduce_to_all_and_none():
    assert _fin(POSTSELECT_LISTED, [0]) == _fin(POSTSELECT_ALL)
    assert _fin(POSTSELECT_LISTED, []) == _fin(POSTSELECT_NONE)
    rng = random.Random(5)
    text = "\n".join(f"M {q}\nDETECTOR rec[-1]" for q in range(6)) + "\nOBSERVABLE_INCLUDE(0) rec[-1]\n"
    c = parse(text)
    for _ in range(50):
        out = [rng.randint(0, 1) for _ in range(6)]
        a = finalize(c, out, POSTSELECT_ALL)
        b = finalize(c, out, POSTSELECT_LISTED, list(range(6)))
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
