"""Pins for the Aaronson-Gottesman tableau oracle."""
import numpy as np
import pytest

from oracle import tableau as tb
from oracle.circuit import parse
from paper_2607_28600_b300.workloads import rotated_surface_code_memory


def test_ghz_parities():
    c = parse("H 0\nCX 0 1\nCX 1 2\nM 0 1 2\nMPP X0*X1*X2\n")
    o = tb.sample(c, 3, range(200))
    r = o["records"]
    assert (r[:, 0] == r[:, 1]).all() and (r[:, 1] == r[:, 2]).all()
    assert 0.3 < r[:, 0].mean() < 0.7
    c2 = parse("H 0\nCX 0 1\nCX 1 2\nMPP X0*X1*X2 Z0*Z1 Y0*Y1*X2\n")
    o2 = tb.sample(c2, 3, range(50))
    # |GHZ> is a +1 eigenstate of XXX and ZZI; YYX = -XXX (Y Y = -X Z X Z ...) -> outcome 1
    assert (o2["records"][:, 0] == 0).all() and (o2["records"][:, 1] == 0).all()
    assert (o2["records"][:, 2] == 1).all()


@pytest.mark.parametrize("d,r,nq,ndet", [(3, 3, 17, 24), (7, 7, 97, 336), (9, 9, 161, 720)])
def test_generator_counts_match_paper(d, r, nq, ndet):
    # Sec. 7.2: d=7,r=7 has 97 qubits and 336 detectors; d=9,r=9 161 and 720.
    c = parse(rotated_surface_code_memory(d, r, p=1e-3))
    assert c.num_qubits == nq and c.num_dets == ndet and c.num_obs == 1


@pytest.mark.parametrize("d", [3, 5])
def test_noiseless_qec_fires_no_detector(d):
    c = parse(rotated_surface_code_memory(d, d, p=0.0))
    o = tb.sample(c, 8, range(128))
    assert o["dets"].sum() == 0 and o["obs"].sum() == 0


def test_single_error_fires_its_detectors():
    # one certain X error on a data qubit between rounds flips the two adjacent Z checks
    txt = rotated_surface_code_memory(3, 2, p=0.0).replace("TICK", "TICK", 1)
    lines = txt.splitlines()
    second_tick = [i for i, l in enumerate(lines) if l == "TICK"][1]
    lines.insert(second_tick, "X_ERROR(1.0) 4")
    c = parse("\n".join(lines) + "\n")
    o = tb.sample(c, 1, range(64))
    fired = o["dets"].sum(axis=0)
    assert set(np.nonzero(fired)[0]) and (fired[fired > 0] == 64).all()
    assert (fired > 0).sum() == 2
