"""Commutation-aware simplification before planning (Sec. 6), host side: the
rewrites fire on circuits built for them and never widen the active state or
add dense instructions.  (Whether the simplified plan samples the same
distribution is checked on the GPU against the unsimplified oracle.)"""
import random

import paper_2607_28600_b300 as S
from paper_2607_28600_b300.workloads import cultivation_shaped
from tests.circuits_for_tests import fusion_circuit_text

DENSE = ("PromoteRot", "ActiveDiagRot", "ActivePairRot", "ActiveDiagMeas", "ActivePairMeas")


def _dense(info):
    return sum(info["n_instr"][k] for k in DENSE)


def test_cancelling_pair_across_commuting_operations_is_removed():
    # R_Z(t) on qubit 0, operations on other qubits, R_Z(-t) on qubit 0; the
    # R_X on qubit 1 pulls back to X1 X2 through the CX, commutes with the Z1 Z2
    # of M 2, and meets MX 1 (X1 X2 too): a branch phase
    txt = "H 0 1 2\nR_Z(0.7) 0\nCX 1 2\nR_X(0.3) 1\nM 2\nR_Z(-0.7) 0\nMX 0 1\n"
    a = S.symft_compile(txt, simplify=False).info
    b = S.symft_compile(txt).info
    assert b["simplified"] == {"fused": 1, "cancelled": 1, "branch_phase": 1}
    assert b["n_instr"]["PromoteRot"] == a["n_instr"]["PromoteRot"] - 1
    assert b["k_max"] <= a["k_max"]


def test_no_fusion_across_noise_on_the_support_or_an_anticommuting_operation():
    # a noise symbol on qubit 0 makes the two signs differ by a symbol
    txt = "H 0 1\nR_Z(0.7) 0\nDEPOLARIZE1(0.1) 0\nR_Z(-0.7) 0\nMX 0 1\n"
    assert S.symft_compile(txt).info["simplified"]["fused"] == 0
    # an X measurement of qubit 0 anticommutes with Z_0
    txt2 = "H 0 1\nR_Z(0.7) 0\nMX 0\nR_Z(-0.7) 0\nMX 0 1\n"
    assert S.symft_compile(txt2).info["simplified"]["fused"] == 0
    # a detector between them is a segment boundary
    txt3 = "H 0 1\nR_Z(0.7) 0\nM 1\nDETECTOR rec[-1]\nR_Z(-0.7) 0\nMX 0 1\n"
    assert S.symft_compile(txt3).info["simplified"]["fused"] == 0


def test_deterministic_sign_difference_fuses_with_the_opposite_angle():
    # X on qubit 0 between two R_Z(0.7) flips the second's sign by a constant:
    # R_Z(0.7) X R_Z(0.7) = X R_Z(-0.7) R_Z(0.7) -> cancelled
    txt = "H 0 1\nR_Z(0.7) 0\nX 0\nR_Z(0.7) 0\nMX 0 1\n"
    assert S.symft_compile(txt).info["simplified"] == {"fused": 1, "cancelled": 1, "branch_phase": 0}


def test_rotation_before_a_same_body_measurement_is_a_branch_phase():
    txt = "H 0 1\nCX 0 1\nR_PAULI(0.4) X0*X1\nM 2\nMPP X0*X1\nMX 0\n"
    assert S.symft_compile(txt).info["simplified"]["branch_phase"] == 1


def test_random_fusion_circuits_never_grow_the_plan():
    rng = random.Random(7)
    fired = 0
    for _ in range(40):
        txt = fusion_circuit_text(rng)
        a = S.symft_compile(txt, simplify=False).info
        b = S.symft_compile(txt).info
        assert b["k_max"] <= a["k_max"]
        assert _dense(b) <= _dense(a)
        fired += sum(b["simplified"].values())
    assert fired > 10


def test_cultivation_shaped_check_layers_cancel():
    a = S.symft_compile(cultivation_shaped(1e-3), postselect=1, simplify=False).info
    b = S.symft_compile(cultivation_shaped(1e-3), postselect=1).info
    assert b["simplified"]["cancelled"] >= 7
    assert _dense(b) < _dense(a)
    assert b["dense_amp_traffic"] < a["dense_amp_traffic"]
