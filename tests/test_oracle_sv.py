"""Pins for the dense state-vector oracle: closed forms and the tableau cross-check."""
import math
import random

import numpy as np
import pytest

from oracle import statevector as sv
from oracle import tableau as tb
from oracle.circuit import parse
from tests.circuits_for_tests import random_clifford_text


def p_record(text, bits):
    return sv.exact_distribution(parse(text)).get(tuple(bits), 0.0)


def test_t_rotated_plus_measured_in_x():
    # H; R_Z(pi/4) = exp(-i pi/8 Z); MX  ->  p(+) = cos^2(pi/8) = 0.853553...
    p0 = p_record("H 0\nR_Z(0.7853981633974483) 0\nMX 0\n", [0])
    assert abs(p0 - math.cos(math.pi / 8) ** 2) < 1e-12
    assert abs(p0 - 0.8535533905932737) < 1e-12


def test_two_t_make_s_and_t_tdag_cancel():
    assert abs(p_record("H 0\nT 0\nT 0\nMX 0\n", [0]) - 0.5) < 1e-12
    assert abs(p_record("H 0\nT 0\nT_DAG 0\nMX 0\n", [0]) - 1.0) < 1e-12


@pytest.mark.parametrize("theta", [0.3, 1.1, -2.0])
def test_zz_rotation_on_plus_plus(theta):
    base = f"H 0 1\nR_PAULI({theta!r}) Z0*Z1\n"
    assert abs(p_record(base + "MX 0\n", [0]) - math.cos(theta / 2) ** 2) < 1e-12
    assert abs(p_record(base + "MPP X0*X1\n", [0]) - 1.0) < 1e-12


@pytest.mark.parametrize("p", [0.1, 0.37])
def test_noise_closed_forms(p):
    assert abs(p_record(f"X_ERROR({p}) 0\nM 0\n", [1]) - p) < 1e-12
    assert abs(p_record(f"DEPOLARIZE1({p}) 0\nM 0\n", [1]) - 2 * p / 3) < 1e-12
    assert abs(p_record(f"Z_ERROR({p}) 0\nM 0\n", [1])) < 1e-12
    # DEPOLARIZE2: qubit 0 flipped by X or Y on it: 8 of 15 cells
    assert abs(p_record(f"DEPOLARIZE2({p}) 0 1\nM 0\n", [1]) - 8 * p / 15) < 1e-12


def test_y_conventions():
    # Y|0> = i|1>: measurement gives 1; S H |0> = |+i>: MY gives 0
    assert p_record("Y 0\nM 0\n", [1]) == pytest.approx(1.0)
    assert p_record("H 0\nS 0\nMY 0\n", [0]) == pytest.approx(1.0)
    assert p_record("H 0\nS_DAG 0\nMY 0\n", [1]) == pytest.approx(1.0)
    assert p_record("SQRT_X 0\nMY 0\n", [1]) == pytest.approx(1.0)


def test_feedback_and_reset():
    # Bell pair, measure 0, feedback X on 1 -> qubit 1 always 0
    d = sv.exact_distribution(parse("H 0\nCX 0 1\nM 0\nCX rec[-1] 1\nM 1\n"))
    assert d.get((0, 0), 0) == pytest.approx(0.5) and d.get((1, 0), 0) == pytest.approx(0.5)
    assert p_record("H 0\nR 0\nM 0\n", [0]) == pytest.approx(1.0)
    assert p_record("RX 0\nMX 0\n", [0]) == pytest.approx(1.0)


def test_distribution_sums_to_one():
    txt = "H 0\nR_PAULI(0.7) X0*Y1\nDEPOLARIZE1(0.2) 1\nMPP Z0*Z1\nR_X(1.3) 0\nM 0 1\n"
    d = sv.exact_distribution(parse(txt))
    assert sum(d.values()) == pytest.approx(1.0, abs=1e-12)


def test_sampled_frequencies_match_exact():
    txt = "H 0\nR_Z(0.7853981633974483) 0\nMX 0\n"
    c = parse(txt)
    o = sv.sample(c, 21, range(3000))
    p1 = o["records"][:, 0].mean()
    assert abs(p1 - math.sin(math.pi / 8) ** 2) < 4 * math.sqrt(0.15 * 0.85 / 3000)


@pytest.mark.parametrize("trial", range(8))
def test_statevector_equals_tableau_shot_by_shot(trial):
    rng = random.Random(100 + trial)
    txt = random_clifford_text(rng, rng.randint(2, 6), 40)
    c = parse(txt)
    shots = list(range(0, 260, 5))
    a = sv.sample(c, 17, shots)
    b = tb.sample(c, 17, shots)
    np.testing.assert_array_equal(a["outcomes"], b["outcomes"])
