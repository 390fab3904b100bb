"""Pins for the plain SymFT oracle (Secs. 3-5) against brute force and closed forms."""
import math
import random

import numpy as np
import pytest

from oracle import statevector as sv
from oracle import symft
from oracle.circuit import parse
from paper_2607_28600_b300.workloads import rotated_surface_code_memory
from tests.circuits_for_tests import random_clifford_text

KINDS = {"PromoteRot", "ActiveDiagRot", "ActivePairRot", "RandomMeas", "DetMeas",
         "ActiveDiagMeas", "ActivePairMeas"}


@pytest.mark.parametrize("trial", range(12))
def test_symft_equals_statevector_shot_by_shot(trial):
    rng = random.Random(500 + trial)
    n = rng.randint(2, 6)
    c = parse(random_clifford_text(rng, n, 45, rot=0.25))
    plan = symft.Plan(c)
    shots = list(range(0, 150, 3))
    a = sv.sample(c, 9, shots)
    b = symft.sample(c, 9, shots, plan=plan)
    np.testing.assert_array_equal(a["outcomes"], b["outcomes"])
    st = plan.stats
    n_act = st["hist"].get("ActiveDiagMeas", 0) + st["hist"].get("ActivePairMeas", 0)
    assert st["k_final"] == st["hist"].get("PromoteRot", 0) - n_act


def test_all_instruction_kinds_exercised():
    seen = set()
    for trial in range(12):
        rng = random.Random(500 + trial)
        n = rng.randint(2, 6)
        plan = symft.Plan(parse(random_clifford_text(rng, n, 45, rot=0.25)))
        seen |= set(plan.stats["hist"])
    assert seen == KINDS


def test_branch_probabilities_match_statevector():
    rng = random.Random(77)
    c = parse(random_clifford_text(rng, 4, 50, rot=0.3, noise=False))
    plan = symft.Plan(c)
    for r in range(20):
        log_sv, log_sf = [], []
        sv.sample_shot(c, 4, r, prob_log=log_sv)
        from oracle.noise import NoiseSampler
        symft.sample_shot(plan, 4, r, NoiseSampler(c, 4), prob_log=log_sf)
        d = dict(log_sv)
        for t, p0 in log_sf:
            assert abs(d[t] - p0) < 1e-12


def test_norm_preserved_after_measurements():
    rng = random.Random(12)
    c = parse(random_clifford_text(rng, 5, 60, rot=0.3))
    plan = symft.Plan(c)
    from oracle.noise import NoiseSampler
    ns = NoiseSampler(c, 1)
    for r in range(10):
        norms = []
        symft.sample_shot(plan, 1, r, ns, norm_log=norms)
        for v in norms:
            assert abs(v - 1.0) < 1e-12


def test_closed_form_t_on_plus():
    c = parse("H 0\nR_Z(0.7853981633974483) 0\nMX 0\n")
    plan = symft.Plan(c)
    log = []
    from oracle.noise import NoiseSampler
    symft.sample_shot(plan, 1, 0, NoiseSampler(c, 1), prob_log=log)
    assert abs(log[0][1] - math.cos(math.pi / 8) ** 2) < 1e-15


def test_surface_code_with_t_after_round0():
    # at p = 0 exactly one X-check detector (the one on data qubit 0) sees the rotation
    c = parse(rotated_surface_code_memory(3, 3, p=0.0, t_on_data0_after_round=0))
    plan = symft.Plan(c)
    assert plan.stats["k_max"] == 1
    o = symft.sample(c, 1, range(1500), plan=plan)
    rates = o["dets"].mean(axis=0)
    assert (rates > 0).sum() == 1
    s2 = math.sin(math.pi / 8) ** 2
    assert abs(rates.max() - s2) < 4 * math.sqrt(s2 * (1 - s2) / 1500)


def test_pure_clifford_has_kmax_zero():
    plan = symft.Plan(parse(rotated_surface_code_memory(3, 3, p=1e-3)))
    assert plan.stats["k_max"] == 0
    assert set(plan.stats["hist"]) <= {"RandomMeas", "DetMeas"}
