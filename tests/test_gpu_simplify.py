"""Commutation-aware simplification before planning (Sec. 6) on the GPU: a
plan compiled with the rewrites samples the same records, detectors and
observables as the unsimplified oracle, bit for bit in FP64 (the oracle is the
plain circuit's state vector, or the plain SymFT interpreter, which never
simplifies), and its branch probabilities agree with the state vector's."""
import random

import numpy as np
import pytest

from paper_2607_28600_b300.workloads import cultivation_shaped
from tests.circuits_for_tests import fusion_circuit_text
from tests.helpers import gpu_sample, oracle_sample, unpack
from tests.test_gpu_outputs import _gpu_probs, _sv_probs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _outputs(text, shots, seed, simplify, precision=1, postselect=0):
    import paper_2607_28600_b300 as S
    plan = S.symft_compile(text, postselect=postselect, simplify=simplify)
    info = plan.info
    W = (shots + 63) // 64
    cols = [torch.zeros((max(1, info[k]), W), dtype=torch.int64, device="cuda")
            for k in ("n_records", "n_dets", "n_obs")]
    disc = torch.zeros((W,), dtype=torch.int64, device="cuda")
    S.symft_sample_ex(plan, shots, seed, meas_out=cols[0], det_out=cols[1], obs_out=cols[2],
                      discard_out=disc, precision=precision, check=True)
    torch.cuda.synchronize()
    return plan, [unpack(c.cpu().numpy().view(np.uint64)[: max(1, info[k])], shots)
                  for c, k in zip(cols, ("n_records", "n_dets", "n_obs"))] + \
        [unpack(disc.cpu().numpy().view(np.uint64).reshape(1, -1), shots)[:, 0]]


@pytest.mark.parametrize("case", range(6))
def test_simplified_plan_equals_state_vector(case):
    rng = random.Random(1000 + case)
    text = fusion_circuit_text(rng, n=6, blocks=8)
    shots, seed = 400, 11 + case
    plan, g = _outputs(text, shots, seed, simplify=True)
    o = oracle_sample(text, seed, range(shots), kind="sv")
    for got, key in zip(g, ("records", "dets", "obs")):
        np.testing.assert_array_equal(got[:, : o[key].shape[1]], o[key], err_msg=key)
    # the unsimplified plan gives the same bits
    _, g0 = _outputs(text, shots, seed, simplify=False)
    for a, b in zip(g, g0):
        np.testing.assert_array_equal(a, b)


def test_simplified_plan_branch_probabilities():
    rng = random.Random(77)
    text = fusion_circuit_text(rng, n=6, blocks=10)
    shots, seed = 200, 5
    plan, _, p64 = _gpu_probs(text, shots, seed, precision=1)
    act = plan.active_meas()
    if not act:
        pytest.skip("no active measurement in this draw")
    ref = _sv_probs(text, seed, shots, act)
    assert np.abs(p64 - ref).max() <= 1e-9


def test_cultivation_simplified_equals_unsimplified():
    text = cultivation_shaped(1e-3)
    shots, seed = 3000, 19
    p1, g1 = _outputs(text, shots, seed, simplify=True, postselect=1)
    p0, g0 = _outputs(text, shots, seed, simplify=False, postselect=1)
    assert p1.info["simplified"]["cancelled"] >= 7
    for a, b in zip(g1, g0):
        np.testing.assert_array_equal(a, b)
    o = oracle_sample(text, seed, range(400), postselect=1, kind="symft")
    for got, key in zip(g1, ("records", "dets", "obs", "discard")):
        np.testing.assert_array_equal(got[:400], o[key], err_msg=key)
