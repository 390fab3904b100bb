"""symft_sample_noalloc: the entry point for callers that cannot allocate device memory.

Frameworks whose caching allocator owns the device heap, and services with a
fixed memory budget, cannot let the library call cudaMalloc.  For them the
library keeps one fixed 32 MiB device array and symft_sample_noalloc draws all
its scratch from it.  These tests call it through the C ABI on plans whose
near-Clifford instructions need that scratch (dense-sign and active-outcome
columns) and require the same bits as the allocating entry point,
symft_sample_ex, on two calls in a row (the second call must not see the first
call's leftovers).  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_28600_b300 as S  # noqa: E402
from paper_2607_28600_b300.workloads import (coherent_surface_code_memory, distillation_15_to_1,  # noqa: E402
                                             random_near_clifford, rotated_surface_code_memory)
from tests.helpers import unpack  # noqa: E402


def _outputs(plan, shots):
    info = plan.info
    W = (shots + 63) // 64
    mk = lambda n: torch.zeros((max(n, 1), W), dtype=torch.int64, device="cuda")
    return mk(info["n_records"]), mk(info["n_dets"]), mk(info["n_obs"]), \
        torch.zeros((W,), dtype=torch.int64, device="cuda")


def _run(fn, plan, shots, seed, precision, offset=0):
    meas, det, obs, disc = _outputs(plan, shots)
    fn(plan, shots, seed, shot_offset=offset, meas_out=meas, det_out=det, obs_out=obs,
       discard_out=disc, precision=precision)
    torch.cuda.synchronize()
    return [t.cpu().numpy().view(np.uint64) for t in (meas, det, obs, disc)]


CIRCUITS = {
    "surface_d3_t": rotated_surface_code_memory(3, 3, 1e-3, t_on_data0_after_round=0),
    "random_near_clifford": random_near_clifford(8, 10, 6, p=2e-3, seed=11),
}


@pytest.mark.parametrize("name", sorted(CIRCUITS))
@pytest.mark.parametrize("precision", [S.FP64, S.FP32])
def test_noalloc_matches_allocating_entry_point_twice(name, precision):
    plan = S.symft_compile(CIRCUITS[name])
    assert plan.info["k_max"] >= 1        # the plan uses the dense scratch
    shots = 3000
    for seed in (5, 6):                    # two calls in a row
        ref = _run(S.symft_sample_ex, plan, shots, seed, precision)
        got = _run(S.symft_sample_noalloc, plan, shots, seed, precision)
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", [S.FP64, S.FP32])
def test_noalloc_global_vectors_k15(precision):
    """The literal 15-to-1 circuit reaches k = 15: its vectors (256 KB in FP32,
    512 KB in FP64) exceed shared memory, so the no-allocation call keeps them
    in warp slots carved from its array, with the grid cut to the slots that
    fit; every slot serves many shots in turn."""
    plan = S.symft_compile(distillation_15_to_1(1e-3, "literal"))
    assert plan.info["k_max"] == 15
    shots = 1500
    for seed in (3, 4):
        ref = _run(S.symft_sample_ex, plan, shots, seed, precision)
        got = _run(S.symft_sample_noalloc, plan, shots, seed, precision)
        if precision == S.FP64:
            for a, b in zip(ref, got):
                np.testing.assert_array_equal(a, b)
        else:
            # FP32: the two executors add branch sums in different orders, so a
            # shot whose uniform sits within rounding of its FP32 probability
            # may flip; every other shot is bit-exact
            ra, ga = unpack(ref[0], shots), unpack(got[0], shots)
            flipped = (ra != ga).any(axis=1)
            assert flipped.mean() <= 0.01
            for a, b in zip(ref[1:3], got[1:3]):
                np.testing.assert_array_equal(unpack(a, shots)[~flipped], unpack(b, shots)[~flipped])


@pytest.mark.parametrize("precision", [S.FP64, S.FP32])
def test_noalloc_early_exit_before_later_active_measurements(precision):
    """Coherent-noise surface code, 3 rounds, every detector postselected:
    many shots are rejected in round 1, before the active measurements of the
    later rounds, and stop their dense work there.  The no-allocation call
    must give the same bits as symft_sample_ex."""
    plan = S.symft_compile(coherent_surface_code_memory(3, 3, 5e-3, 0.02), postselect=S.POSTSELECT_ALL)
    assert plan.info["k_max"] >= 4
    shots = 2000
    for seed in (8, 9):
        ref = _run(S.symft_sample_ex, plan, shots, seed, precision)
        got = _run(S.symft_sample_noalloc, plan, shots, seed, precision)
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)
        disc = unpack(ref[3].reshape(1, -1), shots)[:, 0]
        assert 0.05 < disc.mean() < 0.95


@pytest.mark.parametrize("precision", [S.FP64, S.FP32])
def test_noalloc_shot_offset_ragged(precision):
    """A shard that starts at a nonzero multiple of 512 shots and ends inside a
    64-shot word: the sign kernel's noise blocks and the dense executor's shot
    indices are offset, and padding bits stay zero."""
    plan = S.symft_compile(CIRCUITS["random_near_clifford"])
    shots, offset = 1000 + 37, 512 * 7
    for seed in (5, 6):
        ref = _run(S.symft_sample_ex, plan, shots, seed, precision, offset=offset)
        got = _run(S.symft_sample_noalloc, plan, shots, seed, precision, offset=offset)
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)
        assert (got[0][:, -1] >> np.uint64(shots % 64) == 0).all()


def test_noalloc_postselection_without_detector_output():
    plan = S.symft_compile(rotated_surface_code_memory(3, 3, 5e-3, t_on_data0_after_round=0),
                           postselect=S.POSTSELECT_ALL)
    shots = 2048
    W = shots // 64
    for seed in (1, 2):
        ref_meas = torch.zeros((plan.info["n_records"], W), dtype=torch.int64, device="cuda")
        ref_disc = torch.zeros((W,), dtype=torch.int64, device="cuda")
        S.symft_sample_ex(plan, shots, seed, meas_out=ref_meas, discard_out=ref_disc,
                          precision=S.FP64)
        meas = torch.zeros_like(ref_meas)
        disc = torch.zeros_like(ref_disc)
        S.symft_sample_noalloc(plan, shots, seed, meas_out=meas, discard_out=disc,
                               precision=S.FP64)
        torch.cuda.synchronize()
        assert torch.equal(meas, ref_meas) and torch.equal(disc, ref_disc)
        assert int(disc.count_nonzero()) > 0


def test_noalloc_rejects_requests_beyond_its_array():
    plan = S.symft_compile(CIRCUITS["surface_d3_t"])
    shots = 1 << 29                        # dense-sign columns alone exceed 32 MiB
    with pytest.raises(S.SymftError) as ei:
        S.symft_sample_noalloc(plan, shots, 1, meas_out=None)
    assert ei.value.code == -4
    assert "32 MiB" in str(ei.value)
