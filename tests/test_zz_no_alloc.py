"""symft_sample_noalloc: the entry point for callers that cannot allocate device memory.

Frameworks that own the device heap, fixed-budget services and code sampling
during stream capture cannot let the library call cudaMalloc.  For them the
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
from paper_2607_28600_b300.workloads import random_near_clifford, rotated_surface_code_memory  # noqa: E402


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
    return [t.cpu().numpy() for t in (meas, det, obs, disc)]


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
