"""Register-resident dense executor with several shots per warp (Sec. 6, the
dense active-state executor for small k): a warp holds 32 / 2^k_max shots, one
per segment of 2^k_max lanes.  With k_max = 1..4 and postselection, the shots
of one warp are rejected at different active measurements (early exit), so
the segments of a warp stop at different points; a ragged shot count leaves
the last warp with segments past the request, and a shot offset (a multiple
of 512) moves the request's streams.  FP64 bits equal those of the
one-shot-per-warp executor and of the oracle."""
import numpy as np
import pytest

from paper_2607_28600_b300.workloads import (coherent_surface_code_memory, cultivation_shaped,
                                             random_near_clifford, rotated_surface_code_memory)
from tests.helpers import oracle_sample, unpack

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    # name: (circuit text, k_max)
    "surface_d3_T_k1": (rotated_surface_code_memory(3, 2, 2e-2, t_on_data0_after_round=0), 1),
    "random_k2": (random_near_clifford(8, 3, 3, 2e-2, seed=7), 2),
    "random_k3": (random_near_clifford(8, 4, 4, 2e-2, seed=9), 3),
    "coherent_d3_r1_k4": (coherent_surface_code_memory(3, 1, 2e-2, 0.3), 4),
    "cultivation_small_k4": (cultivation_shaped(5e-3, grow_d=5, grow_rounds=1), 4),
}


def _run(text, shots, seed, shot_offset, precision, executor):
    import paper_2607_28600_b300 as S
    plan = S.symft_compile(text, postselect=1, executor=executor)
    info = plan.info
    W = (shots + 63) // 64
    cols = [torch.zeros((max(1, info[k]), W), dtype=torch.int64, device="cuda")
            for k in ("n_records", "n_dets", "n_obs")]
    disc = torch.zeros((W,), dtype=torch.int64, device="cuda")
    S.symft_sample_ex(plan, shots, seed, shot_offset=shot_offset, meas_out=cols[0], det_out=cols[1],
                      obs_out=cols[2], discard_out=disc, precision=precision, check=True)
    torch.cuda.synchronize()
    out = [unpack(c.cpu().numpy().view(np.uint64)[: info[k]], shots)
           for c, k in zip(cols, ("n_records", "n_dets", "n_obs"))]
    out.append(unpack(disc.cpu().numpy().view(np.uint64).reshape(1, -1), shots)[:, 0])
    return plan, out


@pytest.mark.parametrize("name", list(CASES))
def test_segments_equal_one_shot_per_warp(name):
    text, k = CASES[name]
    shots, seed, off = 3000 + 13, 41, 512 * 3
    reg_plan, reg = _run(text, shots, seed, off, 1, "register")
    assert reg_plan.info["k_max"] == k and reg_plan.info["dense_executor"][1] == "register"
    warp_plan, warp = _run(text, shots, seed, off, 1, "warp")
    assert warp_plan.info["dense_executor"][1] == "warp"
    for x, y in zip(reg, warp):
        np.testing.assert_array_equal(x, y)
    # postselection rejects a good share of the shots of these noisy circuits
    # (where they have detectors), so warps hold live and rejected segments
    if reg_plan.info["n_dets"]:
        rate = reg[3].mean()
        assert 0.05 < rate < 0.95


@pytest.mark.parametrize("name", ["surface_d3_T_k1", "random_k3", "coherent_d3_r1_k4"])
def test_segments_match_the_oracle(name):
    text, _ = CASES[name]
    shots, seed, off = 96 + 7, 5, 512
    _, (rec, det, obs, disc) = _run(text, shots, seed, off, 1, "register")
    o = oracle_sample(text, seed, range(off, off + shots), postselect=1)
    np.testing.assert_array_equal(rec, o["records"])
    np.testing.assert_array_equal(det, o["dets"])
    np.testing.assert_array_equal(obs, o["obs"])
    np.testing.assert_array_equal(disc, o["discard"])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["surface_d3_T_k1", "random_k3", "coherent_d3_r1_k4", "cultivation_small_k4"])
def test_shot_bits_do_not_depend_on_the_warp_layout(name, precision):
    """A shot's bits are a function of its absolute index alone: one call over
    N shots equals two calls over the same shots split at a 512-shot offset,
    although the shots land in other warps, segments and register sets (FP32
    lanes carry two sets of shots)."""
    text, _ = CASES[name]
    shots, seed, cut = 3000 + 13, 17, 512 * 3
    plan, whole = _run(text, shots, seed, 0, precision, "register")
    assert plan.info["dense_executor"][precision] == "register"
    _, first = _run(text, cut, seed, 0, precision, "register")
    _, second = _run(text, shots - cut, seed, cut, precision, "register")
    for w, a, b in zip(whole, first, second):
        np.testing.assert_array_equal(w, np.concatenate([a, b], axis=0))
