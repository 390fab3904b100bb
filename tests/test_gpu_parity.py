"""GPU parity: the CUDA sampler (through the C-ABI) against the CPU oracle.

Bit-exact on every record / detector / observable bit of Clifford circuits and
of FP64 runs; FP32 runs may flip an active outcome where the branch
probability lies within FP32 rounding of the measurement uniform, so they are
checked for a bounded flip rate and bit-exactness on unflipped shots.
"""
import math
import random

import numpy as np
import pytest

from oracle import symft as osymft
from oracle.circuit import parse as oparse
from paper_2607_28600_b300.workloads import random_near_clifford, rotated_surface_code_memory
from tests.circuits_for_tests import random_clifford_text
from tests.helpers import gpu_sample, oracle_sample, padding_is_zero, unpack

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _compare(text, shots, seed, precision=1, postselect=0, kind="auto", host=False, offset=0):
    plan, meas, det, obs, disc = gpu_sample(text, shots, seed, shot_offset=offset,
                                            precision=precision, postselect=postselect, host=host)
    for cols in (meas, det, obs):
        assert padding_is_zero(cols, shots)
    o = oracle_sample(text, seed, range(offset, offset + shots), postselect=postselect, kind=kind)
    g = {"records": unpack(meas, shots), "dets": unpack(det, shots), "obs": unpack(obs, shots),
         "discard": unpack(disc.reshape(1, -1), shots)[:, 0]}
    return plan, g, o


@pytest.mark.parametrize("d,p,shots", [(3, 1e-3, 1000), (3, 2e-2, 777), (5, 1e-2, 1300)])
def test_surface_code_bit_exact(d, p, shots):
    text = rotated_surface_code_memory(d, d, p)
    _, g, o = _compare(text, shots, seed=1)
    np.testing.assert_array_equal(g["records"], o["records"])
    np.testing.assert_array_equal(g["dets"], o["dets"])
    np.testing.assert_array_equal(g["obs"], o["obs"])


def test_long_memory_chains_cut_into_paths_bit_exact():
    """A 24-round d=3 memory: each stabilizer's records chain over 24 rounds,
    longer than the 16 records a chain path may hold, so the compile step
    starts new paths within a chain.  Every record, detector and observable
    bit against the tableau oracle."""
    text = rotated_surface_code_memory(3, 24, 2e-2)
    _, g, o = _compare(text, 700, seed=5)
    np.testing.assert_array_equal(g["records"], o["records"])
    np.testing.assert_array_equal(g["dets"], o["dets"])
    np.testing.assert_array_equal(g["obs"], o["obs"])


@pytest.mark.parametrize("shots", [1, 63, 64, 65, 127, 128, 129, 300])
def test_ragged_shot_counts(shots):
    text = rotated_surface_code_memory(3, 2, 5e-2)
    _, g, o = _compare(text, shots, seed=7)
    np.testing.assert_array_equal(g["records"], o["records"])
    np.testing.assert_array_equal(g["dets"], o["dets"])


def test_shot_offset_and_split_calls_agree():
    text = rotated_surface_code_memory(3, 3, 2e-2)
    _, m_all, d_all, _, _ = gpu_sample(text, 1024, 5)
    _, m_a, d_a, _, _ = gpu_sample(text, 512, 5, shot_offset=0)
    _, m_b, d_b, _, _ = gpu_sample(text, 512, 5, shot_offset=512)
    np.testing.assert_array_equal(m_all, np.concatenate([m_a, m_b], axis=1))
    np.testing.assert_array_equal(d_all, np.concatenate([d_a, d_b], axis=1))
    _, g, o = _compare(text, 200, seed=5, offset=1 << 20)
    np.testing.assert_array_equal(g["records"], o["records"])


def test_host_outputs_equal_device_outputs():
    text = rotated_surface_code_memory(3, 3, 2e-2)
    _, m1, d1, o1, _ = gpu_sample(text, 1000, 9)
    _, m2, d2, o2, _ = gpu_sample(text, 1000, 9, host=True)
    np.testing.assert_array_equal(m1, m2)
    np.testing.assert_array_equal(d1, d2)
    np.testing.assert_array_equal(o1, o2)


@pytest.mark.parametrize("trial", range(6))
def test_random_clifford_circuits_bit_exact(trial):
    rng = random.Random(3000 + trial)
    text = random_clifford_text(rng, rng.randint(2, 8), 60)
    _, g, o = _compare(text, 500, seed=trial + 1, kind="tableau")
    np.testing.assert_array_equal(g["records"], o["records"])
    np.testing.assert_array_equal(g["dets"], o["dets"])
    np.testing.assert_array_equal(g["obs"], o["obs"])


@pytest.mark.parametrize("trial", range(8))
def test_near_clifford_fp64_bit_exact(trial):
    rng = random.Random(4000 + trial)
    text = random_clifford_text(rng, rng.randint(2, 7), 60, rot=0.25)
    _, g, o = _compare(text, 300, seed=trial + 11, precision=1, kind="sv")
    np.testing.assert_array_equal(g["records"], o["records"])
    np.testing.assert_array_equal(g["dets"], o["dets"])


@pytest.mark.parametrize("trial", range(6))
def test_near_clifford_fp32_flip_rate(trial):
    rng = random.Random(4000 + trial)
    text = random_clifford_text(rng, rng.randint(2, 7), 60, rot=0.25)
    _, g, o = _compare(text, 300, seed=trial + 11, precision=0, kind="sv")
    diff = (g["records"] != o["records"]).any(axis=1)
    assert diff.mean() <= 0.01


def test_t_after_round0_surface_code():
    text = rotated_surface_code_memory(3, 3, 1e-3, t_on_data0_after_round=0)
    for prec in (1, 0):
        plan, g, o = _compare(text, 2000, seed=1, precision=prec)
        assert plan.info["k_max"] == 1
        diff = (g["records"] != o["records"]).any(axis=1)
        assert diff.sum() <= (0 if prec == 1 else 2)
        np.testing.assert_array_equal(g["dets"][~diff], o["dets"][~diff])


def test_postselection_all_detectors():
    text = rotated_surface_code_memory(3, 3, 2e-2)
    _, g, o = _compare(text, 1000, seed=4, postselect=1)
    np.testing.assert_array_equal(g["discard"], o["discard"])
    np.testing.assert_array_equal(g["records"], o["records"])
    np.testing.assert_array_equal(g["dets"], o["dets"])
    np.testing.assert_array_equal(g["obs"], o["obs"])
    assert 0.05 < g["discard"].mean() < 0.95


def test_postselection_with_active_measurements():
    text = rotated_surface_code_memory(3, 3, 5e-3, t_on_data0_after_round=0)
    _, g, o = _compare(text, 1500, seed=2, postselect=1, precision=1)
    np.testing.assert_array_equal(g["discard"], o["discard"])
    np.testing.assert_array_equal(g["records"], o["records"])


def test_no_noise_no_detector_fires_d5():
    _, meas, det, obs, _ = gpu_sample(rotated_surface_code_memory(5, 5, 0.0), 4096, 3)
    assert int(np.bitwise_or.reduce(det.ravel())) == 0
    assert int(np.bitwise_or.reduce(obs.ravel())) == 0


def test_random_near_clifford_generator_fp64():
    text = random_near_clifford(10, 12, 6, p=2e-3, seed=5)
    _, g, o = _compare(text, 200, seed=3, precision=1, kind="sv")
    np.testing.assert_array_equal(g["records"], o["records"])


def test_d7_full_size_sampled_shots():
    """d=7, 7 rounds at 1e7 shots in the bench's launch shape; 256 sampled shots
    checked one by one against the tableau oracle."""
    import paper_2607_28600_b300 as S
    text = rotated_surface_code_memory(7, 7, 1e-3)
    shots = 10_000_000
    plan = S.symft_compile(text)
    meas, det, obs, disc = S.sample_to_tensors(plan, shots, 1)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(shots, size=256, replace=False))
    pick = np.concatenate([pick, [0, shots - 1]])
    words = torch.as_tensor(pick >> 6, device=meas.device)
    bits = torch.as_tensor(pick & 63, device=meas.device, dtype=torch.int64)

    def gather(cols):
        v = cols[:, words].cpu().numpy().view(np.uint64)  # int64 storage of the words
        return ((v >> (bits.cpu().numpy().astype(np.uint64))[None, :]) & np.uint64(1)).T.astype(np.uint8)

    o = oracle_sample(text, 1, [int(x) for x in pick], kind="tableau")
    np.testing.assert_array_equal(gather(meas), o["records"])
    np.testing.assert_array_equal(gather(det), o["dets"])
    np.testing.assert_array_equal(gather(obs), o["obs"])
    # detector firing rate is a property at any size
    rate = float(unpack(det[:, :1024].cpu().numpy().view(np.uint64), 65536).mean())
    assert 0.005 < rate < 0.05


# ---- plain form (one CTA per shot, unpacked signs): same bits as the batched form ----

@pytest.mark.parametrize("d,p,post", [(3, 2e-2, 0), (5, 1e-2, 0), (3, 2e-2, 1)])
def test_plain_form_equals_batched_clifford(d, p, post):
    text = rotated_surface_code_memory(d, d, p)
    shots = 1000
    _, m1, d1, o1, x1 = gpu_sample(text, shots, 3, postselect=post)
    import paper_2607_28600_b300 as S
    plan = S.symft_compile(text, postselect=post)
    meas, det, obs, disc = S.sample_to_tensors(plan, shots, 3, plain=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(meas.cpu().numpy().view(np.uint64), m1)
    np.testing.assert_array_equal(det.cpu().numpy().view(np.uint64), d1)
    np.testing.assert_array_equal(obs.cpu().numpy().view(np.uint64), o1)
    np.testing.assert_array_equal(disc.cpu().numpy().view(np.uint64), x1)


@pytest.mark.parametrize("trial", range(4))
def test_plain_form_fp64_matches_statevector(trial):
    import paper_2607_28600_b300 as S
    rng = random.Random(4000 + trial)
    text = random_clifford_text(rng, rng.randint(2, 7), 60, rot=0.25)
    plan = S.symft_compile(text)
    shots = 300
    meas, det, obs, disc = S.sample_to_tensors(plan, shots, trial + 11, precision=S.FP64, plain=True)
    torch.cuda.synchronize()
    o = oracle_sample(text, trial + 11, range(shots), kind="sv")
    np.testing.assert_array_equal(unpack(meas.cpu().numpy().view(np.uint64), shots), o["records"])
    np.testing.assert_array_equal(unpack(det.cpu().numpy().view(np.uint64), shots), o["dets"])


# ---- distillation and cultivation-shaped workloads ----

@pytest.mark.parametrize("variant", ["encoded", "literal"])
def test_distillation_fp64_matches_statevector(variant):
    from paper_2607_28600_b300.workloads import distillation_15_to_1
    text = distillation_15_to_1(1e-3, variant)
    plan, g, o = _compare(text, 200, seed=4, precision=1, postselect=1, kind="sv")
    assert plan.info["k_max"] == (15 if variant == "literal" else 5)
    np.testing.assert_array_equal(g["discard"], o["discard"])
    np.testing.assert_array_equal(g["records"], o["records"])
    np.testing.assert_array_equal(g["obs"], o["obs"])


@pytest.mark.parametrize("variant", ["encoded", "literal"])
def test_distillation_fp32_flip_rate_vs_symft_oracle(variant):
    from paper_2607_28600_b300.workloads import distillation_15_to_1
    text = distillation_15_to_1(1e-3, variant)
    _, g, o = _compare(text, 2000, seed=5, precision=0, postselect=1, kind="symft")
    diff = (g["records"] != o["records"]).any(axis=1)
    assert diff.mean() <= 0.005


def test_cultivation_injection_stage_vs_statevector():
    from paper_2607_28600_b300.workloads import cultivation_shaped
    text = cultivation_shaped(1e-3, stage="injection")
    _, g, o = _compare(text, 300, seed=6, precision=1, postselect=1, kind="sv")
    np.testing.assert_array_equal(g["discard"], o["discard"])
    np.testing.assert_array_equal(g["records"], o["records"])


def test_cultivation_full_vs_symft_oracle_sampled():
    from paper_2607_28600_b300.workloads import cultivation_shaped
    text = cultivation_shaped(1e-3)
    for prec in (1, 0):
        plan, g, o = _compare(text, 400, seed=7, precision=prec, postselect=1, kind="symft")
        assert plan.info["n_qubits"] == 161 and plan.info["k_max"] >= 4
        diff = (g["records"] != o["records"]).any(axis=1)
        assert diff.sum() <= (0 if prec == 1 else 2)
        np.testing.assert_array_equal(g["discard"][~diff], o["discard"][~diff])


# ---- autotuning and graph-batched jobs leave every bit unchanged ----

def _dev_outputs(plan, shots):
    W = (shots + 63) // 64
    info = plan.info
    mk = lambda n: torch.zeros((max(1, n), W), dtype=torch.int64, device="cuda")
    return {"meas_out": mk(info["n_records"]), "det_out": mk(info["n_dets"]),
            "obs_out": mk(info["n_obs"]), "discard_out": torch.zeros((W,), dtype=torch.int64, device="cuda")}


def test_autotune_keeps_results():
    import paper_2607_28600_b300 as S
    from paper_2607_28600_b300.workloads import distillation_15_to_1
    for text, post in ((rotated_surface_code_memory(5, 5, 1e-2), 0),
                       (distillation_15_to_1(1e-3, "encoded"), 1)):
        plan = S.symft_compile(text, postselect=post)
        before = _dev_outputs(plan, 5000)
        S.symft_sample_ex(plan, 5000, 9, **before)
        S.symft_autotune(plan, 20000, S.FP32)
        after = _dev_outputs(plan, 5000)
        S.symft_sample_ex(plan, 5000, 9, **after)
        torch.cuda.synchronize()
        for k in before:
            assert torch.equal(before[k], after[k]), k


def test_graph_batch_equals_individual_calls():
    import paper_2607_28600_b300 as S
    from paper_2607_28600_b300.workloads import mixed_batch
    circuits = [c for c in mixed_batch(seed=3, n=12)]
    plans = [S.symft_compile(t, postselect=post) for _, t, post in circuits]
    keep = [i for i, pl in enumerate(plans) if pl.info["k_max"] <= 12]
    plans = [plans[i] for i in keep]
    jobs, refs = [], []
    for i, pl in enumerate(plans):
        shots = 700 + 128 * i
        outs = _dev_outputs(pl, shots)
        jobs.append({"plan": i, "shots": shots, "seed": 40 + i, "precision": S.FP32, **outs})
        ref = _dev_outputs(pl, shots)
        S.symft_sample_ex(pl, shots, 40 + i, **ref)
        refs.append(ref)
    # a second job on plan 0 (same branch, in order)
    extra = _dev_outputs(plans[0], 512)
    jobs.append({"plan": 0, "shots": 512, "seed": 99, "shot_offset": 1024, "precision": S.FP32, **extra})
    extra_ref = _dev_outputs(plans[0], 512)
    S.symft_sample_ex(plans[0], 512, 99, shot_offset=1024, **extra_ref)
    for rep in range(2):                      # second launch reuses / updates the cached graph
        S.symft_sample_batch(plans, jobs)
        torch.cuda.synchronize()
        for j, ref in zip(jobs, refs + [extra_ref]):
            for k in ref:
                assert torch.equal(j[k], ref[k]), (rep, j["plan"], k)
