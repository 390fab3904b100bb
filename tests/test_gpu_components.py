"""Product-component representation (Sec. 6) on the GPU: the executor that
keeps one small vector per independent component, merging components by an
exact Kronecker product when an instruction couples them, samples the same
bits as the state-vector oracle and as the monolithic executors."""
import random

import numpy as np
import pytest

from paper_2607_28600_b300.workloads import (coherent_surface_code_memory, distillation_15_to_1,
                                             random_near_clifford)
from tests.helpers import oracle_sample, unpack
from tests.test_gpu_outputs import _fp32_prefix_check, _gpu_probs, _sv_probs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(text, shots, seed, precision, product_components, postselect=0, executor="auto"):
    import paper_2607_28600_b300 as S
    plan = S.symft_compile(text, postselect=postselect, product_components=product_components,
                           executor=executor)
    info = plan.info
    W = (shots + 63) // 64
    cols = [torch.zeros((max(1, info[k]), W), dtype=torch.int64, device="cuda")
            for k in ("n_records", "n_dets", "n_obs")]
    disc = torch.zeros((W,), dtype=torch.int64, device="cuda")
    S.symft_sample_ex(plan, shots, seed, meas_out=cols[0], det_out=cols[1], obs_out=cols[2],
                      discard_out=disc, precision=precision, check=True)
    torch.cuda.synchronize()
    out = [unpack(c.cpu().numpy().view(np.uint64)[: max(1, info[k])], shots)
           for c, k in zip(cols, ("n_records", "n_dets", "n_obs"))]
    out.append(unpack(disc.cpu().numpy().view(np.uint64).reshape(1, -1), shots)[:, 0])
    return plan, out


def test_literal_distillation_components_vs_statevector():
    """16 qubits, k_max = 15: the component workspace (5,530 amplitudes) sits in
    a global slot per warp in both precisions (the placement that keeps more
    warps resident per SM)."""
    text = distillation_15_to_1(1e-3, "literal")
    shots, seed = 48, 23
    plan, rec64, p64 = _gpu_probs(text, shots, seed, precision=1)
    info = plan.info
    assert info["pc_selected"] == 1
    assert all(e.startswith("components") for e in info["dense_executor"])
    assert info["pc_capacity"] < (1 << info["k_max"])
    act = plan.active_meas()
    ref = _sv_probs(text, seed, shots, act)
    assert np.abs(p64 - ref).max() <= 1e-9
    o = oracle_sample(text, seed, range(shots), kind="sv")
    np.testing.assert_array_equal(rec64, o["records"])
    _, rec32, p32 = _gpu_probs(text, shots, seed, precision=0)
    flips, worst = _fp32_prefix_check(p32, ref, rec32, o["records"], act, seed, shots)
    assert worst <= 1e-5 and flips <= 1


@pytest.mark.parametrize("which", ["literal", "coherent_d5_r1"])
@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("executor", ["components_cta", "components_warp"])
def test_components_equal_monolithic(which, precision, executor):
    """Same plan with and without the product components (on one CTA or one
    warp per shot), postselection on (early exit inside the component
    program): FP64 bit-exact, FP32 equal on every shot without an outcome
    flip."""
    text = (distillation_15_to_1(1e-3, "literal") if which == "literal"
            else coherent_surface_code_memory(5, 1, 1e-3, 0.02))
    shots, seed = (4000, 3) if which == "literal" else (600, 4)
    p1, a = _run(text, shots, seed, precision, True, postselect=1, executor=executor)
    p0, b = _run(text, shots, seed, precision, False, postselect=1)
    assert p1.info["dense_executor"][precision] == executor
    assert not p0.info["dense_executor"][precision].startswith("components")
    if precision == 1:
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    else:
        flipped = (a[0] != b[0]).any(axis=1)
        assert flipped.mean() <= 0.01
        for x, y in zip(a[1:], b[1:]):
            np.testing.assert_array_equal(x[~flipped], y[~flipped])


@pytest.mark.parametrize("case", range(4))
def test_components_random_circuits_vs_statevector(case):
    """Random near-Clifford circuits whose rotations are mostly independent
    (few coupling layers): components open, merge and shrink."""
    import paper_2607_28600_b300 as S
    text = random_near_clifford(14, 4, 12, 2e-3, seed=60 + case)
    plan = S.symft_compile(text)
    shots, seed = 150, 9 + case
    _, g = _run(text, shots, seed, 1, True)
    o = oracle_sample(text, seed, range(shots), kind="sv")
    np.testing.assert_array_equal(g[0], o["records"])
    _, m = _run(text, shots, seed, 1, False)
    np.testing.assert_array_equal(g[0], m[0])
    if plan.info["k_max"] > 5:
        assert plan.info["pc_work"][0] <= plan.info["pc_work"][1] * 2


@pytest.mark.parametrize("which", ["coherent_d3_r3", "random"])
def test_every_executor_gives_the_same_bits(which):
    """Every dense executor that can run a plan (warp, CTA, wide, product
    components on a warp or a CTA; the autotuner may pick any of them)
    samples the same FP64 bits."""
    text = (coherent_surface_code_memory(3, 3, 1e-3, 0.02) if which == "coherent_d3_r3"
            else random_near_clifford(14, 4, 12, 2e-3, seed=61))
    shots, seed = 1500, 12
    outs = {}
    for ex in ("warp", "cta", "wide", "components_warp", "components_cta"):
        plan, o = _run(text, shots, seed, 1, True, postselect=1, executor=ex)
        assert plan.info["dense_executor"][1] == ex
        outs[ex] = o
    for ex, o in outs.items():
        for x, y in zip(outs["warp"], o):
            np.testing.assert_array_equal(x, y, err_msg=ex)


def test_random_circuits_every_executor_same_bits():
    """Random near-Clifford circuits over a range of k_max (seeded), with and
    without postselection: every dense executor that can run a plan (register
    with several shots per warp, warp with one or two shots per warp, CTA,
    wide with its streamed tiles, product components on a warp or a CTA)
    samples the same FP64 bits, at a shot offset and a ragged shot count."""
    import paper_2607_28600_b300 as S
    rng = random.Random(2024)
    compared = 0
    for _ in range(10):
        nq, layers, nrot = rng.randint(6, 16), rng.randint(3, 8), rng.randint(1, 12)
        text = random_near_clifford(nq, layers, nrot, 5e-3, seed=rng.randint(0, 10**6))
        post = rng.randint(0, 1)
        outs = []
        for ex in ("register", "warp", "cta", "wide", "components_warp", "components_cta"):
            try:
                plan = S.symft_compile(text, postselect=post, executor=ex)
            except S.SymftError:
                continue
            if plan.info["k_max"] == 0 or plan.info["dense_executor"][1] != ex:
                continue
            m, d, o, disc = S.sample_to_tensors(plan, 1537, 99, shot_offset=512, precision=S.FP64)
            outs.append((ex, [t.cpu().numpy() for t in (m, d, o, disc)]))
        for ex, o in outs[1:]:
            for x, y in zip(outs[0][1], o):
                np.testing.assert_array_equal(x, y, err_msg=f"{outs[0][0]} vs {ex}")
            compared += 1
    assert compared >= 20
