"""GPU checks of the optional outputs: branch probabilities of the active
measurements (prob_out), listed-detector postselection, and the kept /
discarded / observable tallies (counts_out), all through the C-ABI.

Branch probabilities are compared with the state-vector oracle, which computes
Pr(m = 0) of every measurement from the full state (Sec. 4: the active
measurement formulas must give the same number).  FP64 runs agree to 1e-9 on
every active measurement.  FP32 runs must agree to 1e-5 on every active
measurement up to and including the first outcome flip of a shot (a flip is a
measurement whose FP32 and FP64 probabilities fall on different sides of the
shot's uniform; later measurements of that shot follow a different branch).
"""
import random

import numpy as np
import pytest

from oracle import statevector as osv
from oracle.circuit import parse as oparse
from oracle.noise import NoiseSampler
from oracle.streams import meas_uniform, outcome_from
from paper_2607_28600_b300.workloads import random_near_clifford, rotated_surface_code_memory
from tests.circuits_for_tests import random_clifford_text
from tests.helpers import gpu_sample, oracle_sample, unpack

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cases():
    rng = random.Random(4002)
    return {
        # k <= 5: register-resident warp executor
        "reg": random_clifford_text(rng, 6, 60, rot=0.25),
        # k = 10: warp per shot, vector in shared memory
        "warp": random_near_clifford(12, 24, 12, 1e-3, seed=1),
        # k = 13: CTA per shot, vector in shared memory
        "cta": random_near_clifford(14, 30, 14, 1e-3, seed=1),
        # k = 14: CTA per shot; the FP64 vector (256 KB) lives in a global slot
        "cta_global": random_near_clifford(14, 40, 20, 1e-3, seed=0),
    }


def _gpu_probs(text, shots, seed, precision, plain=False, product_components=True):
    import paper_2607_28600_b300 as S
    plan = S.symft_compile(text, product_components=product_components)
    info = plan.info
    W = (shots + 63) // 64
    meas = torch.zeros((max(1, info["n_records"]), W), dtype=torch.int64, device="cuda")
    prob = torch.full((max(1, info["n_causal"]), shots), float("nan"), dtype=torch.float64, device="cuda")
    S.symft_sample_ex(plan, shots, seed, meas_out=meas, precision=precision, check=True,
                      prob_out=prob, plain=plain)
    torch.cuda.synchronize()
    recs = unpack(meas.cpu().numpy().view(np.uint64)[: info["n_records"]], shots)
    return plan, recs, prob.cpu().numpy()[: info["n_causal"]]


def _sv_probs(text, seed, shots, active_t):
    c = oparse(text)
    noise = NoiseSampler(c, seed)
    probs = np.zeros((len(active_t), shots))
    for r in range(shots):
        log = []
        osv.sample_shot(c, seed, r, noise, prob_log=log)
        p = dict(log)
        probs[:, r] = [p[t] for t in active_t]
    return probs


@pytest.mark.parametrize("case", ["reg", "warp", "cta", "cta_global"])
def test_branch_probabilities_vs_statevector(case):
    text = _cases()[case]
    shots = {"reg": 500, "warp": 300, "cta": 120, "cta_global": 120}[case]
    seed = 21
    plan, rec64, p64 = _gpu_probs(text, shots, seed, precision=1)
    _, rec32, p32 = _gpu_probs(text, shots, seed, precision=0)
    act = plan.active_meas()
    k = plan.info["k_max"]
    assert {"reg": k <= 5, "warp": k == 10, "cta": k == 13, "cta_global": k == 14}[case]
    ref = _sv_probs(text, seed, shots, act)
    # FP64: every active measurement of every shot
    assert np.isfinite(p64).all()
    assert np.abs(p64 - ref).max() <= 1e-9
    o = oracle_sample(text, seed, range(shots), kind="sv")
    np.testing.assert_array_equal(rec64, o["records"])
    # FP32: prefixes up to and including the first flip
    flips, worst = 0, 0.0
    for r in range(shots):
        for j, t in enumerate(act):
            u = meas_uniform(seed, t, r)
            worst = max(worst, abs(p32[j, r] - ref[j, r]))
            if outcome_from(p32[j, r], u) != outcome_from(ref[j, r], u):
                flips += 1
                break
        else:
            np.testing.assert_array_equal(rec32[r], o["records"][r])
    assert worst <= 1e-5, worst
    assert flips <= max(1, shots // 50)


def _fp32_prefix_check(p32, ref, rec32, want_rec, act, seed, shots):
    """FP32 branch probabilities within 1e-5 of the reference on every active
    measurement up to and including a shot's first flip; unflipped shots'
    records bit-exact.  Returns (flips, worst error)."""
    flips, worst = 0, 0.0
    for r in range(shots):
        for j, t in enumerate(act):
            u = meas_uniform(seed, t, r)
            worst = max(worst, abs(p32[j, r] - ref[j, r]))
            if outcome_from(p32[j, r], u) != outcome_from(ref[j, r], u):
                flips += 1
                break
        else:
            np.testing.assert_array_equal(rec32[r], want_rec[r])
    return flips, worst


def test_wide_executor_fp32_branch_probabilities_k15():
    """The literal 15-to-1 circuit (16 qubits, k_max = 15) runs on the wide
    executor, whose FP32 vectors live in HBM: every branch probability up to a
    shot's first flip within 1e-5 of the state vector's Pr(m = 0) (2^16
    amplitudes, FP64), unflipped shots bit-exact, flips rare."""
    from paper_2607_28600_b300.workloads import distillation_15_to_1
    text = distillation_15_to_1(1e-3, "literal")
    shots, seed = 40, 31
    # the monolithic vector (the product-component form is tested on its own)
    plan, rec32, p32 = _gpu_probs(text, shots, seed, precision=0, product_components=False)
    assert plan.info["k_max"] == 15 and plan.info["dense_executor"] == ["wide", "wide"]
    act = plan.active_meas()
    assert len(act) >= 14
    ref = _sv_probs(text, seed, shots, act)
    o = oracle_sample(text, seed, range(shots), kind="sv")
    flips, worst = _fp32_prefix_check(p32, ref, rec32, o["records"], act, seed, shots)
    assert worst <= 1e-5, worst
    assert flips <= 1
    # FP64 on the same executor: every probability to 1e-9, records bit-exact
    _, rec64, p64 = _gpu_probs(text, shots, seed, precision=1, product_components=False)
    assert np.abs(p64 - ref).max() <= 1e-9
    np.testing.assert_array_equal(rec64, o["records"])


def test_plain_form_reports_the_same_probabilities():
    text = _cases()["warp"]
    _, r1, p1 = _gpu_probs(text, 64, 5, precision=1)
    _, r2, p2 = _gpu_probs(text, 64, 5, precision=1, plain=True)
    np.testing.assert_array_equal(r1, r2)
    assert np.abs(p1 - p2).max() <= 1e-12


@pytest.mark.parametrize("rot", [False, True])
def test_listed_postselection_bit_exact(rot):
    text = rotated_surface_code_memory(3, 3, 2e-2, t_on_data0_after_round=0 if rot else None)
    n_dets = oparse(text).num_dets
    listed = sorted(random.Random(8).sample(range(n_dets), n_dets // 3))
    shots = 900
    plan, meas, det, obs, disc = gpu_sample(text, shots, 3, precision=1, postselect=2, post_dets=listed)
    o = oracle_sample(text, 3, range(shots), postselect=2, post_dets=listed)
    g = {"records": unpack(meas, shots), "dets": unpack(det, shots), "obs": unpack(obs, shots),
         "discard": unpack(disc.reshape(1, -1), shots)[:, 0]}
    for key in ("discard", "records", "dets", "obs"):
        np.testing.assert_array_equal(g[key], o[key], err_msg=key)
    assert 0.02 < g["discard"].mean() < 0.98
    # the plain per-shot form applies the same rule
    import paper_2607_28600_b300 as S
    W = (shots + 63) // 64
    d2 = torch.zeros((n_dets, W), dtype=torch.int64, device="cuda")
    x2 = torch.zeros((W,), dtype=torch.int64, device="cuda")
    S.symft_sample_ex(plan, shots, 3, det_out=d2, discard_out=x2, precision=1, plain=True, check=True)
    np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), det)
    np.testing.assert_array_equal(x2.cpu().numpy().view(np.uint64), disc)


def _popcounts(obs, disc, shots):
    o = unpack(obs, shots)
    d = unpack(disc.reshape(1, -1), shots)[:, 0]
    kept = d == 0
    return [int(kept.sum()), int((~kept).sum())] + [int(o[kept, j].sum()) for j in range(o.shape[1])]


def test_counts_match_the_output_columns():
    import paper_2607_28600_b300 as S
    text = rotated_surface_code_memory(3, 3, 2e-2)
    shots = 5000
    plan, meas, det, obs, disc = gpu_sample(text, shots, 4, postselect=1)
    want = _popcounts(obs, disc, shots)
    n = 2 + plan.info["n_obs"]
    # device counts, every output requested
    c = torch.zeros((n,), dtype=torch.int64, device="cuda")
    W = (shots + 63) // 64
    ob = torch.zeros((plan.info["n_obs"], W), dtype=torch.int64, device="cuda")
    dc = torch.zeros((W,), dtype=torch.int64, device="cuda")
    S.symft_sample_ex(plan, shots, 4, obs_out=ob, discard_out=dc, counts_out=c, check=True)
    assert c.cpu().tolist() == want
    # counts alone: the library keeps the observable and discard columns itself
    c.zero_()
    S.symft_sample_ex(plan, shots, 4, counts_out=c, check=True)
    assert c.cpu().tolist() == want
    # host counts
    hc = np.zeros((n,), dtype=np.uint64)
    S.symft_sample_ex(plan, shots, 4, counts_out=hc, out_location=S.OUT_HOST)
    assert hc.tolist() == want
    # without postselection every shot is kept
    plan2 = S.symft_compile(text)
    c2 = torch.zeros((n,), dtype=torch.int64, device="cuda")
    ob2 = torch.zeros((plan2.info["n_obs"], W), dtype=torch.int64, device="cuda")
    S.symft_sample_ex(plan2, shots, 4, obs_out=ob2, counts_out=c2, check=True)
    got = c2.cpu().tolist()
    assert got[:2] == [shots, 0]
    assert got[2] == int(unpack(ob2.cpu().numpy().view(np.uint64), shots)[:, 0].sum())


def test_batch_job_counts():
    import paper_2607_28600_b300 as S
    text = rotated_surface_code_memory(3, 3, 2e-2)
    plan = S.symft_compile(text, postselect=1)
    shots = 3000
    W = (shots + 63) // 64
    n = 2 + plan.info["n_obs"]
    cs = [torch.zeros((n,), dtype=torch.int64, device="cuda") for _ in range(2)]
    ob = torch.zeros((plan.info["n_obs"], W), dtype=torch.int64, device="cuda")
    dc = torch.zeros((W,), dtype=torch.int64, device="cuda")
    jobs = [{"plan": 0, "shots": shots, "seed": 6, "counts_out": cs[0]},
            {"plan": 0, "shots": shots, "seed": 6, "obs_out": ob, "discard_out": dc,
             "counts_out": cs[1]}]
    S.symft_sample_batch([plan], jobs)
    torch.cuda.synchronize()
    want = _popcounts(ob.cpu().numpy().view(np.uint64), dc.cpu().numpy().view(np.uint64), shots)
    assert cs[0].cpu().tolist() == want and cs[1].cpu().tolist() == want


def _mask_by_postselection(text, rec, det, obs):
    """Apply the postselection rule (reject at the first fired detector in
    annotation order; later records and detectors and all observables read 0)
    to unpostselected outputs, from the circuit's event order."""
    c = oparse(text)
    rec, det, obs = rec.copy(), det.copy(), obs.copy()
    shots = rec.shape[0]
    disc = np.zeros(shots, dtype=np.uint8)
    cut = np.zeros(shots, dtype=bool)
    for op in c.ops:
        if op.kind == "meas" and op.rec >= 0:
            rec[cut, op.rec] = 0
        elif op.kind == "det":
            det[cut, op.index] = 0
            cut |= det[:, op.index] == 1
    obs[cut] = 0
    disc[cut] = 1
    return rec, det, obs, disc


@pytest.mark.parametrize("which,precision", [("literal", 0), ("literal", 1), ("coherent", 1)])
def test_early_exit_matches_masked_full_run(which, precision):
    """Shots rejected by a postselected detector stop their dense work early;
    every output still equals the full (unpostselected) run with the
    postselection rule applied afterwards."""
    from paper_2607_28600_b300.workloads import coherent_surface_code_memory, distillation_15_to_1
    text = (distillation_15_to_1(1e-3, "literal") if which == "literal"
            else coherent_surface_code_memory(5, 1, 1e-3, 0.02))
    shots = 3000 if which == "literal" else 1000
    _, m0, d0, o0, _ = gpu_sample(text, shots, 13, precision=precision, postselect=0)
    _, m1, d1, o1, x1 = gpu_sample(text, shots, 13, precision=precision, postselect=1)
    want = _mask_by_postselection(text, unpack(m0, shots), unpack(d0, shots), unpack(o0, shots))
    got = (unpack(m1, shots), unpack(d1, shots), unpack(o1, shots), unpack(x1.reshape(1, -1), shots)[:, 0])
    for w, g, name in zip(want, got, ("records", "dets", "obs", "discard")):
        np.testing.assert_array_equal(g, w, err_msg=name)
    assert 0.05 < got[3].mean() < 0.99


@pytest.mark.parametrize("which", ["coherent", "cultivation"])
def test_plain_form_early_exit_matches_batched(which):
    """Both forms of the paper's GPU design (in-kernel sampling and the
    packed-column prepass, one CTA per shot) end a rejected shot's dense work
    at once; their FP64 outputs equal the batched FP64 path bit for bit."""
    import paper_2607_28600_b300 as S
    from paper_2607_28600_b300.workloads import coherent_surface_code_memory, cultivation_shaped
    text = coherent_surface_code_memory(3, 3, 1e-3, 0.02) if which == "coherent" else cultivation_shaped(1e-3)
    plan = S.symft_compile(text, postselect=S.POSTSELECT_ALL)
    info = plan.info
    shots = 2000
    W = (shots + 63) // 64
    outs = []
    for plain in (S.PLAIN_OFF, S.PLAIN_IN_KERNEL, S.PLAIN_PREPASS):
        cols = [torch.zeros((max(1, info[k]), W), dtype=torch.int64, device="cuda")
                for k in ("n_records", "n_dets", "n_obs")]
        disc = torch.zeros((W,), dtype=torch.int64, device="cuda")
        S.symft_sample_ex(plan, shots, 17, meas_out=cols[0], det_out=cols[1], obs_out=cols[2],
                          discard_out=disc, precision=S.FP64, plain=plain, check=True)
        torch.cuda.synchronize()
        outs.append([c.cpu().numpy() for c in cols] + [disc.cpu().numpy()])
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            np.testing.assert_array_equal(a, b)
    assert 0.02 < unpack(outs[1][3].view(np.uint64).reshape(1, -1), shots).mean() < 0.99


@pytest.mark.parametrize("precision,bits", [(0, (10, 11, 13)), (1, (10, 12))])
def test_wide_tile_shapes_give_the_same_bits(precision, bits):
    """The wide executor's fused-window tile (2^bits amplitudes, a tuning
    parameter) only regroups the same per-amplitude updates into passes: the
    literal 15-to-1 circuit on the wide executor (k = 15) samples the same
    records for every tile size."""
    import paper_2607_28600_b300 as S
    from paper_2607_28600_b300.workloads import distillation_15_to_1
    text = distillation_15_to_1(1e-3, "literal")
    shots, seed = 256, 31
    outs = []
    for b in (0,) + tuple(bits):
        plan = S.symft_compile(text, postselect=1, product_components=False, executor="wide", wide_tile_bits=b)
        assert plan.info["dense_executor"][precision] == "wide"
        assert plan.info["wide_tile_bits"][precision] == (b or (12 if precision == 0 else 11))
        meas, det, obs, disc = S.sample_to_tensors(plan, shots, seed, precision=precision)
        outs.append([t.cpu().numpy() for t in (meas, det, obs, disc)])
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("precision", [0, 1])
def test_wide_register_phases_with_wide_pair_masks_against_the_oracle(precision):
    """Windows of the wide executor split into register phases; a rotation
    whose pair bits above the lanes do not fit in the register bits runs on
    the whole tile in shared memory between two register phases.  A random
    near-Clifford circuit (18 qubits, 20 rotations on weight-1..4 Paulis,
    k_max = 17) has such rotations in both precisions (host analysis of its
    windows: FP32 4 register phases and 2 shared-memory ones, FP64 6 and 2).
    Four shots on the wide executor, outcome by outcome and every active
    branch probability against the plain SymFT oracle: FP64 within 1e-9 and
    equal records; FP32 within 1e-5 up to a shot's first outcome flip."""
    import paper_2607_28600_b300 as S
    from oracle import symft as osymft
    text = random_near_clifford(18, 40, 20, 1e-3, seed=7)
    plan = S.symft_compile(text, product_components=False, executor="wide")
    info = plan.info
    assert info["k_max"] == 17 and info["dense_executor"][precision] == "wide"
    n, seed = 4, 9
    meas = torch.zeros((info["n_records"], 1), dtype=torch.int64, device="cuda")
    prob = torch.zeros((info["n_causal"], n), dtype=torch.float64, device="cuda")
    S.symft_sample_ex(plan, n, seed, meas_out=meas, precision=precision, prob_out=prob, check=True)
    torch.cuda.synchronize()
    recs = unpack(meas.cpu().numpy().view(np.uint64), n)
    c = oparse(text)
    act = plan.active_meas()
    for shot in range(n):
        log = []
        o = osymft.sample_shot(osymft.Plan(c), seed, shot, NoiseSampler(c, seed), prob_log=log)
        want = np.array([o[op.t] for op in c.ops if op.kind == "meas" and op.rec >= 0], dtype=np.uint8)
        ref = dict(log)
        got = prob.cpu().numpy()[:, shot]
        if precision == 1:
            np.testing.assert_array_equal(recs[shot], want)
            assert np.abs(got - np.array([ref[t] for t in act])).max() <= 1e-9
            continue
        flipped = False
        for j, t in enumerate(act):
            assert abs(got[j] - ref[t]) <= 1e-5, (shot, j, got[j], ref[t])
            if outcome_from(got[j], meas_uniform(seed, t, shot)) != outcome_from(ref[t], meas_uniform(seed, t, shot)):
                flipped = True
                break
        if not flipped:
            np.testing.assert_array_equal(recs[shot], want)
