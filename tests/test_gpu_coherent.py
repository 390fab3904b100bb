"""Coherent-noise surface-code workload (Sec. 7: R_Z(0.02) over-rotations with
circuit-level noise) on the GPU against the oracle: the large-active-width
path (k_max up to 24) through the C-ABI."""
import numpy as np
import pytest

from oracle import symft as osymft
from oracle.circuit import parse as oparse
from oracle.noise import NoiseSampler
from paper_2607_28600_b300.workloads import coherent_surface_code_memory
from tests.helpers import gpu_sample, oracle_sample, unpack

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gpu(text, shots, seed, precision):
    plan, meas, det, obs, disc = gpu_sample(text, shots, seed, precision=precision, postselect=1)
    return plan, {"records": unpack(meas, shots), "dets": unpack(det, shots), "obs": unpack(obs, shots),
                  "discard": unpack(disc.reshape(1, -1), shots)[:, 0]}


@pytest.mark.parametrize("d,r,shots,kind,kmax", [(3, 1, 120, "sv", 4), (3, 3, 300, "symft", 8),
                                                 (5, 1, 200, "symft", 12)])
def test_coherent_fp64_bit_exact(d, r, shots, kind, kmax):
    text = coherent_surface_code_memory(d, r, 1e-3, 0.02)
    plan, g = _gpu(text, shots, 9, precision=1)
    assert plan.info["k_max"] == kmax
    o = oracle_sample(text, 9, range(shots), postselect=1, kind=kind)
    for key in ("discard", "records", "dets", "obs"):
        np.testing.assert_array_equal(g[key], o[key], err_msg=key)
    # FP32: unflipped shots bit-exact, flips rare
    _, g32 = _gpu(text, shots, 9, precision=0)
    diff = (g32["records"] != o["records"]).any(axis=1)
    assert diff.mean() <= 0.02
    np.testing.assert_array_equal(g32["dets"][~diff], o["dets"][~diff])


@pytest.mark.parametrize("precision", [1, 0])
def test_coherent_k24_sampled_shot_against_the_oracle(precision):
    """d=5, 2 rounds reaches k_max = 24 (2^24 amplitudes per shot): one shot,
    every outcome and every active branch probability against the plain
    SymFT oracle (FP64).  FP64 vectors: every probability within 1e-9 and
    every record equal.  FP32 vectors (HBM-resident, FP64 branch sums): every
    probability up to the shot's first outcome flip within 1e-5, and the
    records equal if no flip occurs."""
    from oracle.streams import meas_uniform, outcome_from
    import paper_2607_28600_b300 as S
    text = coherent_surface_code_memory(5, 2, 1e-3, 0.02)
    shot, seed = 3, 5
    plan = S.symft_compile(text)
    assert plan.info["k_max"] == 24
    n = shot + 1
    W = (n + 63) // 64
    info = plan.info
    meas = torch.zeros((info["n_records"], W), dtype=torch.int64, device="cuda")
    prob = torch.zeros((info["n_causal"], n), dtype=torch.float64, device="cuda")
    S.symft_sample_ex(plan, n, seed, meas_out=meas, precision=precision, prob_out=prob, check=True)
    torch.cuda.synchronize()
    g = unpack(meas.cpu().numpy().view(np.uint64), n)[shot]
    c = oparse(text)
    log = []
    o = osymft.sample_shot(osymft.Plan(c), seed, shot, NoiseSampler(c, seed), prob_log=log)
    want = np.array([o[op.t] for op in c.ops if op.kind == "meas" and op.rec >= 0], dtype=np.uint8)
    ref = dict(log)
    got = prob.cpu().numpy()[:, shot]
    act = plan.active_meas()
    if precision == 1:
        np.testing.assert_array_equal(g, want)
        assert np.abs(got - np.array([ref[t] for t in act])).max() <= 1e-9
        return
    flipped = False
    for j, t in enumerate(act):
        assert abs(got[j] - ref[t]) <= 1e-5, (j, got[j], ref[t])
        u = meas_uniform(seed, t, shot)
        if outcome_from(got[j], u) != outcome_from(ref[t], u):
            flipped = True
            break
    if not flipped:
        np.testing.assert_array_equal(g, want)
