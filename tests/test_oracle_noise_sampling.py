"""Pin of the oracle's sampled noise (oracle/noise.py, NoiseSampler.shot).

Every oracle simulator (state vector, tableau, plain SymFT) draws its noise
through NoiseSampler, so a mistake there (a wrong cell order, a wrong
threshold, a lane off by one) would agree with itself in every cross-check
between them.  Here sampled frequencies are checked against two things that
do not use the sampler:
  - closed forms of the channels (Sec. 2: a fired cell k applies the Pauli
    N_k with probability q * w_k / sum w): measured in Z, X and Y, the flip
    probabilities of PAULI_CHANNEL_1(px, py, pz) are px + py, py + pz and
    px + pz;
  - the exact outcome distribution from branch enumeration over every noise
    cell (statevector.exact_distribution),
within a 5-sigma binomial bound per outcome and a chi-square bound over all
outcomes.  Unequal weights make every permutation of the cells detectable.
"""
import math

import numpy as np
import pytest

from oracle import statevector as sv
from oracle.circuit import parse

PX, PY, PZ = 0.11, 0.23, 0.05

CIRCUITS = {
    # one channel per qubit, measured in Z, X and Y
    "pauli_channel_1": (f"H 1\nH 2\nS 2\n"
                        f"PAULI_CHANNEL_1({PX},{PY},{PZ}) 0 1 2\n"
                        "M 0\nMX 1\nMY 2\n"),
    # depolarizing on one and two qubits, several bases, a second layer
    "depolarize": ("H 1\n"
                   "DEPOLARIZE1(0.3) 0 1\n"
                   "DEPOLARIZE2(0.4) 0 1\n"
                   "M 0\nMX 1\n"),
    # X_ERROR then Y_ERROR on the same qubit (two channels in sequence)
    "sequence": "X_ERROR(0.2) 0\nY_ERROR(0.35) 0\nZ_ERROR(0.5) 0\nM 0\n",
}


def _frequencies(text, shots, seed):
    c = parse(text)
    out = sv.sample(c, seed, range(shots))["records"]
    keys, counts = np.unique(out, axis=0, return_counts=True)
    return {tuple(int(x) for x in k): int(n) for k, n in zip(keys, counts)}, c


def test_pauli_channel_1_closed_forms():
    d = sv.exact_distribution(parse(CIRCUITS["pauli_channel_1"]))
    marg = [sum(p for k, p in d.items() if k[i] == 1) for i in range(3)]
    assert marg[0] == pytest.approx(PX + PY, abs=1e-12)
    assert marg[1] == pytest.approx(PY + PZ, abs=1e-12)
    assert marg[2] == pytest.approx(PX + PZ, abs=1e-12)
    # independent channels: the joint law is the product of the marginals
    for k, p in d.items():
        want = math.prod(m if b else 1 - m for b, m in zip(k, marg))
        assert p == pytest.approx(want, abs=1e-12)


@pytest.mark.parametrize("name", sorted(CIRCUITS))
def test_sampled_noise_matches_exact_distribution(name):
    shots, seed = 12000, 4242
    freq, c = _frequencies(CIRCUITS[name], shots, seed)
    exact = sv.exact_distribution(c)
    assert set(freq) <= {k for k, p in exact.items() if p > 0}
    chi2, dof = 0.0, 0
    for k, p in exact.items():
        n = freq.get(k, 0)
        sd = math.sqrt(shots * p * (1 - p))
        assert abs(n - shots * p) <= 5 * sd + 1, (k, n, shots * p)
        if shots * p >= 5:
            chi2 += (n - shots * p) ** 2 / (shots * p)
            dof += 1
    # mean dof - 1, standard deviation sqrt(2 (dof - 1)): 6 sigma
    assert chi2 <= (dof - 1) + 6 * math.sqrt(2 * max(1, dof - 1)), (chi2, dof)


def test_flip_rates_of_a_wrong_cell_order_are_detectable():
    """The bound above separates the true law from the one a swapped cell table
    would give: measured in Z, X and Y the three flip rates differ by at least
    0.06, more than 10 binomial standard deviations at 12000 shots."""
    rates = sorted([PX + PY, PY + PZ, PX + PZ])
    sd = math.sqrt(0.34 * 0.66 / 12000)
    assert min(b - a for a, b in zip(rates, rates[1:])) >= 10 * sd
