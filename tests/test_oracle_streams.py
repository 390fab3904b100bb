"""Pins for the shared random-stream specification (oracle side)."""
import math

import numpy as np
import pytest

from oracle import streams as S


def test_theta_table_is_the_geometric_cdf():
    for q in (1e-3, 0.01, 0.3, 0.999):
        th = S.theta_table(q)
        assert len(th) == S.NOISE_BLOCK
        assert all(th[i] <= th[i + 1] for i in range(len(th) - 1))
        for j in (0, 1, 63, 127, 511):
            exact = (1.0 - (1.0 - q) ** (j + 1)) * 2.0 ** 32
            assert abs(th[j] - exact) <= 2.0 + 1e-9 * exact
    assert S.theta_table(0.0) == [0] * S.NOISE_BLOCK
    assert S.theta_table(1.0)[0] == 0xFFFFFFFF


def test_phi_table():
    assert S.phi_table([1.0]) == []
    ph = S.phi_table([1.0, 1.0, 1.0])
    assert ph == [int(2 ** 32 / 3), int(2 * 2 ** 32 / 3)]
    ph = S.phi_table([0.1, 0.0, 0.3])
    assert ph[0] == ph[1] == int(0.25 * 2 ** 32)


def test_first_fire_law_brute_force():
    """The first fired lane is min{j : u < THETA_j}: enumerate u over all cells."""
    q = 0.05
    th = S.theta_table(q)
    # probability mass of 'first fire at lane j' = (THETA_j - THETA_{j-1}) / 2^32
    prev = 0
    for j in range(S.NOISE_BLOCK):
        mass = (th[j] - prev) / 2.0 ** 32
        assert abs(mass - q * (1 - q) ** j) < 1e-9
        prev = th[j]


def _lane_matrix(q, weights, n_blocks, seed=5, c=7):
    th, ph = S.theta_table(q), S.phi_table(weights)
    fired = np.zeros((n_blocks, S.NOISE_BLOCK), dtype=np.int8) - 1
    for b in range(n_blocks):
        for lane, cell in S.channel_block_fires(seed, c, b, th, ph):
            fired[b, lane] = cell
    return fired


def test_lane_marginals_bernoulli():
    q = 0.03
    f = _lane_matrix(q, [1.0], 400)
    hits = (f >= 0)
    n = hits.size
    rate = hits.mean()
    assert abs(rate - q) < 5 * math.sqrt(q * (1 - q) / n)
    # every lane, not only early ones
    per_lane = hits.mean(axis=0)
    assert abs(per_lane[:64].mean() - per_lane[64:].mean()) < 0.02
    assert abs(per_lane[448:].mean() - q) < 0.012


def test_lane_pairs_independent_and_cells_uniform():
    q = 0.2
    f = _lane_matrix(q, [1.0, 1.0, 1.0], 600)
    hits = (f >= 0).astype(float)
    both = (hits[:, :-1] * hits[:, 1:]).mean()
    assert abs(both - q * q) < 0.006
    cells = f[f >= 0]
    for k in range(3):
        assert abs((cells == k).mean() - 1 / 3) < 0.02


def test_process_stops_and_orders_lanes():
    th, ph = S.theta_table(0.5), S.phi_table([1, 1, 1])
    fires = S.channel_block_fires(1, 3, 9, th, ph)
    lanes = [l for l, _ in fires]
    assert lanes == sorted(set(lanes)) and all(0 <= l < S.NOISE_BLOCK for l in lanes)
    assert S.channel_block_fires(1, 3, 9, S.theta_table(0.0), []) == []


def test_measurement_uniform_rule():
    seed = 99
    for t in (0, 5):
        for r in (0, 1, 63, 64, 130, 1 << 20):
            u = S.meas_uniform(seed, t, r)
            bit = (S.mbit_word(seed, t, r >> 6) >> (r & 63)) & 1
            assert 0.0 <= u < 1.0
            assert S.outcome_from(0.5, u) == bit          # Pr = 1/2: the MBIT bit
            assert S.outcome_from(1.0, u) == 0
            assert S.outcome_from(0.0, u) == 1
            assert (u * 2 ** 53) == int(u * 2 ** 53)        # a multiple of 2^-53


def test_mbit_words_vector_matches_scalar():
    v = S.mbit_words(7, 11, 1000, 9)
    for i in range(9):
        assert int(v[i]) == S.mbit_word(7, 11, 1000 + i)


def test_bisection_equals_the_linear_first_index():
    """The bisection in the process returns the linear scan's min{j : u < THETA_j}."""
    import random
    from bisect import bisect_right
    rng = random.Random(3)
    for q in (1e-3, 0.02, 0.4):
        th = S.theta_table(q)
        for _ in range(300):
            u = rng.choice([rng.getrandbits(32), th[rng.randrange(S.NOISE_BLOCK)],
                            max(0, th[rng.randrange(S.NOISE_BLOCK)] - 1)])
            lin = next((j for j in range(S.NOISE_BLOCK) if u < th[j]), S.NOISE_BLOCK)
            assert bisect_right(th, u) == lin
