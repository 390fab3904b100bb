"""Pins for the oracle's Philox4x32-10 (published known answers + cuRAND)."""
import ctypes
import os

import numpy as np
import pytest

from oracle.philox import philox4x32, philox_scalar

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")


def test_known_answer_vectors():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert philox_scalar(v[0:4], v[4:6]) == tuple(v[6:10])


def _curand():
    for name in ("libcurand.so.10", "libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            pass
    return None


@pytest.mark.parametrize("seed", [0, 0x123456789ABCDEF0, 0xFFFFFFFF00000001])
def test_against_curand_host_generator(seed):
    """cuRAND's CURAND_RNG_PSEUDO_PHILOX4_32_10 host generator (run on CPU):
    its first 16384 output blocks for a seed are Philox(ctr=(0,0,j,0), key=seed)."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 4096
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    blocks = out.reshape(-1, 4).astype(np.uint64)
    j = np.arange(blocks.shape[0], dtype=np.uint64)
    o = philox4x32(0, 0, j, 0, seed & 0xFFFFFFFF, seed >> 32)
    for i in range(4):
        np.testing.assert_array_equal(o[i], blocks[:, i])


def test_vectorised_equals_scalar():
    rng = np.random.default_rng(3)
    c = rng.integers(0, 2**32, size=(50, 4), dtype=np.uint64)
    k = rng.integers(0, 2**32, size=(50, 2), dtype=np.uint64)
    o = philox4x32(c[:, 0], c[:, 1], c[:, 2], c[:, 3], k[:, 0], k[:, 1])
    for i in range(50):
        s = philox_scalar([int(x) for x in c[i]], [int(x) for x in k[i]])
        assert s == tuple(int(o[j][i]) for j in range(4))
