"""Pins of the oracle's Philox4x64-10 and Box-Muller normals.

Philox is checked word for word against numpy's independent implementation
(numpy.random.Philox is the same 4x64-10 generator; it increments its 256-bit
counter before producing a block, so counter c is reached by seeding c-1)."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle


def _numpy_block(ctr, key):
    v = sum(int(x) << (64 * i) for i, x in enumerate(ctr)) - 1
    c = [(v >> (64 * i)) & (2 ** 64 - 1) for i in range(4)]
    return np.random.Philox(counter=np.array(c, dtype=np.uint64),
                            key=np.array([int(k) for k in key], dtype=np.uint64)).random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (0, 0)),
    ((0, 5, 2, 9), (20220110, 3)),
    ((123456789, 17, 1, 0), (2 ** 63 + 11, 2 ** 40 + 5)),
    ((2 ** 64 - 1, 2 ** 64 - 1, 7, 2 ** 33), (1, 2)),
])
def test_philox_matches_numpy(ctr, key):
    mine = oracle.philox4x64([np.uint64(x) for x in ctr], key)
    assert (mine == _numpy_block(ctr, key)).all()


def test_philox_vectorised_blocks():
    blk = np.arange(50, dtype=np.uint64)
    mine = oracle.philox4x64([blk, np.uint64(3), np.uint64(1), np.uint64(4)], (99, 7))
    for b in (0, 1, 17, 49):
        assert (mine[b] == _numpy_block((b, 3, 1, 4), (99, 7))).all()


def test_stream_normals_layout():
    """Normal i = Box-Muller of 32-bit halves of block i//8 (definition)."""
    z = oracle.stream_normals(5, 1, 12, oracle.PURPOSE_NC_W1, 3, 20)
    w = _numpy_block((2, 12, oracle.PURPOSE_NC_W1, 3), (5, 1))
    h = [int(w[1]) & 0xFFFFFFFF, int(w[1]) >> 32]          # pair 1 of block 2 = normals 18, 19
    u1 = ((h[0] >> 9) + 0.5) / 2 ** 23
    u2 = ((h[1] >> 9) + 0.5) / 2 ** 23
    r = math.sqrt(-2 * math.log(u1))
    assert z[18] == pytest.approx(r * math.cos(2 * math.pi * u2), rel=1e-15)
    assert z[19] == pytest.approx(r * math.sin(2 * math.pi * u2), rel=1e-15)


def test_stream_normals_are_standard_normal():
    z = oracle.stream_normals(11, 0, 4, oracle.PURPOSE_NC_W2, 0, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # distinct streams are uncorrelated
    z2 = oracle.stream_normals(11, 0, 5, oracle.PURPOSE_NC_W2, 0, 200000)
    assert abs(np.corrcoef(z, z2)[0, 1]) < 0.01


def test_gain_normals_are_standard_normal():
    z = np.array([oracle.gain_normal(3, 0, q, 0) for q in range(5000)])
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_omega_conventions_are_permutations():
    n = 96
    z1 = oracle.stream_normals(4, 2, 7, oracle.PURPOSE_NC_W1, 1, n)
    z2 = oracle.stream_normals(4, 2, 7, oracle.PURPOSE_NC_W2, 1, n)
    w1 = oracle.omega1(4, 2, 7, 1, n)
    w2 = oracle.omega2(4, 2, 7, 1, n)
    assert np.array_equal(np.sort(w1), np.sort(z1)) and np.array_equal(np.sort(w2), np.sort(z2))
    assert w1[0] == z1[0] and w1[1] == z1[n - 1] and w1[2] == z1[1] and w1[3] == z1[n - 2]
    assert w2[0] == z2[0] and w2[n // 2] == z2[1] and w2[5] == z2[10] and w2[n - 5] == z2[11]
