"""Pins of the reference's random-number layer against things other than itself.

* Philox4x64-10 against numpy's independent implementation of the same
  generator (numpy.random.Philox, which advances the counter by one before
  each block).
* The unit-vector sampler (Algorithm 3, read as a uniform direction)
  against its definition: unit norm, the first accepted lattice point of the
  cube drawn from numpy's Philox stream, and uniformity of the angle (2D) and
  of cos(theta) and the azimuth (3D).
"""
import numpy as np
import pytest
from scipy import stats

import oracle

MASK = (1 << 64) - 1
TAG_MOVE = 0x53524D2D4D4F5645


def numpy_philox(ctr, key):
    c = 0
    for i, w in enumerate(ctr):
        c |= int(w) << (64 * i)
    c = (c - 1) & ((1 << 256) - 1)
    bg = np.random.Philox(counter=np.array([(c >> (64 * i)) & MASK for i in range(4)],
                                           dtype=np.uint64),
                          key=np.array(key, dtype=np.uint64))
    return bg.random_raw(4)


def test_philox_matches_numpy():
    rng = np.random.default_rng(12345)
    for _ in range(300):
        ctr = [int(x) for x in rng.integers(0, 2**64, size=4, dtype=np.uint64)]
        key = [int(x) for x in rng.integers(0, 2**64, size=2, dtype=np.uint64)]
        np.testing.assert_array_equal(oracle.philox4x64_10(ctr, key), numpy_philox(ctr, key))
    # the counter layouts the method uses: small ids, sweep, try, candidate
    for pid in (0, 1, 999, 2**32 + 5):
        for sweep in (0, 7):
            ctr = [pid, sweep, 3, 1]
            key = [42, TAG_MOVE]
            np.testing.assert_array_equal(oracle.philox4x64_10(ctr, key), numpy_philox(ctr, key))


def _lattice(words, dim):
    return np.array([float((int(w) >> 10) - (1 << 53)) * 2.0**-53 for w in words[:dim]])


@pytest.mark.parametrize("dim", [2, 3])
def test_unit_dir_is_first_accepted_lattice_point(dim):
    seed = 7
    for pid in range(60):
        for l in range(3):
            u, m = oracle.unit_dir(seed, 5, pid, l, dim)
            # candidates before m fall outside the unit ball, candidate m inside
            for mm in range(m + 1):
                v = _lattice(numpy_philox([pid, 5, l, mm], [seed, TAG_MOVE]), dim)
                s = float(np.sum(v * v))
                if mm < m:
                    assert not (0.0 < s <= 1.0)
                else:
                    assert 0.0 < s <= 1.0
                    # direction of v, unit length
                    np.testing.assert_allclose(u, v / np.sqrt(s), rtol=0, atol=4e-16)
            assert abs(np.linalg.norm(u) - 1.0) < 4e-16


def _sample(dim, n, seed=11):
    U = np.array([oracle.unit_dir(seed, 0, i, 0, dim)[0] for i in range(n)])
    return U


def test_unit_dir_uniform_2d():
    U = _sample(2, 20000)
    ang = np.arctan2(U[:, 1], U[:, 0])
    assert stats.kstest((ang + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3
    assert np.all(np.abs(U.mean(axis=0)) < 0.03)


def test_unit_dir_uniform_3d():
    U = _sample(3, 20000)
    # Archimedes: z = cos(theta) is uniform on [-1, 1] for a uniform direction
    assert stats.kstest((U[:, 2] + 1) / 2, "uniform").pvalue > 1e-3
    phi = np.arctan2(U[:, 1], U[:, 0])
    assert stats.kstest((phi + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3
    assert np.all(np.abs(U.mean(axis=0)) < 0.03)


def test_streams_distinct():
    a = oracle.unit_dir(1, 0, 0, 0, 3)[0]
    for args in [(2, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 0), (1, 0, 0, 1)]:
        b = oracle.unit_dir(*args, 3)[0]
        assert not np.array_equal(a, b)
