"""Pins of the reference's random-number layer against things other than itself.

* Philox4x32-10 against the known-answer vectors published with the
  generator (tests/golden/philox4x32_10_kat.txt).
* The unit-vector sampler (Algorithm 3, read as a uniform direction)
  against its definition: unit norm, the first accepted lattice point of the
  cube drawn from the (pinned) Philox blocks at the documented counters, and
  uniformity of the angle (2D) and of cos(theta) and the azimuth (3D).
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")


def kat_vectors():
    out = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out.append((w[0:4], w[4:6], w[6:10]))
    return out


def test_philox_known_answers():
    vs = kat_vectors()
    assert len(vs) == 3
    for ctr, key, want in vs:
        np.testing.assert_array_equal(oracle.philox4x32_10(ctr, key), np.array(want, dtype=np.uint32))


def test_philox_counter_words_matter():
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert not np.array_equal(oracle.philox4x32_10(c, [5, 6]), base)
    for i in range(2):
        k = [5, 6]
        k[i] ^= 1
        assert not np.array_equal(oracle.philox4x32_10([1, 2, 3, 4], k), base)


def _block(seed, sweep, pid, l, m):
    ctr = [pid & 0xFFFFFFFF, sweep & 0xFFFFFFFF, (l + (m << 16)) & 0xFFFFFFFF, (sweep >> 32) & 0xFFFFFFFF]
    return oracle.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])


def _lattice(words, dim):
    return np.array([float(int(w) - (1 << 31)) * 2.0**-31 for w in words[:dim]])


@pytest.mark.parametrize("dim", [2, 3])
def test_unit_dir_is_first_accepted_lattice_point(dim):
    for seed, sweep in ((7, 5), (2**40 + 3, 2**33 + 9)):
        for pid in range(60):
            for l in range(3):
                u, m = oracle.unit_dir(seed, sweep, pid, l, dim)
                # candidates before m fall outside the unit ball, candidate m inside
                for mm in range(m + 1):
                    v = _lattice(_block(seed, sweep, pid, l, mm), dim)
                    s = float(np.sum(v * v))
                    if mm < m:
                        assert not (0.0 < s <= 1.0)
                    else:
                        assert 0.0 < s <= 1.0
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
    for args in [(2, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 0), (1, 0, 0, 1), (2**32 + 1, 0, 0, 0), (1, 2**32, 0, 0)]:
        b = oracle.unit_dir(*args, 3)[0]
        assert not np.array_equal(a, b)
