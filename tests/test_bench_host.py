"""Host-side logic of bench.py: the extrapolated reference time of a whole
generation from per-sweep samples at a few states of the run."""
import pytest

import bench


def test_weighted_oracle_time_interpolates_and_weights():
    # per-sweep seconds: 1 at scale 1, 3 at scale 2 (linear in between)
    samples = [(1.0, 1.0), (2.0, 3.0)]
    # 10 sweeps around scale 1.0..1.2 (midpoint 1.1 -> 1.2 s), then 5 sweeps
    # around 1.8..2.0 (midpoint 1.9 -> 2.8 s), then 2 sweeps past the last sample
    record = [(1.0, 0), (1.2, 10), (1.8, 10), (2.0, 15), (2.2, 17)]
    got = bench.weighted_oracle_time(samples, record)
    assert got == pytest.approx(10 * 1.2 + 0 + 5 * 2.8 + 2 * 3.0)


def test_weighted_oracle_time_duplicate_scales():
    samples = [(1.0, 1.0), (1.5, 2.0), (1.5, 2.0)]
    record = [(1.0, 0), (1.5, 4)]
    assert bench.weighted_oracle_time(samples, record) == pytest.approx(4 * 1.5)
