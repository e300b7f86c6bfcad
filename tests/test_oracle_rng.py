"""Pins for oracle.rng: published Philox KAT vectors and Gaussian moments."""
import os

import numpy as np
import pytest

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x, 16) for x in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat())
def test_philox_known_answers(row):
    c, k, want = row[:4], row[4:6], row[6:]
    got = rng.philox4x32_10(*[np.array([x], dtype=np.uint64) for x in c], k[0], k[1])
    assert [int(g[0]) for g in got] == want


def test_gaussian_is_a_pure_function_of_the_counter():
    a = rng.gaussian(7, rng.stream_id(rng.STAGE_W, 3), np.arange(100), 0, 8)
    b = rng.gaussian(7, rng.stream_id(rng.STAGE_W, 3), np.arange(50, 100), 3, 8)
    assert np.array_equal(a[50:, 3:], b)            # any sub-block, same values
    c = rng.gaussian(7, rng.stream_id(rng.STAGE_W, 4), np.arange(100), 0, 8)
    d = rng.gaussian(8, rng.stream_id(rng.STAGE_W, 3), np.arange(100), 0, 8)
    assert not np.allclose(a, c) and not np.allclose(a, d)


def test_gaussian_moments():
    z = rng.gaussian(123, rng.stream_id(rng.STAGE_R, 2), np.arange(20000), 0, 20).ravel()
    N = z.size
    assert abs(z.mean()) < 5 / np.sqrt(N)
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 5 * np.sqrt(1.0 / N)     # E|z|^2 = 1
    assert abs(np.mean(z * z)) < 5 / np.sqrt(N)                            # circular: E z^2 = 0
    re = np.sqrt(2) * z.real
    assert abs(np.mean(re ** 4) - 3.0) < 0.1                               # normal kurtosis
    # adjacent rows (shared Philox call) are uncorrelated
    zz = rng.gaussian(5, 1, np.arange(20000), 0, 1)[:, 0]
    assert abs(np.mean(zz[0::2] * np.conj(zz[1::2]))) < 5 / np.sqrt(10000)
