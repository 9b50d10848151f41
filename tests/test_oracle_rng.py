"""Pins for the oracle's ray generation (Sec. 3.1): its Philox4x64-10 against
numpy's independent implementation, the (0,1) mapping, and uniform-area
sampling of the lens disk."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle


def _numpy_philox_block(counter, key):
    # numpy's Philox increments its 256-bit counter *before* producing a
    # block, so start it one below the counter we want.
    c = int(counter[0]) | int(counter[1]) << 64 | int(counter[2]) << 128 | int(counter[3]) << 192
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=(c - 1) % (1 << 256))
    return bg.random_raw(4)


@pytest.mark.parametrize("seed", [0, 1, 2, 99])
def test_philox_matches_numpy(seed):
    rng = np.random.default_rng(seed)
    for _ in range(50):
        ctr = [int(x) for x in rng.integers(0, 2**63, 4, dtype=np.uint64)]
        if seed == 99:
            ctr = [int(rng.integers(0, 100)), int(rng.integers(0, 1000)), 0, 0]
        key = [int(x) for x in rng.integers(0, 2**63, 2, dtype=np.uint64)]
        assert np.array_equal(oracle.philox4x64(ctr, key), _numpy_philox_block(ctr, key))


def test_u01_open_interval_and_resolution():
    assert oracle.u01(0) == 0.5 * 2.0 ** -53
    assert oracle.u01(2**64 - 1) == 1.0 - 0.5 * 2.0 ** -53
    assert 0.0 < oracle.u01(2**63) < 1.0
    assert oracle.u01(2**63) == 0.5 + 0.5 * 2.0 ** -53


def test_u01_uniform_chi_square():
    n = 20000
    words = np.array([oracle.philox4x64([i, 3, 0, 0], [7, 0])[0] for i in range(n)], dtype=np.uint64)
    u = np.array([oracle.u01(int(w)) for w in words])
    hist, _ = np.histogram(u, bins=50, range=(0, 1))
    chi2 = ((hist - n / 50) ** 2 / (n / 50)).sum()
    assert stats.chi2.sf(chi2, 49) > 1e-4


def test_lens_points_uniform_over_disk():
    a, z = 0.0125, 1.1
    n = 20000
    pts = np.array([oracle.lens_point(5, 17, i, 0, a, z) for i in range(n)])
    assert np.all(pts[:, 2] == z)
    r2 = (pts[:, 0] ** 2 + pts[:, 1] ** 2) / a**2
    assert r2.max() <= 1.0
    # equal-area annuli <=> r^2/a^2 uniform on (0,1); angle uniform on (-pi, pi]
    h1, _ = np.histogram(r2, bins=40, range=(0, 1))
    h2, _ = np.histogram(np.arctan2(pts[:, 1], pts[:, 0]), bins=40, range=(-math.pi, math.pi))
    for h in (h1, h2):
        chi2 = ((h - n / 40) ** 2 / (n / 40)).sum()
        assert stats.chi2.sf(chi2, 39) > 1e-4


def test_lens_point_keyed_by_source_ray_frame_seed():
    base = oracle.lens_point(1, 2, 3, 4, 0.01, 1.0)
    for args in [(2, 2, 3, 4), (1, 3, 3, 4), (1, 2, 4, 4), (1, 2, 3, 5)]:
        assert not np.allclose(oracle.lens_point(*args, 0.01, 1.0), base)
    assert np.array_equal(oracle.lens_point(1, 2, 3, 4, 0.01, 1.0), base)
