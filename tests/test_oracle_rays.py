"""Pins of the oracle's ray sets against the geometry of the sphere: region counts, exactly equal
zone areas, unit directions, Leopardi's diameter bound, the Fibonacci lattice's z spacing."""
import math

import numpy as np
import pytest

from oracle import rays


@pytest.mark.parametrize("n", [1, 2, 3, 6, 7, 12, 33, 100, 1000, 10_000, 65_537])
def test_zonal_counts_areas_and_units(n):
    d = rays.zonal(n).astype(np.float64)
    assert d.shape == (n, 3)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
    cum, counts = rays.zonal_collars(n)
    assert cum[-1] == n and all(m >= 1 for m in counts)
    # each zone's area equals its region count times 4 pi / n (caps closing cumulative counts)
    for z in range(len(counts)):
        t0, t1 = rays.zone_theta(cum[z], n), rays.zone_theta(cum[z + 1], n)
        area = 2 * math.pi * (math.cos(t0) - math.cos(t1))
        assert abs(area - counts[z] * 4 * math.pi / n) <= 1e-9 * 4 * math.pi
        # every point of the zone lies inside its colatitude range
        th = np.arccos(np.clip(d[cum[z]:cum[z + 1], 2], -1, 1))
        assert np.all(th >= t0 - 1e-6) and np.all(th <= t1 + 1e-6)


@pytest.mark.parametrize("n", [100, 1000, 10_000])
def test_zonal_small_diameter(n):
    """Leopardi's bound for S^2: every region's diameter is below 7 / sqrt(n); hence each centre's
    nearest neighbour lies within it and no two centres coincide."""
    d = rays.zonal(n).astype(np.float64)
    rng = np.random.default_rng(0)
    idx = rng.choice(n, size=min(n, 300), replace=False)
    g = d[idx] @ d.T
    g[np.arange(len(idx)), idx] = -2.0
    nearest = np.arccos(np.clip(g.max(1), -1, 1))
    assert nearest.max() <= 7.0 / math.sqrt(n)
    assert nearest.min() > 0.0


def test_fibonacci_lattice():
    d = rays.fibonacci(1000).astype(np.float64)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
    assert np.allclose(np.diff(d[:, 2]), -2.0 / 1000, atol=1e-6)
