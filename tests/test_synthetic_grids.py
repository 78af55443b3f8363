"""The paper's grids as synthetic generators: the polar grid reproduces the point counts that
the paper prints for its polar-grid experiments (tests/golden/polar_grid_counts.txt)."""
import os

import numpy as np

from synthetic import polar_grid, random_grid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "polar_grid_counts.txt")


def test_polar_grid_point_counts_match_the_paper():
    rows = [tuple(int(v) for v in line.split()) for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    assert len(rows) == 5
    for n, M in rows:
        x, y = polar_grid(n)
        assert x.size == M, (n, x.size, M)
        assert np.all((x >= 0) & (x < 1) & (y >= 0) & (y < 1))
        # about 0.47 N log4 N points
        assert abs(M / (0.47 * n * n * np.log(n * n) / np.log(4)) - 1) < 0.05


def test_polar_grid_geometry():
    x, y = polar_grid(32)
    r = np.hypot(x - 0.5, y - 0.5)
    assert r[0] == 0 and np.isclose(r[1:].min(), np.sqrt(2) / 2 / 32)
    rings = np.unique(np.round(r[1:] * 32 / (np.sqrt(2) / 2), 9))
    assert np.allclose(rings, np.round(rings)) and rings.min() == 1 and rings.max() == 31


def test_random_grid():
    x, y = random_grid(1536, 9)
    assert x.size == 1536 and np.all((x >= 0) & (x < 1) & (y >= 0) & (y < 1))
    assert np.array_equal(x, random_grid(1536, 9)[0])
