"""Pins for the oracle's exact hash grid (the index of the exact deposit): properties that hold
for any correct grid, independent of the hash formula."""
import numpy as np

import oracle as O


def test_grid_orders_by_bucket_then_index_and_starts_count():
    rng = np.random.default_rng(1)
    x = rng.normal(scale=0.5, size=(5000, 3)).astype(np.float32)
    T = 1024
    b, order, starts, near = O.hash_grid(x, 0.07, T)
    assert sorted(order.tolist()) == list(range(len(x)))           # a permutation
    key = b[order].astype(np.int64) * len(x) + order               # (bucket, index) ascending
    assert np.all(np.diff(key) > 0)
    np.testing.assert_array_equal(np.diff(starts), np.bincount(b, minlength=T))
    assert starts[0] == 0 and starts[-1] == len(x)
    assert np.all(b < T)


def test_points_of_one_cell_share_a_bucket_and_cells_spread():
    rng = np.random.default_rng(2)
    h = 0.25
    # 200 points inside one cell (away from its faces), lattice shifted by 0.381966 of a cell
    lo = (np.array([3, -2, 7]) - 0.381966) * h
    pts = (lo + rng.uniform(0.1, 0.9, (200, 3)) * h).astype(np.float32)
    b, _, _, near = O.hash_grid(pts, h, 1 << 16)
    assert np.all(b == b[0]) and not near.any()
    # one point per cell of a 40^3 block: buckets of distinct cells rarely collide
    g = np.stack(np.meshgrid(*[np.arange(40)] * 3, indexing="ij"), -1).reshape(-1, 3)
    centres = ((g + 0.5 - 0.381966) * h).astype(np.float32)
    b, _, _, _ = O.hash_grid(centres, h, 1 << 20)
    assert len(np.unique(b)) > 0.9 * len(g)
    # the flag marks coordinates on a cell face
    face = np.array([[(5 - 0.381966) * h, 0.1, 0.1]], np.float32)
    assert O.hash_grid(face, h, 64)[3][0] == 1
