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


def test_teschner_buckets_by_hand():
    # Teschner et al. 2003: (ix * 73856093) ^ (iy * 19349663) ^ (iz * 83492791) in 32-bit
    # arithmetic, then mod the table size. Worked by hand:
    #   cell (1, 2, 3):   73856093 ^ 38699326 ^ 250478373 = 147163718; mod 2^20 = 363078
    #   cell (-1, 0, 5):  (2^32 - 73856093) ^ 0 ^ 417463955 = 4221111203 ^ 417463955
    #                     = 3816355120; mod 2^20 = 587056
    #   cell (7, -3, -2): 516992651 ^ 4236918307 ^ 4127981714 = 341217338; mod 2^16 = 36922
    # A wrong constant, + instead of ^, or a negative cell that does not wrap mod 2^32 fails.
    h = 0.25
    cells = np.array([[1, 2, 3], [-1, 0, 5], [7, -3, -2]], np.float64)
    pts = ((cells + 0.5 - 0.381966) * h).astype(np.float32)  # cell centres of the shifted lattice
    b, _, _, near = O.hash_grid(pts[:2], h, 1 << 20)
    assert list(b) == [363078, 587056] and not near.any()
    b, _, _, _ = O.hash_grid(pts[2:], h, 1 << 16)
    assert list(b) == [36922]
