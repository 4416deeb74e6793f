"""Pins for the oracle's closest-hit queries (Fig. 3 leaf test, Moller-Trumbore).

The oracle's brute force is checked against an independent formulation (a batched LU solve
of o + t d = v0 + u e1 + v e2), closed forms, and the tie/edge rules; the oracle BVH is
checked against brute force.
"""
import numpy as np
import pytest

import oracle as O
from paper_1505_06022_gb300 import inputs as I


def lu_closest(verts, tris, rays):
    """Closest hit by solving [e1 e2 -d] [u v t]^T = o - v0 with numpy.linalg.solve (FP64)."""
    v = verts.astype(np.float64)[tris]
    v0, e1, e2 = v[:, 0], v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]
    ids = np.full(len(rays), -1)
    ts = np.full(len(rays), np.inf)
    for i, r in enumerate(rays.astype(np.float64)):
        o, d, tmin, tmax = r[0:3], r[4:7], r[3], r[7]
         # singular systems (ray parallel to the plane) are skipped
        A = np.stack([e1, e2, np.broadcast_to(-d, e1.shape)], axis=-1)
        ok = np.abs(np.linalg.det(A)) > 1e-300
        sol = np.full((len(tris), 3), np.nan)
        sol[ok] = np.linalg.solve(A[ok], (o - v0)[ok][..., None])[..., 0]
        u, w, t = sol[:, 0], sol[:, 1], sol[:, 2]
        good = ok & (u >= 0) & (w >= 0) & (u + w <= 1) & (t > tmin) & (t < tmax)
        if good.any():
            cand = np.nonzero(good)[0]
            best = cand[np.lexsort((cand, t[cand]))[0]]
            ids[i], ts[i] = best, t[best]
    return ids, ts


def test_mt_closed_form_axis_aligned():
    hit, t, u, v = O.mt([0, 0, 0], [1, 0, 0], [0, 1, 0], [0.2, 0.3, 5, 0, 0, 0, -1, np.inf])
    assert hit and t == pytest.approx(5.0, abs=1e-12)
    assert u == pytest.approx(0.2, abs=1e-7) and v == pytest.approx(0.3, abs=1e-7)
    # oblique ray: t is the distance along d to the plane z = 0
    d = np.array([0.3, -0.2, -1.0])
    d /= np.linalg.norm(d)
    hit, t, _, _ = O.mt([0, 0, 0], [1, 0, 0], [0, 1, 0], [0.1, 0.5, 2, 0, *d, np.inf])
    assert hit and t == pytest.approx(2.0 / -d[2], rel=1e-6)
    # parallel ray: det == 0 -> miss
    hit, *_ = O.mt([0, 0, 0], [1, 0, 0], [0, 1, 0], [0.2, 0.2, 1, 0, 1, 0, 0, np.inf])
    assert not hit
    # outside the triangle (u + v > 1)
    hit, *_ = O.mt([0, 0, 0], [1, 0, 0], [0, 1, 0], [0.6, 0.6, 1, 0, 0, 0, -1, np.inf])
    assert not hit


def test_brute_force_matches_lu_solve():
    sc = I.random_soup(48, seed=11)
    rays = I.random_rays(1500, seed=12)
    mesh = O.Mesh(sc.verts, sc.tris)
    ids, t, *_ , nd = mesh.closest_hit(rays, brute=True)
    ref_ids, ref_t = lu_closest(sc.verts, sc.tris, rays)
    sel = nd.astype(bool)
    assert sel.mean() > 0.95
    assert np.array_equal(ids[sel], ref_ids[sel])
    hit = sel & (ids >= 0)
    assert hit.sum() > 150
    np.testing.assert_allclose(t[hit], ref_t[hit], rtol=1e-9)


@pytest.mark.parametrize("kind", ["soup", "sphere"])
def test_bvh_matches_brute_force(kind):
    if kind == "soup":
        sc = I.random_soup(3000, seed=21, size=0.1)
        rays = I.random_rays(8000, seed=22)
    else:
        sc = I.traversal_sphere(n=24, seed=2)
        rays = I.traversal_rays(64, 32, n_random=4096, seed=23)
    mesh = O.Mesh(sc.verts, sc.tris)
    a = mesh.closest_hit(rays, brute=True)
    b = mesh.closest_hit(rays, brute=False)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[4], b[4])
    assert (a[0] >= 0).mean() > 0.2


def test_range_is_open_and_ties_pick_smaller_id():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    verts = np.concatenate([v, v])  # the same triangle twice
    tris = np.array([[3, 4, 5], [0, 1, 2]], np.int32)
    mesh = O.Mesh(verts, tris)
    ray = np.array([[0.2, 0.2, 1, 0, 0, 0, -1, np.inf]], np.float32)
    ids, t, *_ = mesh.closest_hit(ray, brute=True)
    assert ids[0] == 0 and t[0] == 1.0  # equal t: lower triangle id wins
    ray_t = ray.copy()
    ray_t[0, 7] = 1.0  # tmax == t excluded
    assert mesh.closest_hit(ray_t, brute=True)[0][0] == -1
    ray_t = ray.copy()
    ray_t[0, 3] = 1.0  # tmin == t excluded
    assert mesh.closest_hit(ray_t, brute=True)[0][0] == -1
    # an edge is inside (u + v == 1 exactly)
    edge = np.array([[0.5, 0.5, 1, 0, 0, 0, -1, np.inf]], np.float32)
    ids, _, _, _, nd = mesh.closest_hit(edge, brute=True)
    assert ids[0] == 0 and nd[0] == 0  # hit, but flagged degenerate


def test_classification_flags_shared_edges():
    # two triangles sharing the edge x + y = 1 in the plane z = 0
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], np.float32)
    tris = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    mesh = O.Mesh(verts, tris)
    rays = np.array([[0.5, 0.5, 1, 0, 0, 0, -1, np.inf],      # on the shared edge
                     [0.25, 0.25, 1, 0, 0, 0, -1, np.inf],    # inside triangle 0
                     [0.75, 0.75, 1, 0, 0, 0, -1, np.inf],    # inside triangle 1
                     [0.5, 0.5, 1, 0, 1, 0, 0, np.inf],       # grazing (parallel) miss
                     [3, 3, 1, 0, 0, 0, -1, np.inf]], np.float32)
    ids, t, u, v, nd = mesh.closest_hit(rays, brute=True)
    assert list(ids) == [0, 0, 1, -1, -1]
    assert list(nd) == [0, 1, 1, 1, 1]
