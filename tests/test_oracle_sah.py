"""Pins for the oracle's binned SAH split (Sec. 3.1: the tree is built top-down with the surface
area heuristic on the CPU, after Wald 2007), and the library's host build checked against it at
every node of three scenes.

The oracle's split is pinned by a hand-computed cost, by the textbook full sweep over every
position in centroid order (equal to the binned search when every centroid has a bin of its
own), and by a case whose answer is obvious. A median split, a cost without the node counts or
without the parent's area, or an off-by-one bin boundary fails one of them."""
import numpy as np
import pytest

import oracle as O
from paper_1505_06022_gb300 import gsp, inputs as I


def box_area(lo, hi):
    d = hi - lo
    return 2.0 * (d[0] * d[1] + d[1] * d[2] + d[2] * d[0])


def test_two_triangle_cost_by_hand():
    # unit right triangles at x = 0 and x = 3 in the plane z = 0: each box has area 2 (1 x 1
    # faces, both sides), the parent [0, 4] x [0, 1] x [0, 0] has area 8, so every boundary that
    # separates them costs 1 + (2 * 1 + 2 * 1) / 8 = 1.5; the first such boundary is 1
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [3, 0, 0], [4, 0, 0], [3, 1, 0]], np.float32)
    t = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    r = O.sah_split(v, t, [0, 1])
    assert r["split"] and r["axis"] == 0 and r["boundary"] == 1
    assert r["cost"] == 1.5
    assert list(r["left"]) == [0]
    # one triangle, or coincident centroids: no split
    assert not O.sah_split(v, t, [1])["split"]
    assert not O.sah_split(np.concatenate([v[:3], v[:3]]), t, [0, 1])["split"]


def triangle_around(c, half):
    """A triangle whose bounding box is c +- half exactly (so its centroid is c)."""
    return np.array([[c[0] - half[0], c[1] - half[1], c[2] - half[2]],
                     [c[0] + half[0], c[1], c[2] + half[2]],
                     [c[0], c[1] + half[1], c[2]]])


def test_binned_split_equals_the_full_sweep_when_bins_resolve_every_centroid():
    # 16 triangles whose centroids sit on 16 evenly spaced values along every axis (a different
    # permutation per axis): the 16 bins over the centroid range then hold one centroid each, and
    # the binned search must find the optimum of the textbook sweep over all 15 cuts of the
    # centroid order on all three axes
    rng = np.random.default_rng(7)
    k = np.arange(16)
    cen = np.stack([k * 0.5, rng.permutation(k) * 0.37 + 1.0, rng.permutation(k) * 0.61 - 2.0], 1)
    half = rng.uniform(0.02, 0.9, (16, 3))
    verts = np.concatenate([triangle_around(c, h) for c, h in zip(cen, half)]).astype(np.float32)
    tris = np.arange(48, dtype=np.int32).reshape(16, 3)
    lo = verts[tris].min(axis=1).astype(np.float64)
    hi = verts[tris].max(axis=1).astype(np.float64)
    c = 0.5 * (lo + hi)
    ap = box_area(lo.min(0), hi.max(0))
    best = (np.inf, None, None)
    for a in range(3):
        order = np.argsort(c[:, a], kind="stable")
        for i in range(1, 16):
            L, R = order[:i], order[i:]
            cost = 1.0 + (box_area(lo[L].min(0), hi[L].max(0)) * i +
                          box_area(lo[R].min(0), hi[R].max(0)) * (16 - i)) / ap
            if cost < best[0]:
                best = (cost, a, set(L.tolist()))
    r = O.sah_split(verts, tris, np.arange(16))
    assert r["split"] and r["axis"] == best[1]
    assert r["cost"] == pytest.approx(best[0], rel=1e-12)
    assert set(r["left"].tolist()) == best[2]
    assert r["near"] > 0.01  # no centroid near a bin boundary


def test_far_apart_clusters_are_separated():
    rng = np.random.default_rng(3)
    a = rng.normal(scale=0.05, size=(30, 3, 3)) + np.array([0.0, 0.0, 0.0])
    b = rng.normal(scale=0.05, size=(20, 3, 3)) + np.array([0.0, 0.0, 9.0])  # apart along z only
    verts = np.concatenate([a, b]).reshape(-1, 3).astype(np.float32)
    tris = np.arange(150, dtype=np.int32).reshape(50, 3)
    r = O.sah_split(verts, tris, rng.permutation(50))
    assert r["split"] and r["axis"] == 2
    assert sorted(r["left"].tolist()) == list(range(30))


# ---------------------------------------------------------------------------- the host build
def subtree_tris(nodes, tris_packed):
    """Triangle ids under every node of one exported link set (preorder, miss links)."""
    n = len(nodes)
    miss = nodes[:, 3].view(np.int32)
    word = nodes[:, 7].view(np.int32)
    end = np.where(miss < 0, n, miss)
    ids = tris_packed[:, 3].view(np.int32)
    leaf_ids = {}
    for i in range(n):
        if word[i] >= 0:
            first, cnt = word[i] >> 3, word[i] & 7
            leaf_ids[i] = ids[first:first + cnt].tolist()
    under = [sorted(sum((leaf_ids.get(j, []) for j in range(i, end[i])), [])) for i in range(n)]
    return under, end, word


def scenes():
    soup = I.random_soup(700, seed=21, size=0.2)
    plane_v, plane_t = I.displaced_plane(24, 2.0, seed=5, amp=0.3)
    # a regular grid puts centroids exactly on bin boundaries: move the vertices off the lattice
    plane_v[:, [0, 2]] += np.random.default_rng(6).uniform(-0.03, 0.03, (len(plane_v), 2))
    sphere = I.traversal_sphere(n=9, seed=8)
    return [("soup", soup.verts, soup.tris), ("plane", plane_v.astype(np.float32), plane_t.astype(np.int32)),
            ("sphere", sphere.verts, sphere.tris)]


@pytest.mark.parametrize("which", [0, 1, 2])
def test_host_build_picks_the_sah_split_at_every_node(which):
    name, verts, tris = scenes()[which]
    sc = I.Scene(verts, tris, np.zeros(len(tris), np.int32), I.material(I.DIFFUSE, (0.5,) * 3),
                 I.camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 40, 4, 4))
    leaf_thr, max_leaf = 4, 7
    s = gsp.Scene(None, sc, bins=16, leaf_threshold=leaf_thr, max_leaf=max_leaf, link_sets=1)
    nodes, packed = gsp.bvh_export_full(s.h, sc.ntris, 0)
    under, end, word = subtree_tris(nodes, packed)
    checked = skipped = 0
    for i in range(len(nodes)):
        sub = np.array(under[i], np.int32)
        r = O.sah_split(verts, tris, sub)
        if r["near"] < 1e-4:  # a centroid within FP32 rounding of a bin boundary
            skipped += 1
            continue
        count = len(sub)
        split_wanted = count > leaf_thr and not (count <= max_leaf and (not r["split"] or count <= r["cost"]))
        if word[i] >= 0:
            assert not split_wanted, (name, i, count, r)
        else:
            assert split_wanted, (name, i, count, r)
            if r["split"]:
                kids = [set(under[i + 1]), set(under[end[i + 1]])]
                assert set(r["left"].tolist()) in kids, (name, i)
        checked += 1
    assert checked > 0.97 * len(nodes) and checked > 150, (checked, skipped)
