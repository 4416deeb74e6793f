"""Host-side checks of the library (no GPU): C-ABI exports, the SAH build and its threaded
link sets (Sec. 3.1, Fig. 3), the instrumented host walk against the oracle, argument checks."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1505_06022_gb300 import gsp, inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "gsp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsp_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert len(names) >= 18
    L = gsp.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(gsp.ABI) == names
    assert L.gsp_status_string(-4) == b"traversal exceeded its step limit (corrupt BVH links)"


def links(nodes):
    miss = nodes[:, 3].view(np.int32).copy()
    word = nodes[:, 7].view(np.int32).copy()
    return miss, word


def check_threaded_tree(nodes, tris_packed, nt):
    """Structural invariants of one link set."""
    n = len(nodes)
    miss, word = links(nodes)
    internal = word < 0
    # always-true box test: hit links of internal nodes (i+1), leaves follow their miss link;
    # the walk must visit 0..n-1 in order and stop
    seq, node, steps = [], 0, 0
    while node >= 0 and steps <= 2 * n + 8:
        seq.append(node)
        node = node + 1 if internal[node] else miss[node]
        steps += 1
    assert seq == list(range(n))
    assert miss[n - 1] == -1
    # every miss link skips exactly the node's subtree: children of i are i+1 and miss[i+1],
    # and the second child's subtree ends where the parent's does
    end = np.where(miss < 0, n, miss)
    covered = np.zeros(nt, np.int32)
    for i in range(n):
        if internal[i]:
            a, b = i + 1, end[i + 1]
            assert b < end[i] and end[b] == end[i]
            for c in (a, b):  # child boxes inside the parent box
                assert np.all(nodes[c, 0:3] >= nodes[i, 0:3]) and np.all(nodes[c, 4:7] <= nodes[i, 4:7])
        else:
            assert end[i] == i + 1
            first, cnt = word[i] >> 3, word[i] & 7
            assert 1 <= cnt <= 7
            covered[first:first + cnt] += 1
            v0 = tris_packed[first:first + cnt, 0:3]
            v1 = tris_packed[first:first + cnt, 4:7]
            v2 = tris_packed[first:first + cnt, 8:11]
            for v in (v0, v1, v2):  # leaf box holds its triangles exactly
                assert np.all(v >= nodes[i, 0:3]) and np.all(v <= nodes[i, 4:7])
    assert np.all(covered == 1)  # leaves partition the triangles


def subtree_key(nodes, i, end, internal):
    return (tuple(nodes[i, 0:3]), tuple(nodes[i, 4:7]))


@pytest.mark.parametrize("which", ["cornell", "sphere"])
def test_six_link_sets_thread_the_same_tree(which):
    sc = I.cornell_box() if which == "cornell" else I.traversal_sphere(n=12)
    s = gsp.Scene(None, sc)
    stats = s.stats
    assert stats["link_sets"] == 6 and stats["nodes"] == 2 * stats["leaves"] - 1
    boxes = None
    for c in range(6):
        nodes, tris = gsp.bvh_export_full(s.h, sc.ntris, c)
        check_threaded_tree(nodes, tris, sc.ntris)
        miss, word = links(nodes)
        internal = word < 0
        end = np.where(miss < 0, len(nodes), miss)
        axis, sign = c // 2, (1.0 if c % 2 == 0 else -1.0)
        for i in np.nonzero(internal)[0]:  # children front to back along the class direction
            a, b = i + 1, end[i + 1]
            ka = sign * (nodes[a, axis] + nodes[a, 4 + axis])
            kb = sign * (nodes[b, axis] + nodes[b, 4 + axis])
            assert ka <= kb
        key = sorted(map(tuple, np.concatenate([nodes[:, 0:3], nodes[:, 4:7], (word >= 0)[:, None] * word[:, None].astype(np.float64)], 1).tolist()))
        boxes = key if boxes is None else boxes
        assert key == boxes  # the same nodes, only reordered


def test_build_is_deterministic_and_respects_leaf_limits():
    sc = I.traversal_sphere(n=16)
    a = gsp.Scene(None, sc)
    b = gsp.Scene(None, sc)
    na, ta = gsp.bvh_export_full(a.h, sc.ntris, 3)
    nb, tb = gsp.bvh_export_full(b.h, sc.ntris, 3)
    assert np.array_equal(na.view(np.int32), nb.view(np.int32)) and np.array_equal(ta, tb)
    s = gsp.Scene(None, sc, leaf_threshold=2, max_leaf=3)
    nodes, _ = gsp.bvh_export_full(s.h, sc.ntris, 0)
    word = nodes[:, 7].view(np.int32)
    assert np.all((word[word >= 0] & 7) <= 3)


def test_degenerate_centroids_are_split_by_count():
    # 40 copies of one triangle: no SAH split exists, leaves must still hold <= 7
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]] * 40, np.float32)
    t = np.arange(120, dtype=np.int32).reshape(40, 3)
    sc = I.Scene(v, t, np.zeros(40, np.int32), I.material(I.DIFFUSE, (0.5,) * 3), I.camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 40, 4, 4))
    s = gsp.Scene(None, sc)
    nodes, tris = gsp.bvh_export_full(s.h, 40, 0)
    check_threaded_tree(nodes, tris, 40)


@pytest.mark.parametrize("link_sets", [1, 6])
def test_host_walk_matches_oracle_closest_hit(link_sets):
    sc = I.traversal_sphere(n=20)
    rays = I.traversal_rays(64, 32, n_random=3000, seed=9)
    s = gsp.Scene(None, sc, link_sets=link_sets)
    tri, t, visits, tests = s.host_walk(rays)
    ids, tt, _, _, nd = O.Mesh(sc.verts, sc.tris).closest_hit(rays)
    sel = nd.astype(bool)
    assert sel.mean() > 0.98
    assert np.array_equal(tri[sel], ids[sel])
    hit = sel & (ids >= 0)
    np.testing.assert_allclose(t[hit], tt[hit], rtol=1e-5)


def test_multiple_threading_visits_fewer_nodes_than_single():
    sc = I.traversal_sphere(n=24)
    rays = I.traversal_rays(64, 32, n_random=4096, seed=4)
    v1 = gsp.Scene(None, sc, link_sets=1).host_walk(rays)[2].mean()
    v6 = gsp.Scene(None, sc, link_sets=6).host_walk(rays)[2].mean()
    assert v6 < 0.8 * v1


def test_upload_rejects_bad_input():
    sc = I.cornell_box()
    bad = sc.verts.copy()
    bad[3, 1] = np.nan
    with pytest.raises(gsp.GspError):
        gsp.gsp_scene_upload(None, bad, sc.tris, sc.tri_mat, sc.mats, sc.camera)
    bt = sc.tris.copy()
    bt[0, 0] = len(sc.verts)
    with pytest.raises(gsp.GspError):
        gsp.gsp_scene_upload(None, sc.verts, bt, sc.tri_mat, sc.mats, sc.camera)
    bm = sc.tri_mat.copy()
    bm[0] = len(sc.mats)
    with pytest.raises(gsp.GspError):
        gsp.gsp_scene_upload(None, sc.verts, sc.tris, bm, sc.mats, sc.camera)
    h = gsp.gsp_scene_upload(None, sc.verts, sc.tris, sc.tri_mat, sc.mats, sc.camera)
    with pytest.raises(gsp.GspError):
        gsp.gsp_build_bvh(h, bins=1)
    with pytest.raises(gsp.GspError):
        gsp.gsp_build_bvh(h, link_sets=3)
    with pytest.raises(gsp.GspError) as e:  # no BVH yet
        gsp.gsp_bvh_host_walk(h, I.random_rays(4, 0))
    assert e.value.code == -6
    gsp.gsp_scene_destroy(h)


def test_shading_data_argument_checks_on_a_host_scene():
    """gsp_scene_set_attributes / gsp_scene_set_texture validate on a host-only scene: zero or
    non-finite normals, textures without texture coordinates or on a non-diffuse material, sizes,
    negative texels, and coordinates that cannot be dropped while a texture uses them."""
    sc = I.full_scene(width=8, height=8, plane_quads=4, sphere_n=2)
    s = gsp.Scene(None, sc)
    nv = len(sc.verts)
    ok_n, ok_st = np.tile([0.0, 1.0, 0.0], (nv, 1)).astype(np.float32), np.zeros((nv, 2), np.float32)
    tex = np.full((4, 4, 3), 0.5, np.float32)
    for bad in (np.zeros((nv, 3), np.float32), np.full((nv, 3), np.nan, np.float32)):
        with pytest.raises(gsp.GspError):
            gsp.gsp_scene_set_attributes(s.h, bad, None)
    with pytest.raises(gsp.GspError):
        gsp.gsp_scene_set_attributes(s.h, None, np.full((nv, 2), np.inf, np.float32))
    with pytest.raises(gsp.GspError):  # no texture coordinates
        gsp.gsp_scene_set_texture(s.h, 0, tex)
    gsp.gsp_scene_set_attributes(s.h, ok_n, ok_st)
    for m, t in [(1, tex), (2, tex), (4, tex), (99, tex), (0, -tex), (0, np.zeros((0, 4, 3), np.float32))]:
        with pytest.raises(gsp.GspError):  # dielectric, mirror, emitter, out of range, negative, empty
            gsp.gsp_scene_set_texture(s.h, m, t)
    gsp.gsp_scene_set_texture(s.h, 0, tex)
    gsp.gsp_scene_set_texture(s.h, 3, tex)
    with pytest.raises(gsp.GspError):  # textures still use the coordinates
        gsp.gsp_scene_set_attributes(s.h, ok_n, None)
    gsp.gsp_scene_set_texture(s.h, 0, None)
    gsp.gsp_scene_set_texture(s.h, 3, None)
    gsp.gsp_scene_set_attributes(s.h, None, None)
    s.close()


def test_launch_timing_needs_a_device_scene():
    """gsp_trace_time_launches / gsp_trace_launch_times refuse a host-only scene (it has no device
    traversal to time) with GSP_ERR_INVALID_ARG, before any CUDA call."""
    s = gsp.Scene(None, I.cornell_box(width=8, height=8))
    for call in (lambda: gsp.gsp_trace_time_launches(s.h, 4), lambda: gsp.gsp_trace_launch_times(s.h, 4)):
        with pytest.raises(gsp.GspError) as e:
            call()
        assert e.value.code == -1
