"""BVH built on the device (Morton-order LBVH, threaded into the packed MTBVH layout): the same
closest hits as the host SAH tree and the oracle, a well-formed threading for every link set,
and degenerate inputs (one triangle, coincident centroids)."""
import numpy as np
import pytest

import oracle as O
from paper_1505_06022_gb300 import gsp, inputs as I
from gpu_util import parity_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gsp.Context(0)
    yield c
    c.close()


def trace(scene, rays, method="mtbvh"):
    d = torch.from_numpy(np.ascontiguousarray(rays)).cuda()
    tri, t = scene.trace(d, method=method)
    torch.cuda.synchronize()
    return tri.cpu().numpy(), t.cpu().numpy()


@pytest.mark.parametrize("link_sets,max_leaf", [(6, 4), (1, 4), (6, 1), (6, 7)])
def test_device_bvh_same_hits(ctx, link_sets, max_leaf):
    sc = I.traversal_sphere(n=40, seed=7)
    rays = I.traversal_rays(128, 64, n_random=12000, seed=41)
    dev = gsp.Scene(ctx, sc, builder="device", link_sets=link_sets, max_leaf=max_leaf)
    host = gsp.Scene(ctx, sc)
    ids, tt, _, _, nd = O.Mesh(sc.verts, sc.tris).closest_hit(rays)
    a = trace(dev, rays)
    parity_hits(a[0], a[1], ids, tt, nd)
    b = trace(host, rays)
    sel = nd.astype(bool)
    assert np.array_equal(a[0][sel], b[0][sel])
    assert np.array_equal(a[1][sel].view(np.int32), b[1][sel].view(np.int32))
    s = trace(dev, rays, method="stack")
    assert np.array_equal(s[0][sel], a[0][sel])
    ctx.sync()
    assert dev.stats["nodes"] > 0 and dev.stats["depth"] > 0


def test_device_bvh_threading_is_well_formed(ctx):
    sc = I.random_soup(3001, seed=42, size=0.05)
    s = gsp.Scene(ctx, sc, builder="device", link_sets=6, max_leaf=4)
    for c in range(6):
        nodes, tris = gsp.bvh_export_full(s.h, sc.ntris, c)
        nn = len(nodes)
        miss = nodes[:, 3].view(np.int32)
        word = nodes[:, 7].view(np.int32)
        # following hit links under an always-hit test visits every node once, in order
        seen, node, steps = [], 0, 0
        while node >= 0 and steps <= 2 * nn:
            seen.append(node)
            node = node + 1 if word[node] < 0 else miss[node]
            node = -1 if node >= nn else node
            steps += 1
        assert seen == list(range(nn))
        # the leaves partition the triangles
        leaves = word[word >= 0]
        first, count = leaves >> 3, leaves & 7
        assert count.min() >= 1 and count.max() <= 4 and count.sum() == sc.ntris
        order = np.argsort(first)
        assert np.array_equal(np.cumsum(count[order])[:-1], first[order][1:])
        ids = np.sort(tris[:, 3].view(np.int32))
        assert np.array_equal(ids, np.arange(sc.ntris))
        # a node's box holds its subtree's triangles (checked on the leaves)
        for q in np.nonzero(word >= 0)[0][:200]:
            f, k = word[q] >> 3, word[q] & 7
            v = tris[f:f + k].reshape(k, 3, 4)[:, :, :3].reshape(-1, 3)
            assert (v >= nodes[q, 0:3] - 1e-6).all() and (v <= nodes[q, 4:7] + 1e-6).all()


def test_device_bvh_degenerate_inputs(ctx):
    # one triangle
    one = I.random_soup(1, seed=43)
    s1 = gsp.Scene(ctx, one, builder="device")
    rays = I.random_rays(4000, seed=44)
    ids, tt, _, _, nd = O.Mesh(one.verts, one.tris).closest_hit(rays, brute=True)
    a = trace(s1, rays)
    parity_hits(a[0], a[1], ids, tt, nd, max_excluded=1.0)
    assert np.array_equal(trace(s1, rays, method="stack")[0], a[0])
    # many triangles with the same centroid (identical Morton codes) and a duplicate-heavy soup
    base = I.random_soup(64, seed=45, size=0.2)
    v = base.verts.reshape(-1, 3, 3)
    v = v - v.mean(axis=1, keepdims=True)  # every centroid at the origin
    same = I.Scene(np.ascontiguousarray(v.reshape(-1, 3)), base.tris, base.tri_mat, base.mats, base.camera)
    s2 = gsp.Scene(ctx, same, builder="device", max_leaf=2)
    ids, tt, _, _, nd = O.Mesh(same.verts, same.tris).closest_hit(rays, brute=True)
    a = trace(s2, rays)
    parity_hits(a[0], a[1], ids, tt, nd)
    ctx.sync()


def test_sppm_on_device_bvh_matches_host_bvh(ctx):
    sc = I.full_scene(seed=9, width=64, height=48, plane_quads=32, sphere_n=6)
    params = gsp.sppm_params(sc, 20000, seed=8, r0_frac=0.01)
    imgs = []
    for builder in ("host", "device"):
        s = gsp.Scene(ctx, sc, builder=builder)
        r = gsp.Renderer(s, params)
        r.run(3)
        imgs.append(r.image().cpu().numpy())
        r.close()
        s.close()
    from gpu_util import image_parity
    image_parity(imgs[1], imgs[0], min_frac=0.9999)
