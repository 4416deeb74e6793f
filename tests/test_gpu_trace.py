"""GPU closest-hit traversal (Fig. 3, MTBVH and TBVH) against the oracle, through the C-ABI."""
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


def gpu_trace(ctx, sc, rays, method="mtbvh", **bvh):
    s = gsp.Scene(ctx, sc, **bvh)
    d = torch.from_numpy(np.ascontiguousarray(rays)).cuda()
    tri, t, uv = s.trace(d, with_uv=True, method=method)
    torch.cuda.synchronize()
    ctx.sync()
    return tri.cpu().numpy(), t.cpu().numpy(), uv.cpu().numpy(), s


def test_rng_streams_are_bit_exact():
    c = gsp.Context(0)
    ids = np.arange(1 << 22, dtype=np.uint64) * 7919 + 3
    g = gsp.gsp_rng_fill(c.h, 12345, 2, 1, 9, torch.from_numpy(ids.view(np.int64)).cuda(), 24)
    torch.cuda.synchronize()
    got = g.cpu().numpy()
    want = O.rng_draws(12345, 2, 1, 9, ids, 24)  # ~10^8 draws
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    c.close()


@pytest.mark.parametrize("method", ["mtbvh", "stack"])
def test_soup_against_brute_force(ctx, method):
    sc = I.random_soup(300, seed=31, size=0.15)
    rays = I.random_rays(20011, seed=32)  # ragged count
    tri, t, uv, _ = gpu_trace(ctx, sc, rays, method=method)
    ids, tt, uu, vv, nd = O.Mesh(sc.verts, sc.tris).closest_hit(rays, brute=True)
    parity_hits(tri, t, ids, tt, nd)
    hit = nd.astype(bool) & (ids >= 0)
    np.testing.assert_allclose(uv[hit, 0], uu[hit], atol=1e-4)
    np.testing.assert_allclose(uv[hit, 1], vv[hit], atol=1e-4)


@pytest.mark.parametrize("link_sets", [1, 6])
def test_sphere_both_link_sets(ctx, link_sets):
    sc = I.traversal_sphere(n=40, seed=2)
    rays = I.traversal_rays(128, 64, n_random=8192, seed=33)
    tri, t, _, _ = gpu_trace(ctx, sc, rays, link_sets=link_sets)
    ids, tt, _, _, nd = O.Mesh(sc.verts, sc.tris).closest_hit(rays)
    parity_hits(tri, t, ids, tt, nd)


def test_stack_traversal_agrees_with_mtbvh(ctx):
    """Both traversals return the lexicographic minimum over the same FP32 triangle tests."""
    sc = I.traversal_sphere(n=40, seed=6)
    rays = I.traversal_rays(128, 64, n_random=16384, seed=36)
    a = gpu_trace(ctx, sc, rays, method="stack")
    b = gpu_trace(ctx, sc, rays)
    ids, tt, _, _, nd = O.Mesh(sc.verts, sc.tris).closest_hit(rays)
    parity_hits(a[0], a[1], ids, tt, nd)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.int32), b[1].view(np.int32))


def test_link_sets_agree_bitwise(ctx):
    sc = I.traversal_sphere(n=32, seed=5)
    rays = I.traversal_rays(96, 48, n_random=6000, seed=34)
    a = gpu_trace(ctx, sc, rays, link_sets=1)
    b = gpu_trace(ctx, sc, rays, link_sets=6)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.int32), b[1].view(np.int32))


def test_edge_cases(ctx):
    sc = I.cornell_box()
    s = gsp.Scene(ctx, sc)
    # n == 0 is a no-op
    empty = torch.zeros((0, 8), device="cuda")
    gsp.gsp_trace_closest_hit(s.h, empty, torch.zeros(0, dtype=torch.int32, device="cuda"),
                              torch.zeros(0, device="cuda"))
    # axis-aligned directions (zero components), a finite tmax before the hit, tmin past it,
    # origins outside pointing away, one ray alone and a ragged batch of 33
    rays = np.array([[0.5, 0.5, 0.5, 0, 0, 0, -1, np.inf],
                     [0.5, 0.5, 0.5, 0, 0, -1, 0, np.inf],
                     [0.5, 0.5, 0.5, 0, 1, 0, 0, np.inf],
                     [0.5, 0.5, 0.5, 0, 0, 0, -1, 0.1],
                     [0.5, 0.5, 0.5, 5.0, 0, 0, -1, np.inf],
                     [5, 5, 5, 0, 1, 0, 0, np.inf],
                     [0.3, 0.2, 0.25, 0, 0.3, 0.9, -0.2, np.inf]], np.float32)
    for method in ("mtbvh", "stack"):
        for batch in (rays[:1], rays, np.concatenate([rays] * 5)[:33]):
            tri, t, _, _ = gpu_trace(ctx, sc, batch, method=method)
            ids, tt, _, _, nd = O.Mesh(sc.verts, sc.tris).closest_hit(batch, brute=True)
            parity_hits(tri, t, ids, tt, nd, max_excluded=1.0)
        assert gpu_trace(ctx, sc, rays[3:6], method=method)[0].tolist() == [-1, -1, -1]


def test_matches_host_walk(ctx):
    sc = I.traversal_sphere(n=24)
    rays = I.traversal_rays(64, 32, n_random=4096, seed=35)
    tri, t, _, s = gpu_trace(ctx, sc, rays)
    htri, ht, _, _ = s.host_walk(rays)
    ids, tt, _, _, nd = O.Mesh(sc.verts, sc.tris).closest_hit(rays)
    sel = nd.astype(bool)
    assert np.array_equal(tri[sel], htri[sel])


@pytest.fixture(scope="module")
def full_size():
    sc = I.traversal_sphere()  # 1,003,520 triangles
    rays = I.traversal_rays()  # 4,194,304 rays: 2,097,152 coherent + 2,097,152 random
    return sc, rays


@pytest.mark.parametrize("method", ["mtbvh", "stack"])
def test_full_size_traversal_sampled(ctx, full_size, method):
    """The benchmark's workload and launch: all 4M rays in one call; the oracle checks a
    stratified sample of 24,576 rays (both halves) with its FP64 BVH, and 4,096 of them (256 for
    the stack traversal) by brute force over all 1,003,520 triangles (4e9 FP64 tests)."""
    sc, rays = full_size
    tri, t, _, _ = gpu_trace(ctx, sc, rays, method=method)
    n = len(rays)
    rng = np.random.default_rng(77)
    sample = np.sort(np.concatenate([rng.choice(n // 2, 12288, replace=False),
                                     n // 2 + rng.choice(n // 2, 12288, replace=False)]))
    mesh = O.Mesh(sc.verts, sc.tris)
    ids, tt, _, _, nd = mesh.closest_hit(rays[sample])
    parity_hits(tri[sample], t[sample], ids, tt, nd)
    sub = sample[::6] if method == "mtbvh" else sample[::96]
    bids, btt, _, _, bnd = mesh.closest_hit(rays[sub], brute=True)
    parity_hits(tri[sub], t[sub], bids, btt, bnd)
    assert (tri >= 0).mean() > 0.2


def test_host_buffer_entry_matches_device_entry(ctx, full_size):
    """gsp_trace_closest_hit_host: chunked copies over three streams, pinned (direct) and pageable
    (staged) host buffers, a ragged last chunk; results equal the device-buffer call's."""
    sc, rays = full_size
    rays = rays[: len(rays) - 12345]
    s = gsp.Scene(ctx, sc)
    d = torch.from_numpy(rays).cuda()
    tri_d, t_d, uv_d = s.trace(d, with_uv=True)
    torch.cuda.synchronize()
    want = (tri_d.cpu().numpy(), t_d.cpu().numpy(), uv_d.cpu().numpy())
    n = len(rays)
    # pinned
    r_pin = torch.from_numpy(rays).pin_memory()
    tri_p = torch.empty(n, dtype=torch.int32).pin_memory()
    t_p = torch.empty(n, dtype=torch.float32).pin_memory()
    uv_p = torch.empty((n, 2), dtype=torch.float32).pin_memory()
    gsp.gsp_trace_closest_hit_host(s.h, r_pin, tri_p, t_p, uv_p)
    # pageable, without uv, then with uv
    tri_n = np.empty(n, np.int32)
    t_n = np.empty(n, np.float32)
    gsp.gsp_trace_closest_hit_host(s.h, np.ascontiguousarray(rays), tri_n, t_n)
    uv_n = np.empty((n, 2), np.float32)
    tri_u = np.empty(n, np.int32)
    t_u = np.empty(n, np.float32)
    gsp.gsp_trace_closest_hit_host(s.h, np.ascontiguousarray(rays), tri_u, t_u, uv_n)
    ctx.sync()
    assert np.array_equal(tri_u, want[0]) and np.array_equal(uv_n.view(np.int32), want[2].view(np.int32))
    assert np.array_equal(tri_p.numpy(), want[0]) and np.array_equal(t_p.numpy().view(np.int32), want[1].view(np.int32))
    assert np.array_equal(uv_p.numpy().view(np.int32), want[2].view(np.int32))
    assert np.array_equal(tri_n, want[0]) and np.array_equal(t_n.view(np.int32), want[1].view(np.int32))
    # a small call after a large one reuses the lanes
    gsp.gsp_trace_closest_hit_host(s.h, np.ascontiguousarray(rays[:1000]), tri_n[:1000], t_n[:1000])
    assert np.array_equal(tri_n[:1000], want[0][:1000])


def test_warp_walk_of_a_lone_last_ray(ctx):
    """When a warp has no rays left to take and one lane still walks, the whole warp walks that
    ray through windows of 32 nodes. Rays traced one per call go almost entirely that way; their
    ids and t are bit-identical to the same rays traced in one launch, and agree with the
    oracle. The rays are the longest walks of the sample (the ones a launch ends on) plus
    ordinary ones."""
    sc = I.traversal_sphere(n=64, seed=5)  # 81,920 triangles
    rays = I.traversal_rays(128, 64, n_random=8192, seed=36)
    s = gsp.Scene(ctx, sc)
    _, _, vis, _ = s.host_walk(rays)
    pick = np.concatenate([np.argsort(-vis, kind="stable")[:192], np.arange(0, len(rays), 257)])
    sub = np.ascontiguousarray(rays[pick])
    d = torch.from_numpy(sub).cuda()
    tri_all, t_all = s.trace(d)
    tri_one = torch.empty_like(tri_all)
    t_one = torch.empty_like(t_all)
    for i in range(len(sub)):
        a, b = s.trace(d[i:i + 1])
        tri_one[i:i + 1] = a
        t_one[i:i + 1] = b
    torch.cuda.synchronize()
    ctx.sync()
    tri_all, t_all = tri_all.cpu().numpy(), t_all.cpu().numpy()
    tri_one, t_one = tri_one.cpu().numpy(), t_one.cpu().numpy()
    assert vis[pick[:192]].min() > 4 * vis.mean()
    assert np.array_equal(tri_one, tri_all)
    assert np.array_equal(t_one.view(np.int32), t_all.view(np.int32))
    ids, tt, _, _, nd = O.Mesh(sc.verts, sc.tris).closest_hit(sub)
    parity_hits(tri_one, t_one, ids, tt, nd)


def test_launch_timing_records_the_traversal_kernel(ctx):
    """gsp_trace_time_launches: the next n calls record their traversal kernel's duration, the
    results do not change, a read restarts the recording, and n = 0 turns it off."""
    sc = I.traversal_sphere(n=24, seed=3)
    rays = torch.from_numpy(I.traversal_rays(64, 32, n_random=4000, seed=52)).cuda()
    s = gsp.Scene(ctx, sc)
    n = rays.shape[0]
    ref = [torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.float32, device="cuda")]
    gsp.gsp_trace_closest_hit(s.h, rays, *ref)
    gsp.gsp_trace_time_launches(s.h, 3)
    outs = []
    for _ in range(5):  # two more calls than pairs: they are not timed
        o = [torch.empty_like(ref[0]), torch.empty_like(ref[1])]
        gsp.gsp_trace_closest_hit(s.h, rays, *o)
        outs.append(o)
    ms = gsp.gsp_trace_launch_times(s.h, 8)
    assert len(ms) == 3 and np.all(ms > 0) and np.all(ms < 1000)
    for o in outs:
        assert torch.equal(o[0], ref[0]) and torch.equal(o[1].view(torch.int32), ref[1].view(torch.int32))
    assert len(gsp.gsp_trace_launch_times(s.h, 8)) == 0  # nothing recorded since the read
    gsp.gsp_trace_closest_hit(s.h, rays, *outs[0])
    assert len(gsp.gsp_trace_launch_times(s.h, 8)) == 1  # recording restarted from the first pair
    gsp.gsp_trace_time_launches(s.h, 0)
    gsp.gsp_trace_closest_hit(s.h, rays, *outs[0])
    assert len(gsp.gsp_trace_launch_times(s.h, 8)) == 0
    with pytest.raises(gsp.GspError):
        gsp.gsp_trace_time_launches(s.h, -1)
    ctx.sync()
