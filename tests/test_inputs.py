"""The seeded synthetic workloads have the structure their configurations state (sizes, materials,
camera, ray layout), and the same seed gives the same arrays. No method arithmetic: these are the
inputs both the CUDA path and the oracle read."""
import numpy as np

from paper_1505_06022_gb300 import inputs as I


def test_traversal_workload():
    """1,003,520-triangle displaced icosphere (20 x 224^2, closed) and 4,194,304 rays: 2048 x 1024
    pinhole rays from (0, 0, 3), then as many with origins in [-2, 2]^3, all of unit direction."""
    sc = I.traversal_sphere(224, 2)
    assert sc.ntris == 20 * 224 * 224 == 1_003_520
    assert sc.verts.dtype == np.float32 and sc.tris.dtype == np.int32
    # closed surface: every undirected edge is shared by exactly two triangles
    e = np.sort(np.concatenate([sc.tris[:, [0, 1]], sc.tris[:, [1, 2]], sc.tris[:, [2, 0]]]), axis=1)
    key = e[:, 0].astype(np.int64) * len(sc.verts) + e[:, 1]
    _, counts = np.unique(key, return_counts=True)
    assert np.all(counts == 2)
    r = np.linalg.norm(sc.verts.astype(np.float64), axis=1)  # radius 1 + 0.05 x a bounded sine sum
    assert 0.85 < r.min() and r.max() < 1.15
    rays = I.traversal_rays(2048, 1024, seed=2)
    n = 2048 * 1024
    assert rays.shape == (2 * n, 8) and rays.dtype == np.float32
    assert np.all(rays[:n, 0:3] == np.float32([0, 0, 3]))
    assert np.all(np.abs(rays[n:, 0:3]) <= 2)
    assert np.allclose(np.linalg.norm(rays[:, 4:7], axis=1), 1, atol=1e-6)
    assert np.all(rays[:, 3] == 0) and np.all(np.isinf(rays[:, 7]))
    assert np.array_equal(rays, I.traversal_rays(2048, 1024, seed=2))


def test_full_scene():
    """247,234 triangles: 256 x 256-quad displaced plane, three 38,720-triangle icospheres
    (glass of IOR 1.5, mirror, diffuse) and a two-triangle light; 512 x 512 camera."""
    sc = I.full_scene()
    assert sc.ntris == 2 * 256 * 256 + 3 * 20 * 44 * 44 + 2 == 247_234
    types = sorted(int(t) for t in sc.mats["type"])
    assert types.count(I.DIELECTRIC) == 1 and types.count(I.MIRROR) == 1
    glass = sc.mats[sc.mats["type"] == I.DIELECTRIC][0]
    assert glass["ior"] == np.float32(1.5)
    emitting = [m for m in sc.mats if max(m["emission"]) > 0]
    assert len(emitting) == 1
    assert int((sc.tri_mat == list(sc.mats).index(emitting[0])).sum()) == 2
    assert int(sc.camera["width"][0]) == 512 and int(sc.camera["height"][0]) == 512


def test_cornell_box():
    """36 triangles (5 wall quads, two boxes, a light quad), 64 x 64, Le = 10, albedos in [0.2, 0.8]."""
    sc = I.cornell_box(seed=1)
    assert sc.ntris == 36
    lights = [m for m in sc.mats if max(m["emission"]) > 0]
    assert len(lights) == 1 and np.all(lights[0]["emission"] == np.float32(10))
    diffuse = sc.mats[(sc.mats["type"] == I.DIFFUSE) & (sc.mats["emission"].max(axis=1) == 0)]
    assert len(diffuse) > 0 and np.all((diffuse["albedo"] >= 0.2) & (diffuse["albedo"] <= 0.8))
    assert np.all(sc.verts >= -1e-6) and np.all(sc.verts <= 1 + 1e-6)  # the unit box
    assert int(sc.camera["width"][0]) == 64 and int(sc.camera["height"][0]) == 64


def test_gradient_scene():
    """50,770 triangles, 16 diffuse materials and one light, 256 x 256."""
    sc = I.grad_scene()
    assert sc.ntris == 50_770
    emits = sc.mats["emission"].max(axis=1) > 0
    assert int(emits.sum()) == 1
    assert int(((sc.mats["type"] == I.DIFFUSE) & ~emits).sum()) == 16
    assert int(sc.camera["width"][0]) == 256 and int(sc.camera["height"][0]) == 256


def test_batch_scenes():
    """64 scenes, triangle counts spread log-uniformly over about [1e3, 2e5], sides in
    {64, 128, 256, 512}, reproducible from the seed."""
    a = I.batch_scenes(64, 5)
    assert len(a) == 64
    nt = np.array([s.ntris for s in a])
    assert nt.min() >= 1000 and nt.max() <= 210_000
    assert np.log10(nt).std() > 0.4  # spread over two decades, not clustered
    sides = {int(s.camera["width"][0]) for s in a}
    assert sides == {64, 128, 256, 512}
    assert all(int(s.camera["width"][0]) == int(s.camera["height"][0]) for s in a)
    b = I.batch_scenes(64, 5)
    assert all(np.array_equal(x.verts, y.verts) and np.array_equal(x.tris, y.tris) for x, y in zip(a, b))
