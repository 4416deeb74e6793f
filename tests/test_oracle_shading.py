"""Pins for the oracle's per-vertex shading data (Sec. 3.1's triangle with a normal and texture
coordinates per vertex): the blended normal of a sphere with radial vertex normals is the radial
direction at the hit; per-vertex face normals change nothing; bilinear lookup reproduces affine
texel ramps exactly, texel centres, wrap-around and constants; a constant texture is the same as
scaling the albedo; the white furnace with a textured albedo; the albedo gradient through a
texture against central differences."""
import copy

import numpy as np
import pytest

import oracle as O
from paper_1505_06022_gb300 import inputs as I


def _quad_scene(tex_st, mtype=I.DIFFUSE):
    """Unit quad z = 0 over [0, 1]^2 (diffuse, front +z), texture coordinates given per corner,
    plus a small light far above; camera looking down."""
    verts = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                      [0.4, 0.4, 5], [0.6, 0.4, 5], [0.6, 0.6, 5], [0.4, 0.6, 5]], np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3], [4, 6, 5], [4, 7, 6]], np.int32)
    mats = np.concatenate([I.material(mtype, (0.5, 0.5, 0.5)), I.material(I.EMITTER, (0, 0, 0), (10, 10, 10))])
    cam = I.camera((0.5, 0.5, 3), (0.5, 0.5, 0), (0, 1, 0), 30.0, 8, 8)
    st = np.concatenate([np.asarray(tex_st, np.float32), np.zeros((4, 2), np.float32)])
    return I.Scene(verts, tris, np.array([0, 0, 1, 1], np.int32), mats, cam, texcoords=st)


def _down_rays(xy):
    xy = np.asarray(xy, np.float64)
    r = np.zeros((len(xy), 8), np.float32)
    r[:, 0:2] = xy
    r[:, 2] = 1.0
    r[:, 6] = -1.0
    r[:, 7] = np.inf
    return r


def test_sphere_blended_normal_is_radial():
    n, c, rad = 8, np.array([0.3, -0.2, 0.1]), 0.7
    v, t = I.icosphere_unit(n)
    verts = (v * rad + c).astype(np.float32)
    normals = ((verts - c) / np.linalg.norm(verts - c, axis=1, keepdims=True)).astype(np.float32)
    mats = np.concatenate([I.material(I.MIRROR, (0.9, 0.9, 0.9)), I.material(I.EMITTER, (0, 0, 0), (1, 1, 1))])
    sc = I.Scene(verts, t.astype(np.int32), np.zeros(len(t), np.int32), mats,
                 I.camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 40.0, 4, 4), normals=normals)
    orc = O.Sppm(sc, O.default_params(sc, 10))
    rng = np.random.default_rng(1)
    o = c + rng.normal(size=(2000, 3)) * 0.2 + np.array([0, 0, 3.0])
    target = c + rng.normal(size=(2000, 3)) * 0.3
    d = target - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.zeros((2000, 8), np.float32)
    rays[:, 0:3], rays[:, 4:7], rays[:, 7] = o, d, np.inf
    sf = orc.surface(rays)
    hit = sf["id"] >= 0
    assert hit.mean() > 0.5 and np.all(sf["smooth"][hit])
    ids, tt, _, _, _ = orc.mesh.closest_hit(rays, classify=False)
    x = rays[hit, 0:3].astype(np.float64) + rays[hit, 4:7].astype(np.float64) * tt[hit, None]
    radial = (x - c) / np.linalg.norm(x - c, axis=1, keepdims=True)
    # blending the vertices' radial directions with the hit's barycentrics gives x - c exactly;
    # what remains is the FP32 rounding of the vertices and their normals
    assert np.abs(sf["ns"][hit] - radial).max() < 2e-6
    # the face normal differs from the radial direction by the tessellation angle (~ edge / r)
    tri = t[ids[hit]]
    fn = np.cross(verts[tri[:, 1]] - verts[tri[:, 0]], verts[tri[:, 2]] - verts[tri[:, 0]]).astype(np.float64)
    fn /= np.linalg.norm(fn, axis=1, keepdims=True)
    assert np.abs(fn - radial).max() > 1e-2


def test_face_normals_per_vertex_change_nothing():
    base = I.cornell_box(width=16, height=16)
    # unshared vertices: every triangle carries its own face normal at its three corners
    tri = base.tris
    verts = base.verts[tri.reshape(-1)]
    tris = np.arange(3 * len(tri), dtype=np.int32).reshape(-1, 3)
    v = verts.astype(np.float64).reshape(-1, 3, 3)
    fn = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    fn /= np.linalg.norm(fn, axis=1, keepdims=True)
    plain = I.Scene(verts, tris, base.tri_mat, base.mats, base.camera)
    smooth = I.Scene(verts, tris, base.tri_mat, base.mats, base.camera,
                     normals=np.repeat(fn, 3, axis=0).astype(np.float32))
    p = O.default_params(base, 4000)
    a, b = O.Sppm(plain, p), O.Sppm(smooth, p)
    a.run(2)
    b.run(2)
    ia, ib = a.image(), b.image()
    assert ia.max() > 0
    np.testing.assert_allclose(ib, ia, rtol=1e-9, atol=1e-12 * ia.max())


def test_bilinear_reproduces_affine_texels_exactly():
    w, h = 8, 5
    j, i = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    coef = np.array([[0.2, 0.03, 0.05], [0.4, 0.01, 0.07], [0.1, 0.06, 0.02]])  # per channel a, b, c
    tex = np.stack([coef[k, 0] + coef[k, 1] * i + coef[k, 2] * j for k in range(3)], -1).astype(np.float32)
    sc = _quad_scene([[0, 0], [1, 0], [1, 1], [0, 1]])
    orc = O.Sppm(sc, O.default_params(sc, 10))
    orc.set_texture(0, tex)
    rng = np.random.default_rng(2)
    # away from the wrap: texel-space x = s w - 0.5 in [0, w - 1]
    s = rng.uniform(0.5 / w, (w - 0.5) / w, 500)
    t = rng.uniform(0.5 / h, (h - 0.5) / h, 500)
    sf = orc.surface(_down_rays(np.stack([s, t], 1)))
    assert np.all(sf["id"] >= 0)
    x, y = s * w - 0.5, t * h - 0.5
    want = np.stack([coef[k, 0] + coef[k, 1] * x + coef[k, 2] * y for k in range(3)], -1)
    np.testing.assert_allclose(sf["tex"], want, rtol=0, atol=2e-7)  # float32 texels, exact blend
    # texel centres return the texel (up to the FP32 rounding of the ray origin: ~1e-7 texel)
    ci, cj = rng.integers(0, w, 50), rng.integers(0, h, 50)
    sf = orc.surface(_down_rays(np.stack([(ci + 0.5) / w, (cj + 0.5) / h], 1)))
    np.testing.assert_allclose(sf["tex"], tex[cj, ci].astype(np.float64), rtol=0, atol=5e-8)


def test_texture_wraps_and_constants():
    w, h = 6, 4
    tex = np.random.default_rng(3).uniform(0.2, 1.0, (h, w, 3)).astype(np.float32)
    pts = np.random.default_rng(4).uniform(0.01, 0.99, (300, 2))
    # the same quad with texture coordinates shifted by whole periods samples the same values
    a = O.Sppm(_quad_scene([[0, 0], [1, 0], [1, 1], [0, 1]]), O.default_params(_quad_scene([[0, 0]] * 4), 10))
    b = O.Sppm(_quad_scene([[3, -2], [4, -2], [4, -1], [3, -1]]), O.default_params(_quad_scene([[0, 0]] * 4), 10))
    a.set_texture(0, tex)
    b.set_texture(0, tex)
    ta, tb = a.surface(_down_rays(pts))["tex"], b.surface(_down_rays(pts))["tex"]
    np.testing.assert_allclose(tb, ta, rtol=0, atol=1e-12)
    # across the border the blend takes the opposite side's texels: at s = 0 (x = -0.5) the
    # value is the mean of the first and last columns
    edge = a.surface(_down_rays(np.stack([np.full(h, 1e-9), (np.arange(h) + 0.5) / h], 1)))["tex"]
    np.testing.assert_allclose(edge, 0.5 * (tex[:, 0] + tex[:, -1]), rtol=0, atol=1e-6)
    # a constant texture is that constant everywhere
    a.set_texture(0, np.full((h, w, 3), 0.625, np.float32))
    np.testing.assert_allclose(a.surface(_down_rays(pts))["tex"], 0.625, rtol=0, atol=1e-15)


def test_constant_texture_equals_scaled_albedo():
    sc = I.cornell_box(width=16, height=16)
    rng = np.random.default_rng(5)
    sc.texcoords = rng.uniform(-2, 2, (len(sc.verts), 2)).astype(np.float32)
    k = np.array([0.5, 0.25, 0.125], np.float32)  # powers of two: rho * k is exact in FP32
    diffuse = [m for m in range(len(sc.mats)) if sc.mats["type"][m] == I.DIFFUSE]
    sc.textures = {m: np.tile(k, (3, 4, 1)) for m in diffuse}
    scaled = copy.copy(sc)
    scaled.texcoords, scaled.textures = None, {}
    scaled.mats = sc.mats.copy()
    for m in diffuse:
        scaled.mats["albedo"][m] = sc.mats["albedo"][m] * k
    p = O.default_params(sc, 4000)
    a, b = O.Sppm(sc, p), O.Sppm(scaled, p)
    a.run(2)
    b.run(2)
    ia, ib = a.image(), b.image()
    assert ia.max() > 0
    np.testing.assert_allclose(ia, ib, rtol=1e-9, atol=1e-12 * ib.max())


@pytest.mark.parametrize("rho,c", [(0.5, 0.8), (0.8, 0.75)])
def test_white_furnace_with_texture(rho, c):
    sc = I.furnace_scene(n=32, albedo=rho, le=1.0, width=12, height=12)
    n = sc.verts.astype(np.float64)
    sc.texcoords = np.stack([0.5 + np.arctan2(n[:, 2], n[:, 0]) / (2 * np.pi), np.arccos(np.clip(n[:, 1], -1, 1)) / np.pi],
                            1).astype(np.float32)
    sc.textures = {0: np.full((8, 16, 3), c, np.float32)}
    r = O.Sppm(sc, O.default_params(sc, 120000, r0=0.15))
    r.run(4)
    img = r.image()
    want = 1.0 / (1.0 - rho * c)
    assert img.mean() == pytest.approx(want, rel=0.01)
    assert np.all(np.abs(img / want - 1) < 0.05)


def test_albedo_gradient_through_texture_matches_central_differences():
    sc = I.grad_scene(width=20, height=20, plane_quads=20, sphere_n=3)
    v = sc.verts.astype(np.float64)
    sc.texcoords = np.stack([v[:, 0] * 0.7, v[:, 2] * 0.7], 1).astype(np.float32)
    sc.textures = {m: I.pattern_texture(16, 10 + m, 4) for m in (0, 4, 13)}
    kw = dict(photons_per_pass=2500, seed=4, r0_frac=0.02)

    def render(mats):
        s2 = copy.copy(sc)
        s2.mats = mats
        r = O.Sppm(s2, O.default_params(s2, **kw))
        r.run(2)
        return r.image()

    target = sc.mats.copy()
    target["albedo"] = np.clip(target["albedo"] * 1.1, 0.05, 0.95)
    T = render(target)
    r = O.Sppm(sc, O.default_params(sc, **kw))
    r.enable_grad()
    r.run(2)
    ga, _ = r.grad(r.image() - T)
    loss = lambda img: 0.5 * np.sum((img - T) ** 2)
    scale = np.abs(ga).max()
    for m, c in [(0, 0), (4, 1), (13, 2), (7, 0)]:
        mp, mm = sc.mats.copy(), sc.mats.copy()
        mp["albedo"][m, c] += 1e-3
        mm["albedo"][m, c] -= 1e-3
        dh = float(mp["albedo"][m, c]) - float(mm["albedo"][m, c])
        fd = (loss(render(mp)) - loss(render(mm))) / dh
        assert abs(fd - ga[m, c]) <= 1e-5 * scale, (m, c, fd, ga[m, c])
