"""Seeded synthetic inputs: procedural scenes, cameras and ray batches.

This module only builds input data (geometry, materials, cameras, rays) with numpy. It holds
none of the renderer's arithmetic: no intersection, no sampling, no photon mapping. Both the
CUDA path and the CPU oracle are fed from it, so it imports neither of them.

Scene conventions shared by every consumer:

* ``verts``  float32 [nv, 3]    vertex positions
* ``tris``   int32   [nt, 3]    vertex indices; the geometric normal is (v1-v0) x (v2-v0)
* ``tri_mat`` int32  [nt]       material index per triangle
* ``mats``   MATERIAL_DTYPE [nm] material table (type, albedo RGB, emission RGB, ior)
* ``camera`` CAMERA_DTYPE  [1]  pinhole camera (eye, look-at point, up, vertical fov, w, h)
* optional shading data: ``normals`` float32 [nv, 3] per-vertex normals, ``texcoords`` float32
  [nv, 2] per-vertex texture coordinates, ``textures`` {material index: float32 [h, w, 3]}
  albedo factors of diffuse materials

Material types: DIFFUSE (two-sided Lambertian; may also emit from its front face), MIRROR,
DIELECTRIC, EMITTER (one-sided Lambertian emitter that absorbs everything it receives).

Rays are float32 [n, 8] rows ``ox, oy, oz, tmin, dx, dy, dz, tmax``.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

DIFFUSE, MIRROR, DIELECTRIC, EMITTER = 0, 1, 2, 3

MATERIAL_DTYPE = np.dtype(
    [("type", "<i4"), ("albedo", "<f4", (3,)), ("emission", "<f4", (3,)), ("ior", "<f4")],
    align=True,
)
CAMERA_DTYPE = np.dtype(
    [("eye", "<f4", (3,)), ("look", "<f4", (3,)), ("up", "<f4", (3,)), ("vfov_deg", "<f4"),
     ("width", "<i4"), ("height", "<i4")],
    align=True,
)
assert MATERIAL_DTYPE.itemsize == 32 and CAMERA_DTYPE.itemsize == 48


@dataclass
class Scene:
    verts: np.ndarray
    tris: np.ndarray
    tri_mat: np.ndarray
    mats: np.ndarray
    camera: np.ndarray
    name: str = "scene"
    info: dict = field(default_factory=dict)
    normals: np.ndarray | None = None
    texcoords: np.ndarray | None = None
    textures: dict = field(default_factory=dict)

    @property
    def ntris(self) -> int:
        return int(self.tris.shape[0])

    def extent(self) -> float:
        """Diagonal of the axis-aligned box around all vertices."""
        lo = self.verts.min(axis=0).astype(np.float64)
        hi = self.verts.max(axis=0).astype(np.float64)
        return float(np.linalg.norm(hi - lo))


def material(mtype, albedo=(0.0, 0.0, 0.0), emission=(0.0, 0.0, 0.0), ior=1.0):
    m = np.zeros(1, dtype=MATERIAL_DTYPE)
    m["type"] = mtype
    m["albedo"] = albedo
    m["emission"] = emission
    m["ior"] = ior
    return m


def camera(eye, look, up, vfov_deg, width, height):
    c = np.zeros(1, dtype=CAMERA_DTYPE)
    c["eye"], c["look"], c["up"] = eye, look, up
    c["vfov_deg"], c["width"], c["height"] = vfov_deg, width, height
    return c


# ----------------------------------------------------------------------------------------
# geometry builders
# ----------------------------------------------------------------------------------------

class _MeshBuilder:
    def __init__(self):
        self.v, self.t, self.m = [], [], []
        self.nv = 0

    def add(self, verts, tris, mat):
        verts = np.asarray(verts, dtype=np.float64)
        tris = np.asarray(tris, dtype=np.int64)
        self.v.append(verts)
        self.t.append(tris + self.nv)
        self.m.append(np.full(len(tris), mat, dtype=np.int32))
        self.nv += len(verts)

    def quad(self, p0, p1, p2, p3, mat):
        """Two triangles (p0,p1,p2), (p0,p2,p3); front face follows p0->p1->p2 winding."""
        self.add([p0, p1, p2, p3], [[0, 1, 2], [0, 2, 3]], mat)

    def box(self, lo, hi, mat):
        x0, y0, z0 = lo
        x1, y1, z1 = hi
        c = [[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
             [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]]
        faces = [[0, 3, 2, 1], [4, 5, 6, 7], [0, 4, 7, 3], [1, 2, 6, 5], [0, 1, 5, 4], [3, 7, 6, 2]]
        tris = []
        for a, b, cc, d in faces:  # outward-facing quads
            tris += [[a, b, cc], [a, cc, d]]
        self.add(c, tris, mat)

    def build(self):
        verts = np.concatenate(self.v).astype(np.float32)
        tris = np.concatenate(self.t).astype(np.int32)
        mats = np.concatenate(self.m).astype(np.int32)
        return verts, tris, mats


def _icosahedron():
    """12 vertices at the cyclic permutations of (0, +-1, +-phi); faces = triples at mutual
    edge length 2, wound so the normal points away from the origin."""
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v += [[0.0, s1, s2 * phi], [s1, s2 * phi, 0.0], [s2 * phi, 0.0, s1]]
    v = np.array(v)
    faces = []
    for a, b, c in itertools.combinations(range(12), 3):
        if all(abs(np.linalg.norm(v[x] - v[y]) - 2.0) < 1e-9 for x, y in ((a, b), (b, c), (a, c))):
            n = np.cross(v[b] - v[a], v[c] - v[a])
            faces.append([a, b, c] if np.dot(n, v[a] + v[b] + v[c]) > 0 else [a, c, b])
    assert len(faces) == 20
    return v, np.array(faces)


def icosphere_unit(n: int):
    """Unit icosphere with every icosahedron edge split into n segments: 20*n*n triangles,
    10*n*n+2 shared vertices (watertight), outward winding. Returns float64 (verts, tris)."""
    v, faces = _icosahedron()
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    keep = (ii + jj) <= n
    ii, jj = ii[keep], jj[keep]
    kk = n - ii - jj
    local = {(int(a), int(b)): idx for idx, (a, b) in enumerate(zip(ii, jj))}
    up, dn = [], []
    for a in range(n):
        for b in range(n - a):
            up.append([local[(a, b)], local[(a + 1, b)], local[(a, b + 1)]])
            if a + b <= n - 2:
                dn.append([local[(a + 1, b)], local[(a + 1, b + 1)], local[(a, b + 1)]])
    lt = np.array(up + dn)
    npf = len(ii)
    pts, tri = [], []
    for f, (A, B, C) in enumerate(faces):
        # two-term sums are commutative, so points on a shared edge come out bit-identical
        p = (ii[:, None] * v[A] + jj[:, None] * v[B]) + kk[:, None] * v[C]
        pts.append(p + 0.0)
        tri.append(lt + f * npf)
    pts = np.concatenate(pts) + 0.0
    tri = np.concatenate(tri)
    uniq, inv = np.unique(pts, axis=0, return_inverse=True)
    tri = inv.reshape(-1)[tri]
    uniq = uniq / np.linalg.norm(uniq, axis=1, keepdims=True)
    # orient outward
    a, b, c = uniq[tri[:, 0]], uniq[tri[:, 1]], uniq[tri[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    assert tri.shape[0] == 20 * n * n and uniq.shape[0] == 10 * n * n + 2
    return uniq, tri


def _sine_sum(rng, nterms=4):
    dirs = rng.normal(size=(nterms, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    freq = rng.uniform(2.0, 9.0, size=nterms)
    phase = rng.uniform(0.0, 2 * np.pi, size=nterms)
    return dirs, freq, phase


def displaced_icosphere(n: int, seed: int, amp: float = 0.05, center=(0, 0, 0), radius=1.0):
    """Icosphere radially displaced by r = 1 + amp * sum_k sin(f_k <p, a_k> + phi_k) / k."""
    rng = np.random.default_rng(seed)
    v, t = icosphere_unit(n)
    dirs, freq, phase = _sine_sum(rng)
    disp = np.zeros(len(v))
    for k in range(len(freq)):
        disp += np.sin(freq[k] * (v @ dirs[k]) + phase[k]) / (k + 1)
    r = radius * (1.0 + amp * disp)
    return v * r[:, None] + np.asarray(center, dtype=np.float64), t


def displaced_plane(g: int, half: float, seed: int, amp: float = 0.05, y0: float = 0.0):
    """g x g quads over x,z in [-half, half], height y0 + amp * sum_k sin(f_k <p, a_k> + phi_k)/k,
    normals facing +y."""
    rng = np.random.default_rng(seed)
    xs = np.linspace(-half, half, g + 1)
    X, Z = np.meshgrid(xs, xs, indexing="ij")
    dirs, freq, phase = _sine_sum(rng)
    H = np.zeros_like(X)
    for k in range(len(freq)):
        H += np.sin(freq[k] * (X * dirs[k, 0] + Z * dirs[k, 2]) / half * 2.0 + phase[k]) / (k + 1)
    v = np.stack([X, y0 + amp * H, Z], axis=-1).reshape(-1, 3)
    idx = np.arange((g + 1) * (g + 1)).reshape(g + 1, g + 1)
    a, b = idx[:-1, :-1].ravel(), idx[1:, :-1].ravel()
    c, d = idx[1:, 1:].ravel(), idx[:-1, 1:].ravel()
    # (a, d, c) winding: (d-a) x (c-a) = (+z) x (+x) = +y
    t = np.concatenate([np.stack([a, d, c], 1), np.stack([a, c, b], 1)])
    return v, t


# ----------------------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------------------

def cornell_box(seed: int = 1, width: int = 64, height: int = 64, le: float = 10.0) -> Scene:
    """Cornell-box-like scene: unit box [0,1]^3 open at z=1 (5 wall quads), two axis-aligned
    boxes, one 0.25 x 0.25 area-light quad at y=0.999 facing down: 36 triangles. Lambertian
    albedos U[0.2, 0.8] per RGB channel per material."""
    rng = np.random.default_rng(seed)
    mb = _MeshBuilder()
    mats = [material(DIFFUSE, rng.uniform(0.2, 0.8, 3)) for _ in range(7)]
    mats.append(material(EMITTER, (0, 0, 0), (le, le, le)))
    P = lambda x, y, z: [x, y, z]
    mb.quad(P(0, 0, 0), P(0, 0, 1), P(1, 0, 1), P(1, 0, 0), 0)   # floor
    mb.quad(P(0, 1, 0), P(1, 1, 0), P(1, 1, 1), P(0, 1, 1), 1)   # ceiling
    mb.quad(P(0, 0, 0), P(1, 0, 0), P(1, 1, 0), P(0, 1, 0), 2)   # back
    mb.quad(P(0, 0, 0), P(0, 1, 0), P(0, 1, 1), P(0, 0, 1), 3)   # left
    mb.quad(P(1, 0, 0), P(1, 0, 1), P(1, 1, 1), P(1, 1, 0), 4)   # right
    mb.box((0.15, 0.0, 0.15), (0.45, 0.6, 0.45), 5)
    mb.box((0.55, 0.0, 0.5), (0.85, 0.3, 0.8), 6)
    s = 0.125
    y = 0.999
    # winding chosen so that (p1-p0) x (p2-p0) points down (-y)
    mb.quad(P(0.5 - s, y, 0.5 - s), P(0.5 + s, y, 0.5 - s), P(0.5 + s, y, 0.5 + s),
            P(0.5 - s, y, 0.5 + s), 7)
    verts, tris, tri_mat = mb.build()
    cam = camera((0.5, 0.5, 2.2), (0.5, 0.5, 0.5), (0, 1, 0), 40.0, width, height)
    return Scene(verts, tris, tri_mat, np.concatenate(mats), cam, name="cornell64")


def traversal_sphere(n: int = 224, seed: int = 2) -> Scene:
    """Displaced subdivided icosphere: 20*n^2 triangles (n=224 -> 1,003,520)."""
    v, t = displaced_icosphere(n, seed)
    mats = material(DIFFUSE, (0.5, 0.5, 0.5))
    cam = camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 45.0, 2048, 1024)
    return Scene(v.astype(np.float32), t.astype(np.int32), np.zeros(len(t), np.int32), mats, cam,
                 name=f"icosphere{20 * n * n}")


def traversal_rays(width: int = 2048, height: int = 1024, n_random: int | None = None,
                   seed: int = 2, eye=(0.0, 0.0, 3.0), vfov_deg: float = 45.0) -> np.ndarray:
    """Half coherent pinhole rays (pixel centres, row-major, camera at `eye` looking at the
    origin), half incoherent rays with origins U[-2,2]^3 and directions uniform on S^2."""
    rng = np.random.default_rng(seed + 1000)
    n_random = width * height if n_random is None else n_random
    eye = np.asarray(eye, np.float64)
    fwd = -eye / np.linalg.norm(eye)
    right = np.cross(fwd, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    th = np.tan(np.radians(vfov_deg) / 2)
    py, px = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    sx = ((px + 0.5) / width * 2 - 1) * th * width / height
    sy = (1 - (py + 0.5) / height * 2) * th
    d = fwd + sx[..., None] * right + sy[..., None] * up
    d = (d / np.linalg.norm(d, axis=-1, keepdims=True)).reshape(-1, 3)
    coh = np.zeros((width * height, 8), np.float32)
    coh[:, 0:3] = eye
    coh[:, 4:7] = d
    coh[:, 7] = np.inf
    rnd = np.zeros((n_random, 8), np.float32)
    rnd[:, 0:3] = rng.uniform(-2, 2, (n_random, 3))
    dd = rng.normal(size=(n_random, 3))
    rnd[:, 4:7] = dd / np.linalg.norm(dd, axis=1, keepdims=True)
    rnd[:, 7] = np.inf
    return np.concatenate([coh, rnd])


def random_soup(nt: int, seed: int, scale: float = 1.0, size: float = 0.3) -> Scene:
    """Random triangle soup in [-scale, scale]^3 for brute-force checks."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-scale, scale, (nt, 1, 3))
    v = (c + rng.normal(scale=size, size=(nt, 3, 3))).reshape(-1, 3).astype(np.float32)
    t = np.arange(3 * nt, dtype=np.int32).reshape(nt, 3)
    mats = material(DIFFUSE, (0.5, 0.5, 0.5))
    cam = camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 45.0, 16, 16)
    return Scene(v, t, np.zeros(nt, np.int32), mats, cam, name=f"soup{nt}")


def random_rays(n: int, seed: int, scale: float = 1.5, tmin: float = 0.0,
                tmax: float = np.inf) -> np.ndarray:
    rng = np.random.default_rng(seed)
    r = np.zeros((n, 8), np.float32)
    r[:, 0:3] = rng.uniform(-scale, scale, (n, 3))
    d = rng.normal(size=(n, 3))
    r[:, 4:7] = d / np.linalg.norm(d, axis=1, keepdims=True)
    r[:, 3] = tmin
    r[:, 7] = tmax
    return r


def full_scene(seed: int = 3, width: int = 512, height: int = 512, plane_quads: int = 256,
               sphere_n: int = 44) -> Scene:
    """Displaced plane (plane_quads^2 quads) + 3 icospheres (dielectric IOR 1.5, mirror,
    diffuse; 20*sphere_n^2 triangles each) + one area light quad (2 triangles).
    Defaults: 131,072 + 3*38,720 + 2 = 247,234 triangles."""
    rng = np.random.default_rng(seed)
    mb = _MeshBuilder()
    mats = [material(DIFFUSE, rng.uniform(0.2, 0.8, 3)),
            material(DIELECTRIC, (1, 1, 1), ior=1.5),
            material(MIRROR, (0.9, 0.9, 0.9)),
            material(DIFFUSE, rng.uniform(0.2, 0.8, 3)),
            material(EMITTER, (0, 0, 0), (40.0, 38.0, 34.0))]
    v, t = displaced_plane(plane_quads, 2.5, seed, amp=0.04)
    mb.add(v, t, 0)
    for k, (cx, cz) in enumerate([(-1.1, 0.0), (0.0, -0.8), (1.1, 0.3)]):
        v, t = displaced_icosphere(sphere_n, seed + 10 + k, amp=0.0, center=(cx, 0.62, cz),
                                   radius=0.5)
        mb.add(v, t, 1 + k)
    s, y = 0.5, 3.0
    mb.quad([-s, y, -s], [s, y, -s], [s, y, s], [-s, y, s], 4)
    verts, tris, tri_mat = mb.build()
    cam = camera((0, 2.2, 5.0), (0, 0.4, 0), (0, 1, 0), 40.0, width, height)
    return Scene(verts, tris, tri_mat, np.concatenate(mats), cam, name=f"full{len(tris)}")


def vertex_normals(verts, tris):
    """Area-weighted average of the faces' normals around each vertex (float64, unit)."""
    v = np.asarray(verts, np.float64)
    t = np.asarray(tris, np.int64)
    fn = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])  # length = 2 * area
    acc = np.zeros_like(v)
    for k in range(3):
        np.add.at(acc, t[:, k], fn)
    return acc / np.linalg.norm(acc, axis=1, keepdims=True)


def pattern_texture(size: int, seed: int, squares: int = 8) -> np.ndarray:
    """Seeded RGB albedo factors in [0.35, 1]: a checkerboard of two random colours with a smooth
    sinusoidal shading on top. float32 [size, size, 3]."""
    rng = np.random.default_rng(seed)
    c0, c1 = rng.uniform(0.5, 1.0, 3), rng.uniform(0.35, 0.7, 3)
    j, i = np.meshgrid(np.arange(size), np.arange(size), indexing="ij")
    check = ((i * squares // size) + (j * squares // size)) % 2
    base = np.where(check[..., None] == 0, c0, c1)
    f = rng.uniform(1.0, 3.0, 2)
    shade = 0.85 + 0.15 * np.sin(2 * np.pi * (f[0] * i / size + f[1] * j / size))[..., None]
    return np.clip(base * shade, 0.35, 1.0).astype(np.float32)


def shaded_scene(seed: int = 6, width: int = 512, height: int = 512, plane_quads: int = 256,
                 sphere_n: int = 44, tex_size: int = 256) -> Scene:
    """The full scene's layout with per-vertex shading data: smooth normals on every sphere
    (radial) and on the displaced plane (area-weighted), texture coordinates (the plane tiled
    4 x 4, the spheres in longitude/latitude) and albedo textures on the plane and the diffuse
    sphere. Defaults: 247,234 triangles, two 256^2 textures."""
    rng = np.random.default_rng(seed)
    mats = [material(DIFFUSE, rng.uniform(0.5, 0.9, 3)),
            material(DIELECTRIC, (1, 1, 1), ior=1.5),
            material(MIRROR, (0.9, 0.9, 0.9)),
            material(DIFFUSE, rng.uniform(0.5, 0.9, 3)),
            material(EMITTER, (0, 0, 0), (40.0, 38.0, 34.0))]
    mb = _MeshBuilder()
    nrm, st = [], []
    half = 2.5
    v, t = displaced_plane(plane_quads, half, seed, amp=0.04)
    mb.add(v, t, 0)
    nrm.append(vertex_normals(v, t))
    st.append(np.stack([(v[:, 0] + half) / (2 * half) * 4.0, (v[:, 2] + half) / (2 * half) * 4.0], 1))
    for k, (cx, cz) in enumerate([(-1.1, 0.0), (0.0, -0.8), (1.1, 0.3)]):
        c = np.array([cx, 0.62, cz])
        v, t = displaced_icosphere(sphere_n, seed + 10 + k, amp=0.0, center=c, radius=0.5)
        mb.add(v, t, 1 + k)
        n = (v - c) / np.linalg.norm(v - c, axis=1, keepdims=True)
        nrm.append(n)
        st.append(np.stack([0.5 + np.arctan2(n[:, 2], n[:, 0]) / (2 * np.pi),
                            np.arccos(np.clip(n[:, 1], -1.0, 1.0)) / np.pi], 1))
    s, y = 0.5, 3.0
    mb.quad([-s, y, -s], [s, y, -s], [s, y, s], [-s, y, s], 4)
    nrm.append(np.tile([0.0, -1.0, 0.0], (4, 1)))
    st.append(np.zeros((4, 2)))
    verts, tris, tri_mat = mb.build()
    cam = camera((0, 2.2, 5.0), (0, 0.4, 0), (0, 1, 0), 40.0, width, height)
    return Scene(verts, tris, tri_mat, np.concatenate(mats), cam, name=f"shaded{len(tris)}",
                 normals=np.concatenate(nrm).astype(np.float32), texcoords=np.concatenate(st).astype(np.float32),
                 textures={0: pattern_texture(tex_size, seed + 1), 3: pattern_texture(tex_size, seed + 2, 6)})


def grad_scene(seed: int = 4, width: int = 256, height: int = 256, plane_quads: int = 128,
               sphere_n: int = 15) -> Scene:
    """Displaced plane split into 4x3 material regions + 4 diffuse icospheres: 16 diffuse
    materials (index 0..15) plus one emitter (index 16). Defaults: 50,770 triangles."""
    rng = np.random.default_rng(seed)
    mb = _MeshBuilder()
    mats = [material(DIFFUSE, rng.uniform(0.2, 0.8, 3)) for _ in range(16)]
    mats.append(material(EMITTER, (0, 0, 0), (30.0, 30.0, 30.0)))
    v, t = displaced_plane(plane_quads, 2.0, seed, amp=0.04)
    cen = v[t].mean(axis=1)
    rx = np.clip(((cen[:, 0] + 2.0) / 4.0 * 4).astype(int), 0, 3)
    rz = np.clip(((cen[:, 2] + 2.0) / 4.0 * 3).astype(int), 0, 2)
    region = rx * 3 + rz
    # the plane keeps its shared vertices: add it once, then set materials per triangle
    mb.add(v, t, 0)
    mb.m[-1] = region.astype(np.int32)
    for k, (cx, cz) in enumerate([(-1.0, -0.6), (0.9, -0.7), (-0.5, 0.8), (0.8, 0.7)]):
        v2, t2 = displaced_icosphere(sphere_n, seed + 20 + k, amp=0.03, center=(cx, 0.45, cz),
                                     radius=0.4)
        mb.add(v2, t2, 12 + k)
    s, y = 0.6, 2.5
    mb.quad([-s, y, -s], [s, y, -s], [s, y, s], [-s, y, s], 16)
    verts, tris, tri_mat = mb.build()
    cam = camera((0, 2.0, 4.2), (0, 0.3, 0), (0, 1, 0), 42.0, width, height)
    return Scene(verts, tris, tri_mat, np.concatenate(mats), cam, name=f"grad{len(tris)}")


def furnace_scene(n: int = 64, albedo: float = 0.5, le: float = 1.0, width: int = 16,
                  height: int = 16) -> Scene:
    """Closed unit icosphere (20*n^2 triangles) wound inward; every triangle is a diffuse
    emitter of radiance `le` with albedo `albedo`. Camera at the centre."""
    v, t = icosphere_unit(n)
    t = t[:, [0, 2, 1]]  # inward normals: emission faces the centre
    mats = material(DIFFUSE, (albedo,) * 3, (le,) * 3)
    cam = camera((0, 0, 0), (0, 0, -1), (0, 1, 0), 60.0, width, height)
    return Scene(v.astype(np.float32), t.astype(np.int32), np.zeros(len(t), np.int32), mats, cam,
                 name=f"furnace{albedo}")


def batch_scenes(count: int = 64, seed: int = 5):
    """`count` independent scenes: triangle counts log-uniform in [1e3, 2e5] (displaced plane
    plus spheres), image side in {64, 128, 256, 512}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        target = float(np.exp(rng.uniform(np.log(1e3), np.log(2e5))))
        side = int(rng.choice([64, 128, 256, 512]))
        g = max(8, int(np.ceil(np.sqrt(target * 0.6 / 2))))
        sn = max(2, int(np.ceil(np.sqrt(target * 0.4 / 60))))
        sc = full_scene(seed=1000 + i, width=side, height=side, plane_quads=g, sphere_n=sn)
        sc.name = f"batch{i}"
        out.append(sc)
    return out


# ----------------------------------------------------------------------------------------
# small specular scenes with closed-form answers (mirror and glass branches)
# ----------------------------------------------------------------------------------------

def _rotated_box(mb, center, half, angles, mat):
    """A box of half extents `half`, rotated by `angles` (radians, about x then y) around its
    centre, outward faces."""
    ax, ay = angles
    rx = np.array([[1, 0, 0], [0, np.cos(ax), -np.sin(ax)], [0, np.sin(ax), np.cos(ax)]])
    ry = np.array([[np.cos(ay), 0, np.sin(ay)], [0, 1, 0], [-np.sin(ay), 0, np.cos(ay)]])
    c = np.array([[x, y, z] for z in (-1, 1) for y in (-1, 1) for x in (-1, 1)], np.float64)
    c = c[[0, 1, 3, 2, 4, 5, 7, 6]]  # the corner order of _MeshBuilder.box
    v = (c * np.asarray(half)) @ (ry @ rx).T + np.asarray(center, np.float64)
    faces = [[0, 3, 2, 1], [4, 5, 6, 7], [0, 4, 7, 3], [1, 2, 6, 5], [0, 1, 5, 4], [3, 7, 6, 2]]
    tris = []
    for a, b, cc, d in faces:
        tris += [[a, b, cc], [a, cc, d]]
    mb.add(v, tris, mat)


def specular_furnace_scene(albedo: float = 0.5, le: float = 1.0, n: int = 32, sphere_n: int = 12,
                           width: int = 12, height: int = 12, mirror_albedo=(1.0, 1.0, 1.0),
                           glass_albedo=(0.3, 0.3, 0.3)) -> Scene:
    """The white furnace (closed unit icosphere wound inward, every wall triangle a diffuse
    emitter of radiance `le` with albedo `albedo`) with a mirror sphere of radius 0.22 and a
    rotated glass box (IOR 1.5, half extents 0.2 x 0.16 x 0.12) in front of a camera at the centre
    looking down -z. A ray inside a box always leaves it again (internal reflections at one pair of
    faces keep its angle to the others), unlike a faceted sphere, which can trap light by total
    internal reflection. The glass albedo is not used by the method (a dielectric only reflects or
    refracts); it is set to 0.3 on purpose."""
    mb = _MeshBuilder()
    v, t = icosphere_unit(n)
    mb.add(v, t[:, [0, 2, 1]], 0)  # walls, normals toward the centre
    v, t = icosphere_unit(sphere_n)
    mb.add(v * 0.22 + np.array([-0.3, -0.05, -0.45]), t, 1)
    _rotated_box(mb, (0.3, 0.05, -0.45), (0.2, 0.16, 0.12), (0.45, 0.6), 2)
    verts, tris, tri_mat = mb.build()
    mats = np.concatenate([material(DIFFUSE, (albedo,) * 3, (le,) * 3), material(MIRROR, mirror_albedo),
                           material(DIELECTRIC, glass_albedo, ior=1.5)])
    cam = camera((0, 0, 0), (0, 0, -1), (0, 1, 0), 60.0, width, height)
    return Scene(verts, tris, tri_mat, mats, cam, name=f"specular_furnace{albedo}")


def mirror_view_scene(mirror_albedo=(0.9, 0.6, 0.3), le=(4.0, 5.0, 6.0), width: int = 8, height: int = 8) -> Scene:
    """A camera at height 0.5 looking straight down at a 20 x 20 mirror floor (y = 0) under a
    20 x 20 emitter ceiling (y = 1) facing down: every eye ray reflects once into the emitter."""
    mb = _MeshBuilder()
    S = 10.0
    mb.quad([-S, 0, -S], [-S, 0, S], [S, 0, S], [S, 0, -S], 0)  # normal +y
    mb.quad([-S, 1, -S], [S, 1, -S], [S, 1, S], [-S, 1, S], 1)  # normal -y
    verts, tris, tri_mat = mb.build()
    mats = np.concatenate([material(MIRROR, mirror_albedo), material(EMITTER, emission=le)])
    cam = camera((0.3, 0.5, 0.2), (0.3, 0.0, 0.2001), (0, 0, 1), 30.0, width, height)
    return Scene(verts, tris, tri_mat, mats, cam, name="mirror_view")


def mirror_corridor_scene(length: int, mirror_albedo=(0.95, 0.9, 0.85), le=(3.0, 3.0, 3.0)) -> Scene:
    """Two parallel mirrors (y = 0 facing up, y = 1 facing down) from x = -1 to x = `length`, an
    emitter wall at x = `length` facing -x, and a one-pixel camera at (0, 0.5, 0) with a tiny field
    of view looking up at 45 degrees along +x: its ray meets the mirrors at x = 0.5, 1.5, ...,
    `length` - 0.5 (`length` reflections) and then the emitter at height 0.5."""
    mb = _MeshBuilder()
    X = float(length)
    z0, z1 = -0.7, 1.0  # quad diagonals cross z = 0 away from the reflection points
    mb.quad([-1, 0, z0], [-1, 0, z1], [X, 0, z1], [X, 0, z0], 0)  # normal +y
    mb.quad([-1, 1, z0], [X, 1, z0], [X, 1, z1], [-1, 1, z1], 0)  # normal -y
    mb.quad([X, -0.5, z0], [X, -0.5, z1], [X, 1.5, z1], [X, 1.5, z0], 1)  # normal -x
    verts, tris, tri_mat = mb.build()
    mats = np.concatenate([material(MIRROR, mirror_albedo), material(EMITTER, emission=le)])
    cam = camera((0, 0.5, 0), (1, 1.5, 0), (0, 0, 1), 0.01, 1, 1)
    return Scene(verts, tris, tri_mat, mats, cam, name=f"mirror_corridor{length}")


def photon_mirror_scene(mirror_albedo=(0.9, 0.6, 0.3), le: float = 5.0, light: float = 0.2,
                        mirror: bool = True, glass_albedo=(0.3, 0.3, 0.3)) -> Scene:
    """A `light` x `light` emitter at y = 1 facing down over a 40 x 40 floor at y = 0, under a
    diffuse ceiling at y = 2 facing down; a camera looks up at the ceiling. mirror=True: the floor
    is a mirror of albedo `mirror_albedo`, so a photon reflects once before it lands on the
    ceiling. mirror=False: the floor is diffuse and a 40 x 40 glass slab (IOR 1.5, y in
    [0.3, 0.5]) lies between the light and the floor."""
    mb = _MeshBuilder()
    S, h = 20.0, light / 2
    mb.quad([-S, 0, -S], [-S, 0, S], [S, 0, S], [S, 0, -S], 0)  # floor, normal +y
    mb.quad([-S, 2, -S], [S, 2, -S], [S, 2, S], [-S, 2, S], 1)  # ceiling, normal -y
    mb.quad([-h, 1, -h], [h, 1, -h], [h, 1, h], [-h, 1, h], 2)  # light, normal -y
    if not mirror:
        mb.box((-S, 0.3, -S), (S, 0.5, S), 3)
    verts, tris, tri_mat = mb.build()
    floor = material(MIRROR, mirror_albedo) if mirror else material(DIFFUSE, (0.5, 0.5, 0.5))
    mats = np.concatenate([floor, material(DIFFUSE, (0.6, 0.6, 0.6)), material(EMITTER, emission=(le,) * 3),
                           material(DIELECTRIC, glass_albedo, ior=1.5)])
    cam = camera((0.0, 1.5, 0.0), (0.0, 2.0, 0.0001), (0, 0, 1), 60.0, 4, 4)
    return Scene(verts, tris, tri_mat, mats, cam, name="photon_mirror" if mirror else "photon_glass")


def rotated(scene: Scene, ax: float, ay: float, center=(0.5, 0.5, 0.5)) -> Scene:
    """The scene turned about `center` by `ax` radians about x, then `ay` about y (geometry,
    vertex normals and camera alike), so that its planar walls are no longer axis planes."""
    rx = np.array([[1, 0, 0], [0, np.cos(ax), -np.sin(ax)], [0, np.sin(ax), np.cos(ax)]])
    ry = np.array([[np.cos(ay), 0, np.sin(ay)], [0, 1, 0], [-np.sin(ay), 0, np.cos(ay)]])
    M = ry @ rx
    c = np.asarray(center, np.float64)
    turn = lambda p: (np.asarray(p, np.float64) - c) @ M.T + c
    cam = scene.camera.copy()
    cam["eye"] = turn(cam["eye"][0])
    cam["look"] = turn(cam["look"][0])
    cam["up"] = np.asarray(cam["up"][0], np.float64) @ M.T
    nrm = None if scene.normals is None else (scene.normals.astype(np.float64) @ M.T).astype(np.float32)
    return Scene(turn(scene.verts).astype(np.float32), scene.tris.copy(), scene.tri_mat.copy(), scene.mats.copy(),
                 cam, name=scene.name + "_rotated", normals=nrm, texcoords=scene.texcoords,
                 textures=dict(scene.textures))
