"""CPU oracle for the MTBVH ray caster and the SPPM renderer (ctypes front end).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it; the product package never imports it and shares no code with it.

The arithmetic lives in ``gsp_oracle.cpp`` (FP64 geometry and density estimation, FP32 PRNG
output). This module only builds that file with gcc and marshals numpy arrays.

Non-degenerate rays (where the FP32 GPU triangle id must equal the FP64 oracle id bit for bit),
decided in FP64: the winner's barycentric margin min(u, v, 1-u-v) exceeds 1e-6; its
|det| / (|e1| |e2| |d|) exceeds 1e-7; its t is more than 1e-5 (relative) away from tmin and
tmax; and every other triangle whose barycentric margin is at least -1e-6 and whose t lies in
the ray's range is more than 1e-5 (relative) away in t and not in front of the winner. A ray that
misses is non-degenerate when no triangle comes within that margin inside the range.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsp_oracle.cpp")
# GSP_ORACLE_SANITIZE=1: a separate build with AddressSanitizer and UndefinedBehaviorSanitizer
# (the host process must preload their runtimes; tests/test_sanitizers.py does that).
_SANITIZE = os.environ.get("GSP_ORACLE_SANITIZE") == "1"
_OUT = os.path.join(_HERE, "_build", "libgsp_oracle_asan.so" if _SANITIZE else "libgsp_oracle.so")
_lock = threading.Lock()
_lib = None

EYE, PHOTON = 0, 1


class Material(C.Structure):
    _fields_ = [("type", C.c_int32), ("albedo", C.c_float * 3), ("emission", C.c_float * 3),
                ("ior", C.c_float)]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class SppmParams(C.Structure):
    _fields_ = [("photons_per_pass", C.c_int64), ("table_size", C.c_int64), ("seed", C.c_uint64),
                ("alpha", C.c_float), ("r0", C.c_float), ("rr_continue", C.c_float),
                ("cell_h", C.c_float), ("eps", C.c_float), ("photon_mode", C.c_int32),
                ("hash_mode", C.c_int32), ("max_eye_depth", C.c_int32),
                ("max_photon_depth", C.c_int32), ("scene_id", C.c_uint32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FP contraction: the FP32 PRNG output must
    be IEEE round-to-nearest on every host)."""
    with _lock:
        if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
            return _OUT
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-pthread", _SRC, "-o", tmp]
        if _SANITIZE:
            cmd[3:3] = ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
        return _OUT


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P, I64, I32, U32, U64 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint32, C.c_uint64
        L.orc_mlcg_step.restype = I64
        L.orc_mlcg_step.argtypes = [I32, I64]
        L.orc_rng_seed.argtypes = [U64, U32, U32, U32, U64, P]
        L.orc_rng_next.restype = C.c_float
        L.orc_rng_next.argtypes = [P]
        L.orc_rng_draws.argtypes = [U64, U32, U32, U32, P, I64, I32, P]
        L.orc_splitmix64.restype = U64
        L.orc_splitmix64.argtypes = [U64]
        L.orc_mesh_create.restype = P
        L.orc_mesh_create.argtypes = [P, I64, P, I64, P]
        L.orc_mesh_destroy.argtypes = [P]
        L.orc_closest_hit.argtypes = [P, P, I64, I32, P, P, P, P, P, C.c_int]
        L.orc_mt.restype = I32
        L.orc_mt.argtypes = [P, P, P, P, P]
        L.orc_sppm_create.restype = P
        L.orc_sppm_create.argtypes = [P, P, I32, P, P]
        L.orc_sppm_destroy.argtypes = [P]
        L.orc_sppm_run.restype = I32
        L.orc_sppm_run.argtypes = [P, I32, I32]
        L.orc_sppm_state.argtypes = [P, P, P, P, P, P, P]
        L.orc_sppm_last_photons.restype = I64
        L.orc_sppm_last_photons.argtypes = [P, P, P, P, P]
        L.orc_sppm_last_gather.argtypes = [P, P, P, P, P, P, P, P]
        L.orc_cosine_dir.argtypes = [P, C.c_float, C.c_float, P]
        L.orc_dielectric.argtypes = [P, P, C.c_double, C.c_float, P]
        L.orc_mlcg_step_many.argtypes = [I32, P, I64, P]
        L.orc_sppm_update.argtypes = [I64, C.c_double, P, P, P, P, P]
        L.orc_hash_grid.argtypes = [P, I64, C.c_double, I64, P, P, P, P]
        L.orc_sppm_enable_grad.restype = I32
        L.orc_sppm_enable_grad.argtypes = [P]
        L.orc_sppm_grad.restype = I32
        L.orc_sppm_grad.argtypes = [P, P, P, P]
        L.orc_mesh_set_attributes.restype = I32
        L.orc_mesh_set_attributes.argtypes = [P, P, P, P, I64]
        L.orc_sppm_set_texture.restype = I32
        L.orc_sppm_set_texture.argtypes = [P, I32, P, I32, I32]
        L.orc_sppm_surface.argtypes = [P, P, I64, P]
        L.orc_sah_split.restype = I32
        L.orc_sah_split.argtypes = [P, P, P, I64, I32, P, P, P, P, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def nthreads_default() -> int:
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------------------- PRNG (Fig. 5)
def mlcg_step(i: int, s: int) -> int:
    return int(lib().orc_mlcg_step(i, s))


def mlcg_step_many(i: int, s) -> np.ndarray:
    s = np.ascontiguousarray(s, np.int64)
    out = np.zeros_like(s)
    lib().orc_mlcg_step_many(i, _p(s), len(s), _p(out))
    return out


def cosine_dir(n, ua, ub) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_cosine_dir(_p(np.ascontiguousarray(n, np.float64)), ua, ub, _p(out))
    return out


def dielectric(d, n, ior, u) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_dielectric(_p(np.ascontiguousarray(d, np.float64)),
                         _p(np.ascontiguousarray(n, np.float64)), ior, u, _p(out))
    return out


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def rng_seed(seed, scene, domain, pass_, sid) -> np.ndarray:
    st = np.zeros(4, np.int64)
    lib().orc_rng_seed(seed, scene, domain, pass_, sid, _p(st))
    return st


def rng_next(state: np.ndarray) -> float:
    return float(lib().orc_rng_next(_p(state)))


def rng_draws(seed, scene, domain, pass_, ids, ndraw) -> np.ndarray:
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    out = np.zeros((len(ids), ndraw), np.float32)
    lib().orc_rng_draws(seed, scene, domain, pass_, _p(ids), len(ids), ndraw, _p(out))
    return out


# ---------------------------------------------------------------------------- closest hit
class Mesh:
    def __init__(self, verts, tris, tri_mat=None):
        self.verts = np.ascontiguousarray(verts, np.float32)
        self.tris = np.ascontiguousarray(tris, np.int32)
        self.tri_mat = None if tri_mat is None else np.ascontiguousarray(tri_mat, np.int32)
        self.h = lib().orc_mesh_create(_p(self.verts), len(self.verts), _p(self.tris),
                                       len(self.tris), _p(self.tri_mat))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_mesh_destroy(self.h)
            self.h = None

    def set_attributes(self, normals=None, texcoords=None):
        """Per-vertex normals [nv, 3] and texture coordinates [nv, 2] (either may be None)."""
        self.normals = None if normals is None else np.ascontiguousarray(normals, np.float32)
        self.texcoords = None if texcoords is None else np.ascontiguousarray(texcoords, np.float32)
        if lib().orc_mesh_set_attributes(self.h, _p(self.normals), _p(self.texcoords), _p(self.tris),
                                         len(self.tris)) != 0:
            raise ValueError("oracle: a vertex normal is zero")

    def closest_hit(self, rays, brute=False, classify=True, nthreads=None):
        """Returns (id int32, t f64, u f64, v f64, nondeg int32 or None). id -1 = miss."""
        rays = np.ascontiguousarray(rays, np.float32)
        n = len(rays)
        ids = np.zeros(n, np.int32)
        t, u, v = np.zeros(n), np.zeros(n), np.zeros(n)
        nd = np.zeros(n, np.int32) if classify else None
        lib().orc_closest_hit(self.h, _p(rays), n, 0 if brute else 1, _p(ids), _p(t), _p(u), _p(v),
                              _p(nd), nthreads or nthreads_default())
        return ids, t, u, v, nd


def sah_split(verts, tris, subset, bins=16):
    """Binned SAH split of the triangles `subset` (Sec. 3.1): None if no boundary leaves both
    sides non-empty, else dict(axis, boundary, cost, left = the subset's triangles in bins below
    the boundary); `near` = smallest centroid distance from an interior bin boundary (bin widths)."""
    v = np.ascontiguousarray(verts, np.float32)
    t = np.ascontiguousarray(tris, np.int32)
    sub = np.ascontiguousarray(subset, np.int32)
    ax, b, cost, near = C.c_int32(), C.c_int32(), C.c_double(), C.c_double()
    left = np.zeros(len(sub), np.int32)
    ok = lib().orc_sah_split(_p(v), _p(t), _p(sub), len(sub), bins, C.byref(ax), C.byref(b), C.byref(cost),
                             C.byref(near), _p(left))
    if not ok:
        return dict(split=False, near=near.value)
    return dict(split=True, axis=ax.value, boundary=b.value, cost=cost.value, near=near.value,
                left=sub[left.astype(bool)])


def mt(v0, v1, v2, ray):
    """Moller-Trumbore on one triangle in FP64: (inside, t, u, v)."""
    tuv = np.zeros(3)
    f = lambda a: np.ascontiguousarray(a, np.float32)
    hit = lib().orc_mt(_p(f(v0)), _p(f(v1)), _p(f(v2)), _p(f(ray)), _p(tuv))
    return bool(hit), tuv[0], tuv[1], tuv[2]


# ---------------------------------------------------------------------------- SPPM
def default_params(scene, photons_per_pass, seed=1, alpha=0.7, r0=None, r0_frac=0.05,
                   photon_mode=0, hash_mode=0, cell_h=None, table_size=None,
                   rr_continue=0.8, eps_frac=1e-4, max_eye_depth=16, max_photon_depth=32,
                   scene_id=0):
    """Parameter values exactly as the CUDA path receives them (float32-rounded)."""
    ext = scene.extent()
    r0 = float(np.float32(r0 if r0 is not None else r0_frac * ext))
    cell_h = float(np.float32(cell_h if cell_h is not None else 2.0 * r0))
    if table_size is None:
        table_size = 1
        while table_size < 2 * photons_per_pass:
            table_size *= 2
    return dict(photons_per_pass=int(photons_per_pass), table_size=int(table_size), seed=int(seed),
                alpha=float(np.float32(alpha)), r0=r0, rr_continue=float(np.float32(rr_continue)),
                cell_h=cell_h, eps=float(np.float32(eps_frac * ext)), photon_mode=int(photon_mode),
                hash_mode=int(hash_mode), max_eye_depth=int(max_eye_depth),
                max_photon_depth=int(max_photon_depth), scene_id=int(scene_id))


def _materials(mats):
    arr = (Material * len(mats))()
    for i, m in enumerate(mats):
        arr[i].type = int(m["type"])
        for c in range(3):
            arr[i].albedo[c] = float(m["albedo"][c])
            arr[i].emission[c] = float(m["emission"][c])
        arr[i].ior = float(m["ior"])
    return arr


def _camera(cam):
    c = cam[0] if cam.shape else cam
    out = Camera()
    for k in ("eye", "look", "up"):
        for i in range(3):
            getattr(out, k)[i] = float(c[k][i])
    out.vfov_deg = float(c["vfov_deg"])
    out.width, out.height = int(c["width"]), int(c["height"])
    return out


class Sppm:
    """FP64 SPPM renderer over one scene (Sec. 2-3.4)."""

    def __init__(self, scene, params: dict, mesh: Mesh | None = None):
        self.scene = scene
        self.mesh = mesh or Mesh(scene.verts, scene.tris, scene.tri_mat)
        self.mats = _materials(scene.mats)
        self.cam = _camera(scene.camera)
        self.params = SppmParams(**params)
        self.w, self.h = self.cam.width, self.cam.height
        self.handle = lib().orc_sppm_create(self.mesh.h, C.cast(self.mats, C.c_void_p), len(self.mats),
                                            C.byref(self.cam), C.byref(self.params))
        # shading data of the scene, if it has any (per-vertex normals, texture coordinates,
        # albedo textures per material)
        nrm, st = getattr(scene, "normals", None), getattr(scene, "texcoords", None)
        if mesh is None and (nrm is not None or st is not None):
            self.mesh.set_attributes(nrm, st)
        for m, rgb in (getattr(scene, "textures", None) or {}).items():
            self.set_texture(m, rgb)

    def set_texture(self, mat: int, rgb):
        """Albedo texture [h, w, 3] of diffuse material `mat`."""
        rgb = np.ascontiguousarray(rgb, np.float32)
        if lib().orc_sppm_set_texture(self.handle, int(mat), _p(rgb), rgb.shape[1], rgb.shape[0]) != 0:
            raise ValueError("oracle: bad texture")

    def surface(self, rays):
        """Shading at each ray's closest hit: dict(id, u, v, ns [n, 3], tex [n, 3], smooth)."""
        rays = np.ascontiguousarray(rays, np.float32)
        out = np.zeros((len(rays), 10))
        lib().orc_sppm_surface(self.handle, _p(rays), len(rays), _p(out))
        return dict(id=out[:, 0].astype(np.int64), u=out[:, 1], v=out[:, 2], ns=out[:, 3:6], tex=out[:, 6:9],
                    smooth=out[:, 9] > 0)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.orc_sppm_destroy(self.handle)
            self.handle = None

    def run(self, npasses: int, nthreads=None):
        rc = lib().orc_sppm_run(self.handle, npasses, nthreads or nthreads_default())
        if rc != 0:
            raise RuntimeError("oracle: scene has no emitter")

    def enable_grad(self):
        """Carry forward-mode derivatives (every material's albedo, the emitter's emission)."""
        if lib().orc_sppm_enable_grad(self.handle) != 0:
            raise RuntimeError("oracle: gradients need full paths, one emitting material, no pass run yet")

    def grad(self, g):
        """Gradient of sum(g * image) w.r.t. (albedo [nmat, 3], emission [3])."""
        g = np.ascontiguousarray(g, np.float64).reshape(-1, 3)
        ga = np.zeros((len(self.mats), 3))
        gl = np.zeros(3)
        if lib().orc_sppm_grad(self.handle, _p(g), _p(ga), _p(gl)) != 0:
            raise RuntimeError("oracle: enable_grad() and run() first")
        return ga, gl

    def state(self):
        n = self.w * self.h
        N, R = np.zeros(n), np.zeros(n)
        tau, direct, img = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
        ne = np.zeros(2)
        lib().orc_sppm_state(self.handle, _p(N), _p(R), _p(tau), _p(direct), _p(img), _p(ne))
        hw = (self.h, self.w)
        return dict(N=N.reshape(hw), R=R.reshape(hw), tau=tau.reshape(hw + (3,)),
                    direct=direct.reshape(hw + (3,)), image=img.reshape(hw + (3,)),
                    Ne=ne[0], passes=int(ne[1]))

    def image(self):
        return self.state()["image"]

    def last_photons(self):
        """Deposits of the last pass: ids, positions, fluxes, incoming directions."""
        n = lib().orc_sppm_last_photons(self.handle, None, None, None, None)
        ids = np.zeros(n, np.uint32)
        x, phi, din = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
        lib().orc_sppm_last_photons(self.handle, _p(ids), _p(x), _p(phi), _p(din))
        return dict(ids=ids, x=x, phi=phi, din=din)

    def last_gather(self):
        """Hit points and gathered (M, Phi) of the last pass, per pixel."""
        n = self.w * self.h
        M, Phi = np.zeros(n), np.zeros((n, 3))
        valid, hx = np.zeros(n, np.int32), np.zeros((n, 3))
        hn, hw, hm = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n, np.int32)
        lib().orc_sppm_last_gather(self.handle, _p(M), _p(Phi), _p(valid), _p(hx), _p(hn), _p(hw),
                                   _p(hm))
        return dict(M=M, Phi=Phi, valid=valid, x=hx, n=hn, w=hw, mat=hm)


def hash_grid(xyz, h, T):
    """Exact hash grid of float32 points: (bucket, order by (bucket, index), bucket starts,
    near-boundary flags)."""
    xyz = np.ascontiguousarray(xyz, np.float32)
    n = len(xyz)
    b, order = np.zeros(n, np.uint32), np.zeros(n, np.uint32)
    starts, near = np.zeros(T + 1, np.uint32), np.zeros(n, np.int32)
    lib().orc_hash_grid(_p(xyz), n, float(h), int(T), _p(b), _p(order), _p(starts), _p(near))
    return b, order, starts, near


def sppm_update(alpha, M, Phi, N, R, tau):
    """Apply the progressive update for one pass in place (FP64)."""
    M = np.ascontiguousarray(M, np.float64)
    Phi = np.ascontiguousarray(Phi, np.float64)
    lib().orc_sppm_update(len(M), float(alpha), _p(M), _p(Phi), _p(N), _p(R), _p(tau))
