"""Python binding of the C ABI in include/gsp.h (ctypes; argument marshalling only).

Every function named ``gsp_*`` here calls the C entry point of the same name in libgsp.so.
Device arrays are torch CUDA tensors (contiguous, 16-byte aligned); host arrays are numpy.
There is no fallback: if the CUDA library is missing or fails to load, calls raise.

``Scene`` and ``Renderer`` are thin owners of the opaque handles for convenience.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
import weakref

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgsp.so")
_lock = threading.Lock()
_lib = None

GSP_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA runtime error",
          -4: "traversal exceeded its step limit", -5: "bounded device wait timed out",
          -6: "scene has no BVH", -7: "call order violated", -8: "checkpoint I/O failed",
          -9: "device buffer overflow"}
FULL_PATH, REGEN = 0, 1
TRAVERSAL_MTBVH, TRAVERSAL_STACK = 1, 2
EXACT, STOCHASTIC = 0, 1

# exported symbols of include/gsp.h
ABI = ["gsp_status_string", "gsp_last_error_message", "gsp_context_create", "gsp_context_destroy",
       "gsp_context_sync", "gsp_scene_upload", "gsp_scene_destroy", "gsp_build_bvh",
       "gsp_build_bvh_device", "gsp_scene_set_step_limit", "gsp_trace_closest_hit", "gsp_trace_closest_hit_stack", "gsp_trace_closest_hit_host", "gsp_bvh_host_walk", "gsp_bvh_export", "gsp_sppm_create",
       "gsp_sppm_destroy", "gsp_sppm_pass", "gsp_sppm_image", "gsp_sppm_state",
       "gsp_sppm_last_deposits", "gsp_sppm_sync", "gsp_rng_fill", "gsp_hash_grid_build",
       "gsp_hash_grid_build_static", "gsp_sppm_tune", "gsp_sppm_enable_grad", "gsp_render_grad",
       "gsp_scene_set_materials", "gsp_batch_create", "gsp_batch_destroy", "gsp_batch_pass",
       "gsp_sppm_autotune", "gsp_sppm_save", "gsp_sppm_load", "gsp_batch_autotune", "gsp_batch_tune",
       "gsp_scene_set_attributes", "gsp_scene_set_texture", "gsp_measure_read_bandwidth", "gsp_sppm_count_work",
       "gsp_sppm_set_state", "gsp_trace_time_launches", "gsp_trace_launch_times"]
GRID_STATIC_MAX_POINTS = 524288
GRID_STATIC_MAX_TABLE = 16777216


class GspError(RuntimeError):
    def __init__(self, fn, code):
        msg = STATUS.get(code, f"status {code}")
        detail = ""
        if _lib is not None:
            detail = _lib.gsp_last_error_message().decode(errors="replace")
        super().__init__(f"{fn}: {msg}" + (f" ({detail})" if detail else ""))
        self.code = code


class BvhParams(C.Structure):
    _fields_ = [("bins", C.c_int32), ("leaf_threshold", C.c_int32), ("max_leaf", C.c_int32),
                ("link_sets", C.c_int32)]


class BvhStats(C.Structure):
    _fields_ = [("nodes", C.c_int64), ("leaves", C.c_int64), ("depth", C.c_int32),
                ("link_sets", C.c_int32), ("build_ms", C.c_double), ("thread_ms", C.c_double),
                ("device_bytes", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneResult(C.Structure):
    _fields_ = [("eye_steps", C.c_int32), ("photon_steps", C.c_int32), ("cell_h", C.c_float),
                ("ms_per_pass", C.c_float), ("first_ms_per_pass", C.c_float), ("candidates", C.c_int32),
                ("gather_lanes", C.c_int32), ("traversal", C.c_int32), ("fused", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SppmParams(C.Structure):
    _fields_ = [("photons_per_pass", C.c_int64), ("table_size", C.c_int64), ("seed", C.c_uint64),
                ("alpha", C.c_float), ("r0", C.c_float), ("rr_continue", C.c_float),
                ("cell_h", C.c_float), ("eps", C.c_float), ("photon_mode", C.c_int32),
                ("hash_mode", C.c_int32), ("max_eye_depth", C.c_int32),
                ("max_photon_depth", C.c_int32), ("scene_id", C.c_uint32)]


def lib():
    """Loads libgsp.so (building it first if the sources are newer). Raises on failure."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            path = _build.build()
            L = C.CDLL(path)
            P, I64, I32 = C.c_void_p, C.c_int64, C.c_int32
            for name in ABI:
                getattr(L, name)  # every declared symbol must be exported
            L.gsp_status_string.restype = C.c_char_p
            L.gsp_status_string.argtypes = [I32]
            L.gsp_last_error_message.restype = C.c_char_p
            L.gsp_last_error_message.argtypes = []
            L.gsp_context_create.argtypes = [I32, C.POINTER(P)]
            L.gsp_context_destroy.argtypes = [P]
            L.gsp_context_destroy.restype = None
            L.gsp_context_sync.argtypes = [P]
            L.gsp_scene_upload.argtypes = [P, P, I64, P, I64, P, P, I32, P, C.POINTER(P)]
            L.gsp_scene_destroy.argtypes = [P]
            L.gsp_scene_destroy.restype = None
            L.gsp_build_bvh.argtypes = [P, P, P]
            L.gsp_build_bvh_device.argtypes = [P, I32, I32, P]
            L.gsp_scene_set_step_limit.argtypes = [P, I32]
            L.gsp_scene_set_attributes.argtypes = [P, P, P]
            L.gsp_scene_set_texture.argtypes = [P, I32, P, I32, I32]
            L.gsp_trace_closest_hit.argtypes = [P, P, I64, P, P, P, P]
            L.gsp_trace_time_launches.argtypes = [P, I64]
            L.gsp_trace_launch_times.argtypes = [P, P, I64, C.POINTER(I64)]
            L.gsp_trace_closest_hit_stack.argtypes = [P, P, I64, P, P, P, P]
            L.gsp_trace_closest_hit_host.argtypes = [P, P, I64, P, P, P]
            L.gsp_bvh_host_walk.argtypes = [P, P, I64, P, P, P, P]
            L.gsp_bvh_export.argtypes = [P, I32, P, P, C.POINTER(I64)]
            L.gsp_sppm_create.argtypes = [P, P, C.POINTER(P)]
            L.gsp_sppm_destroy.argtypes = [P]
            L.gsp_sppm_destroy.restype = None
            L.gsp_sppm_pass.argtypes = [P, I32, P]
            L.gsp_sppm_image.argtypes = [P, P, P]
            L.gsp_sppm_state.argtypes = [P, P, P, P, P, P, P]
            L.gsp_sppm_last_deposits.restype = I64
            L.gsp_sppm_last_deposits.argtypes = [P, P, I64]
            L.gsp_sppm_sync.argtypes = [P]
            L.gsp_hash_grid_build.argtypes = [P, P, I64, C.c_float, I64, P, P, P]
            L.gsp_hash_grid_build_static.argtypes = [P, I64, C.c_float, I64, P, P, P]
            L.gsp_sppm_tune.argtypes = [P, I32, I32, C.c_float, I32, I32]
            L.gsp_sppm_enable_grad.argtypes = [P, I32]
            L.gsp_render_grad.argtypes = [P, P, P, P, P]
            L.gsp_scene_set_materials.argtypes = [P, P, I32]
            L.gsp_batch_create.argtypes = [P, I32, C.POINTER(P)]
            L.gsp_batch_destroy.argtypes = [P]
            L.gsp_batch_destroy.restype = None
            L.gsp_batch_pass.argtypes = [P, I32, P]
            L.gsp_sppm_autotune.argtypes = [P, I32, P]
            L.gsp_batch_autotune.argtypes = [P, I32, P]
            L.gsp_batch_tune.argtypes = [P, I32]
            L.gsp_sppm_save.argtypes = [P, C.c_char_p]
            L.gsp_sppm_load.argtypes = [P, C.c_char_p]
            L.gsp_rng_fill.argtypes = [P, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, P, I64, I32, P, P]
            L.gsp_measure_read_bandwidth.argtypes = [P, I64, I32, C.POINTER(C.c_double)]
            L.gsp_sppm_count_work.argtypes = [P, I32, P]
            L.gsp_sppm_set_state.argtypes = [P, P, P, P, P, I64, P]
            _lib = L
    return _lib


def _check(fn, code):
    if code != GSP_OK:
        raise GspError(fn, code)


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


def _dev(t, dtypes=None, numel=None, what="tensor"):
    """Device pointer of a torch CUDA tensor (or None). dtypes: accepted element types by name
    ("float32", "int32", ...); numel: the fewest elements the call reads or writes."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous CUDA tensor")
    if dtypes is not None and str(t.dtype).replace("torch.", "") not in dtypes:
        raise TypeError(f"{what}: expected {' or '.join(dtypes)} elements, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{what}: expected at least {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


F32, I32 = ("float32",), ("int32",)


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(getattr(stream, "cuda_stream", stream) or 0)


# ------------------------------------------------------------------------- C ABI mirrors
def gsp_context_create(device: int = 0):
    h = C.c_void_p()
    _check("gsp_context_create", lib().gsp_context_create(device, C.byref(h)))
    return h


def gsp_context_destroy(ctx):
    lib().gsp_context_destroy(ctx)


def gsp_context_sync(ctx):
    _check("gsp_context_sync", lib().gsp_context_sync(ctx))


def gsp_rng_fill(ctx, seed, scene, domain, pass_, ids, ndraw, out=None, stream=None):
    """ids: CUDA int64/uint64 tensor [n]; returns CUDA float32 [n, ndraw]."""
    import torch
    if out is None:
        out = torch.empty((ids.shape[0], ndraw), dtype=torch.float32, device=ids.device)
    n = ids.shape[0]
    rc = lib().gsp_rng_fill(ctx, seed, scene, domain, pass_, _dev(ids, ("int64", "uint64"), n, "ids"), n, ndraw,
                            _dev(out, F32, n * ndraw, "out"), _stream(stream))
    _check("gsp_rng_fill", rc)
    return out


def gsp_hash_grid_build(ctx, pos, cell_h, table_size, order=None, bstart=None, stream=None):
    """pos: CUDA float32 [n, 4]; returns (order uint32-as-int32 [n], bstart [table_size + 1])."""
    import torch
    n = pos.shape[0]
    if order is None:
        order = torch.empty(n, dtype=torch.int32, device=pos.device)
    if bstart is None:
        bstart = torch.empty(table_size + 1, dtype=torch.int32, device=pos.device)
    rc = lib().gsp_hash_grid_build(ctx, _dev(pos, F32, 4 * n, "pos"), n, cell_h, table_size,
                                   _dev(order, I32, n, "order"), _dev(bstart, I32, table_size + 1, "bstart"),
                                   _stream(stream))
    _check("gsp_hash_grid_build", rc)
    return order, bstart


WORK_COUNTS = ["eye_rays", "photon_rays", "node_visits", "tri_tests", "deposits", "hit_points",
               "photons_scanned", "hit_points_scanned"]


def gsp_sppm_count_work(r, on):
    """Counts accumulated since the previous call (dict by WORK_COUNTS name); then counting on/off."""
    out = (C.c_uint64 * len(WORK_COUNTS))()
    _check("gsp_sppm_count_work", lib().gsp_sppm_count_work(r, 1 if on else 0, out))
    return dict(zip(WORK_COUNTS, (int(v) for v in out)))


def gsp_measure_read_bandwidth(ctx, nbytes, reps):
    """GB/s of a streaming read over a device buffer of `nbytes` (L2 below its size, HBM above)."""
    out = C.c_double()
    _check("gsp_measure_read_bandwidth", lib().gsp_measure_read_bandwidth(ctx, int(nbytes), int(reps), C.byref(out)))
    return out.value


def gsp_hash_grid_build_static(pos, cell_h, table_size, order, bstart, stream=None):
    """Allocation-free hash-grid build on the current device; order/bstart are caller tensors."""
    n = pos.shape[0]
    rc = lib().gsp_hash_grid_build_static(_dev(pos, F32, 4 * n, "pos"), n, cell_h, table_size,
                                          _dev(order, I32, n, "order"), _dev(bstart, I32, table_size + 1, "bstart"),
                                          _stream(stream))
    _check("gsp_hash_grid_build_static", rc)
    return order, bstart


def gsp_scene_upload(ctx, verts, tris, tri_mat=None, mats=None, camera=None):
    """ctx None = host-only scene (BVH build, export, host walk; no GPU)."""
    v, vp = _host(verts, np.float32)
    t, tp = _host(tris, np.int32)
    if tri_mat is None:
        tm, tmp_ = None, None
    else:
        tm, tmp_ = _host(tri_mat, np.int32)
    if mats is None:
        mats = _inputs.material(_inputs.DIFFUSE, (0.5, 0.5, 0.5))
    m = np.ascontiguousarray(mats, dtype=_inputs.MATERIAL_DTYPE)
    cam = None if camera is None else np.ascontiguousarray(camera, dtype=_inputs.CAMERA_DTYPE)
    h = C.c_void_p()
    rc = lib().gsp_scene_upload(ctx, vp, len(v), tp, len(t), tmp_, m.ctypes.data_as(C.c_void_p), len(m),
                                None if cam is None else cam.ctypes.data_as(C.c_void_p), C.byref(h))
    _check("gsp_scene_upload", rc)
    return h


def gsp_scene_destroy(scene):
    lib().gsp_scene_destroy(scene)


def gsp_build_bvh(scene, bins=16, leaf_threshold=4, max_leaf=7, link_sets=6) -> dict:
    p = BvhParams(bins, leaf_threshold, max_leaf, link_sets)
    st = BvhStats()
    _check("gsp_build_bvh", lib().gsp_build_bvh(scene, C.byref(p), C.byref(st)))
    return st.as_dict()


def gsp_scene_set_step_limit(scene, max_box_tests):
    _check("gsp_scene_set_step_limit", lib().gsp_scene_set_step_limit(scene, max_box_tests))


def gsp_scene_set_attributes(scene, normals=None, texcoords=None):
    """Per-vertex normals float32 [nv, 3] and texture coordinates float32 [nv, 2] (None = none)."""
    n = None if normals is None else np.ascontiguousarray(normals, np.float32)
    st = None if texcoords is None else np.ascontiguousarray(texcoords, np.float32)
    _check("gsp_scene_set_attributes", lib().gsp_scene_set_attributes(
        scene, None if n is None else n.ctypes.data_as(C.c_void_p), None if st is None else st.ctypes.data_as(C.c_void_p)))


def gsp_scene_set_texture(scene, material, rgb):
    """Albedo texture float32 [h, w, 3] of a diffuse material (None removes it)."""
    if rgb is None:
        _check("gsp_scene_set_texture", lib().gsp_scene_set_texture(scene, int(material), None, 0, 0))
        return
    t = np.ascontiguousarray(rgb, np.float32)
    _check("gsp_scene_set_texture", lib().gsp_scene_set_texture(scene, int(material), t.ctypes.data_as(C.c_void_p),
                                                                t.shape[1], t.shape[0]))


def gsp_build_bvh_device(scene, link_sets=6, max_leaf=4) -> dict:
    st = BvhStats()
    _check("gsp_build_bvh_device", lib().gsp_build_bvh_device(scene, link_sets, max_leaf, C.byref(st)))
    return st.as_dict()


def gsp_trace_closest_hit(scene, rays, tri, t, uv=None, stream=None):
    """rays: CUDA float32 [n, 8]; tri: CUDA int32 [n]; t: CUDA float32 [n]; uv: [n, 2] or None."""
    n = rays.shape[0]
    rc = lib().gsp_trace_closest_hit(scene, _dev(rays, F32, 8 * n, "rays"), n, _dev(tri, I32, n, "tri"),
                                     _dev(t, F32, n, "t"), _dev(uv, F32, 2 * n, "uv"), _stream(stream))
    _check("gsp_trace_closest_hit", rc)


def gsp_trace_time_launches(scene, n):
    """The next n gsp_trace_closest_hit calls on `scene` record their traversal kernel's duration."""
    _check("gsp_trace_time_launches", lib().gsp_trace_time_launches(scene, int(n)))


def gsp_trace_launch_times(scene, capacity):
    """Durations (ms, numpy float32) of the traversal kernels recorded since gsp_trace_time_launches."""
    out = np.zeros(max(0, int(capacity)), np.float32)
    cnt = C.c_int64()
    _check("gsp_trace_launch_times",
           lib().gsp_trace_launch_times(scene, out.ctypes.data if len(out) else None, len(out), C.byref(cnt)))
    return out[:min(cnt.value, len(out))]


def gsp_trace_closest_hit_stack(scene, rays, tri, t, uv=None, stream=None):
    """As gsp_trace_closest_hit, by stack-based near-first traversal of the same tree."""
    n = rays.shape[0]
    rc = lib().gsp_trace_closest_hit_stack(scene, _dev(rays, F32, 8 * n, "rays"), n, _dev(tri, I32, n, "tri"),
                                           _dev(t, F32, n, "t"), _dev(uv, F32, 2 * n, "uv"), _stream(stream))
    _check("gsp_trace_closest_hit_stack", rc)


def _host_ptr(x):
    """Address of a host array: a CPU torch tensor (pinned or not) or a C-contiguous numpy array."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if x.is_cuda or not x.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor")
        return x.data_ptr()
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous array")
    return x.ctypes.data


def gsp_trace_closest_hit_host(scene, rays, tri, t, uv=None):
    """Host buffers (numpy arrays or CPU tensors): rays float32 [n, 8] in; tri int32 [n], t float32
    [n], uv float32 [n, 2] or None out. Synchronous; copies overlap the traversal."""
    n = rays.shape[0]
    rc = lib().gsp_trace_closest_hit_host(scene, _host_ptr(rays), n, _host_ptr(tri), _host_ptr(t), _host_ptr(uv))
    _check("gsp_trace_closest_hit_host", rc)


def gsp_bvh_host_walk(scene, rays):
    r, rp = _host(rays, np.float32)
    n = len(r)
    tri, t = np.zeros(n, np.int32), np.zeros(n, np.float32)
    vis, tests = np.zeros(n, np.int32), np.zeros(n, np.int32)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    _check("gsp_bvh_host_walk", lib().gsp_bvh_host_walk(scene, rp, n, p(tri), p(t), p(vis), p(tests)))
    return tri, t, vis, tests


def gsp_bvh_export(scene, link_set=0):
    nn = C.c_int64()
    _check("gsp_bvh_export", lib().gsp_bvh_export(scene, link_set, None, None, C.byref(nn)))
    nodes = np.zeros((nn.value, 8), np.float32)
    return nodes, nn.value


def bvh_export_full(scene, ntris, link_set=0):
    nodes, nn = gsp_bvh_export(scene, link_set)
    tris = np.zeros((ntris, 12), np.float32)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    _check("gsp_bvh_export", lib().gsp_bvh_export(scene, link_set, p(nodes), p(tris), C.byref(C.c_int64())))
    return nodes, tris


def gsp_sppm_create(scene, params: dict):
    p = SppmParams(**params)
    h = C.c_void_p()
    _check("gsp_sppm_create", lib().gsp_sppm_create(scene, C.byref(p), C.byref(h)))
    return h


def gsp_sppm_tune(r, eye_steps=0, photon_steps=0, refine_factor=0.0, gather_lanes=0, traversal=0):
    _check("gsp_sppm_tune", lib().gsp_sppm_tune(r, eye_steps, photon_steps, refine_factor, gather_lanes, traversal))


def gsp_sppm_enable_grad(r, max_passes):
    _check("gsp_sppm_enable_grad", lib().gsp_sppm_enable_grad(r, max_passes))


def gsp_render_grad(r, dloss_dimg, grad_albedo, grad_emission, stream=None):
    rc = lib().gsp_render_grad(r, _dev(dloss_dimg, F32, what="dloss_dimg"), _dev(grad_albedo, F32, what="grad_albedo"),
                               _dev(grad_emission, F32, 3, "grad_emission"), _stream(stream))
    _check("gsp_render_grad", rc)


def gsp_scene_set_materials(scene, mats):
    m = np.ascontiguousarray(mats, dtype=_inputs.MATERIAL_DTYPE)
    _check("gsp_scene_set_materials", lib().gsp_scene_set_materials(scene, m.ctypes.data_as(C.c_void_p), len(m)))


def gsp_sppm_autotune(r, trial_passes=2) -> dict:
    out = TuneResult()
    _check("gsp_sppm_autotune", lib().gsp_sppm_autotune(r, trial_passes, C.byref(out)))
    return out.as_dict()


def gsp_batch_tune(b, fused):
    _check("gsp_batch_tune", lib().gsp_batch_tune(b, 1 if fused else 0))


def gsp_batch_autotune(b, trial_passes=2) -> dict:
    out = TuneResult()
    _check("gsp_batch_autotune", lib().gsp_batch_autotune(b, trial_passes, C.byref(out)))
    return out.as_dict()


def gsp_batch_create(renderer_handles):
    arr = (C.c_void_p * len(renderer_handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in renderer_handles])
    h = C.c_void_p()
    _check("gsp_batch_create", lib().gsp_batch_create(arr, len(renderer_handles), C.byref(h)))
    return h


def gsp_batch_destroy(b):
    lib().gsp_batch_destroy(b)


def gsp_batch_pass(b, npasses=1, stream=None):
    _check("gsp_batch_pass", lib().gsp_batch_pass(b, npasses, _stream(stream)))


def gsp_sppm_save(r, path):
    _check("gsp_sppm_save", lib().gsp_sppm_save(r, os.fsencode(path)))


def gsp_sppm_load(r, path):
    _check("gsp_sppm_load", lib().gsp_sppm_load(r, os.fsencode(path)))


def gsp_sppm_destroy(r):
    lib().gsp_sppm_destroy(r)


def gsp_sppm_pass(r, npasses=1, stream=None):
    _check("gsp_sppm_pass", lib().gsp_sppm_pass(r, npasses, _stream(stream)))


def gsp_sppm_image(r, rgb, stream=None):
    _check("gsp_sppm_image", lib().gsp_sppm_image(r, _dev(rgb, F32, what="rgb"), _stream(stream)))


def gsp_sppm_state(r, N=None, R=None, tau=None, direct=None, stream=None):
    counts = np.zeros(2, np.float64)
    rc = lib().gsp_sppm_state(r, _dev(N, F32, what="N"), _dev(R, F32, what="R"), _dev(tau, F32, what="tau"),
                              _dev(direct, F32, what="direct"),
                              counts.ctypes.data_as(C.c_void_p), _stream(stream))
    _check("gsp_sppm_state", rc)
    return int(counts[0]), float(counts[1])


def gsp_sppm_set_state(r, N, R, tau, direct, passes, stream=None):
    _check("gsp_sppm_set_state", lib().gsp_sppm_set_state(r, _dev(N, F32, what="N"), _dev(R, F32, what="R"),
                                                          _dev(tau, F32, what="tau"),
                                                          _dev(direct, F32, what="direct"), int(passes),
                                                          _stream(stream)))


def gsp_sppm_last_deposits(r):
    n = lib().gsp_sppm_last_deposits(r, None, 0)
    if n < 0:
        raise GspError("gsp_sppm_last_deposits", n)
    ids = np.zeros(max(n, 1), np.uint32)
    n2 = lib().gsp_sppm_last_deposits(r, ids.ctypes.data_as(C.c_void_p), len(ids))
    if n2 < 0:
        raise GspError("gsp_sppm_last_deposits", n2)
    return ids[:n2]


def gsp_sppm_sync(r):
    _check("gsp_sppm_sync", lib().gsp_sppm_sync(r))


# ------------------------------------------------------------------------- convenience owners
class Context:
    """Owns a gsp_context. Closing it first closes every scene (and renderer) made from it, so no
    handle outlives the context it points to."""

    def __init__(self, device: int = 0):
        self.h = gsp_context_create(device)
        self.device = device
        self._children = weakref.WeakSet()

    def sync(self):
        gsp_context_sync(self.h)

    def close(self):
        for ch in list(self._children):
            ch.close()
        if self.h:
            gsp_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scene:
    """Uploaded scene + BVH. `ctx` None makes a host-only scene."""

    def __init__(self, ctx, scene: "_inputs.Scene", builder="host", **bvh):
        """builder "host": binned SAH on the host (bins, leaf_threshold, max_leaf, link_sets);
        "device": Morton-order LBVH built on the GPU (link_sets, max_leaf)."""
        self.ctx = ctx
        self.src = scene
        self._children = weakref.WeakSet()
        self.h = gsp_scene_upload(None if ctx is None else ctx.h, scene.verts, scene.tris, scene.tri_mat,
                                  scene.mats, scene.camera)
        if ctx is not None:
            ctx._children.add(self)
        if builder == "device":
            self.stats = gsp_build_bvh_device(self.h, bvh.get("link_sets", 6), bvh.get("max_leaf", 4))
        else:
            self.stats = gsp_build_bvh(self.h, **bvh)
        # per-vertex shading data and albedo textures, when the input scene has them
        nrm, st = getattr(scene, "normals", None), getattr(scene, "texcoords", None)
        if nrm is not None or st is not None:
            gsp_scene_set_attributes(self.h, nrm, st)
        for m, rgb in (getattr(scene, "textures", None) or {}).items():
            gsp_scene_set_texture(self.h, m, rgb)

    def trace(self, rays, stream=None, with_uv=False, method="mtbvh"):
        """Closest hits; method "mtbvh" (stackless, the scene's link sets) or "stack"."""
        import torch
        n = rays.shape[0]
        tri = torch.empty(n, dtype=torch.int32, device=rays.device)
        t = torch.empty(n, dtype=torch.float32, device=rays.device)
        uv = torch.empty((n, 2), dtype=torch.float32, device=rays.device) if with_uv else None
        fn = {"mtbvh": gsp_trace_closest_hit, "stack": gsp_trace_closest_hit_stack}[method]
        fn(self.h, rays, tri, t, uv, stream)
        return (tri, t, uv) if with_uv else (tri, t)

    def host_walk(self, rays):
        return gsp_bvh_host_walk(self.h, rays)

    def close(self):
        for ch in list(self._children):
            ch.close()
        if self.h:
            gsp_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Renderer:
    """SPPM renderer over an uploaded scene."""

    def __init__(self, scene: Scene, params: dict):
        self.scene = scene
        self.params = dict(params)
        self.h = gsp_sppm_create(scene.h, self.params)
        scene._children.add(self)
        cam = scene.src.camera[0]
        self.w, self.h_px = int(cam["width"]), int(cam["height"])

    def run(self, npasses=1, stream=None):
        gsp_sppm_pass(self.h, npasses, stream)

    def tune(self, eye_steps=0, photon_steps=0, refine_factor=0.0, gather_lanes=0, traversal=0):
        """traversal: 0 keep, TRAVERSAL_MTBVH or TRAVERSAL_STACK (path kernel)."""
        gsp_sppm_tune(self.h, eye_steps, photon_steps, refine_factor, gather_lanes, traversal)

    def autotune(self, trial_passes=2) -> dict:
        return gsp_sppm_autotune(self.h, trial_passes)

    def image(self, stream=None):
        import torch
        img = torch.empty((self.h_px, self.w, 3), dtype=torch.float32, device=f"cuda:{self.scene.ctx.device}")
        gsp_sppm_image(self.h, img, stream)
        return img

    def state(self, stream=None):
        import torch
        dev = f"cuda:{self.scene.ctx.device}"
        n = self.w * self.h_px
        N = torch.empty(n, device=dev)
        R = torch.empty(n, device=dev)
        tau = torch.empty((n, 3), device=dev)
        direct = torch.empty((n, 3), device=dev)
        passes, ne = gsp_sppm_state(self.h, N, R, tau, direct, stream)
        hw = (self.h_px, self.w)
        return dict(N=N.view(hw), R=R.view(hw), tau=tau.view(hw + (3,)), direct=direct.view(hw + (3,)),
                    passes=passes, Ne=ne)

    def last_deposits(self):
        return gsp_sppm_last_deposits(self.h)

    def set_state(self, N, R, tau, direct, passes, stream=None):
        """Replace the progressive state (device float32 arrays shaped as state() returns them)."""
        npix = self.w * self.h_px
        for t, k, name in ((N, 1, "N"), (R, 1, "R"), (tau, 3, "tau"), (direct, 3, "direct")):
            if t.numel() != k * npix:
                raise ValueError(f"set_state: {name} has {t.numel()} elements, expected {k * npix}")
        c = lambda t: t.contiguous()
        gsp_sppm_set_state(self.h, c(N), c(R), c(tau), c(direct), passes, stream)

    def count_work(self, on):
        """Work counts of the passes since the previous call; then counting on or off."""
        return gsp_sppm_count_work(self.h, on)

    def save(self, path):
        gsp_sppm_save(self.h, path)

    def load(self, path):
        gsp_sppm_load(self.h, path)

    def enable_grad(self, max_passes):
        gsp_sppm_enable_grad(self.h, max_passes)

    def grad(self, dloss_dimg, stream=None):
        """(d loss / d albedo [nmat, 3], d loss / d emission [3]) for the given image gradient."""
        import torch
        dev = dloss_dimg.device
        nmat = len(self.scene.src.mats)
        ga = torch.empty((nmat, 3), dtype=torch.float32, device=dev)
        gl = torch.empty(3, dtype=torch.float32, device=dev)
        gsp_render_grad(self.h, dloss_dimg.contiguous(), ga, gl, stream)
        return ga, gl

    def sync(self):
        gsp_sppm_sync(self.h)

    def close(self):
        if self.h:
            gsp_sppm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Renderers whose passes run together as one CUDA graph (gsp_batch_*). Closing a renderer's
    scene or context first closes the batch."""

    def __init__(self, renderers):
        self.renderers = list(renderers)
        self.h = gsp_batch_create([r.h for r in self.renderers])
        for r in self.renderers:
            r.scene._children.add(self)

    def run(self, npasses=1, stream=None):
        gsp_batch_pass(self.h, npasses, stream)

    def autotune(self, trial_passes=2) -> dict:
        return gsp_batch_autotune(self.h, trial_passes)

    def tune(self, fused):
        """fused: one persistent path launch for all renderers per pass (else one per renderer)."""
        gsp_batch_tune(self.h, fused)

    def close(self):
        if self.h:
            gsp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sppm_params(scene, photons_per_pass, seed=1, alpha=0.7, r0=None, r0_frac=0.05, photon_mode=FULL_PATH,
                hash_mode=EXACT, cell_h=None, table_size=None, rr_continue=0.8, eps_frac=1e-4,
                max_eye_depth=16, max_photon_depth=32, scene_id=0) -> dict:
    """SPPM parameters for a scene; radius and ray offset scale with the scene's diagonal. The
    hash cell edge and table size are left to the library (0: its defaults) unless given."""
    ext = scene.extent()
    r0 = float(np.float32(r0 if r0 is not None else r0_frac * ext))
    return dict(photons_per_pass=int(photons_per_pass), table_size=int(table_size or 0), seed=int(seed),
                alpha=float(np.float32(alpha)), r0=r0, rr_continue=float(np.float32(rr_continue)),
                cell_h=float(np.float32(cell_h)) if cell_h else 0.0, eps=float(np.float32(eps_frac * ext)),
                photon_mode=int(photon_mode), hash_mode=int(hash_mode), max_eye_depth=int(max_eye_depth),
                max_photon_depth=int(max_photon_depth), scene_id=int(scene_id))


def emitting_material(mats) -> int:
    """Index of the single emitting material (the one whose emission the gradient covers)."""
    em = [i for i, m in enumerate(mats) if m["type"] in (_inputs.DIFFUSE, _inputs.EMITTER) and max(m["emission"]) > 0]
    if len(em) != 1:
        raise ValueError("gradients need exactly one emitting material")
    return em[0]


def _make_render_function():
    import torch

    class SPPMRender(torch.autograd.Function):
        """image = SPPM render of `scene` with the given material albedos [nmat, 3] and emission [3]
        of the emitting material; backward = gsp_render_grad (path-replay adjoint)."""

        @staticmethod
        def forward(ctx, albedo, emission, scene, params, passes):
            mats = scene.src.mats.copy()
            mats["albedo"] = albedo.detach().cpu().numpy()
            em = emitting_material(mats)
            mats["emission"][em] = emission.detach().cpu().numpy()
            gsp_scene_set_materials(scene.h, mats)
            r = Renderer(scene, params)
            r.enable_grad(passes)
            r.run(passes)
            img = r.image()
            ctx.renderer = r
            return img

        @staticmethod
        def backward(ctx, grad_img):
            ga, gl = ctx.renderer.grad(grad_img.float())
            return ga, gl, None, None, None

    return SPPMRender


_render_fn = None


def render(albedo, emission, scene, params, passes):
    """Differentiable SPPM render (torch autograd): see SPPMRender."""
    global _render_fn
    if _render_fn is None:
        _render_fn = _make_render_function()
    return _render_fn.apply(albedo, emission, scene, params, passes)
