"""Handle ownership in the Python binding (no GPU): closing a context first closes the scenes and
renderers made from it, so no C handle is destroyed after the handle it points to."""
import numpy as np

from paper_1505_06022_gb300 import gsp


def test_parents_close_children_first(monkeypatch):
    calls = []

    class FakeLib:
        def __getattr__(self, name):
            return lambda *a: calls.append(name) or 0

    monkeypatch.setattr(gsp, "_lib", FakeLib())
    monkeypatch.setattr(gsp, "gsp_context_create", lambda d: 11)
    monkeypatch.setattr(gsp, "gsp_scene_upload", lambda *a: 22)
    monkeypatch.setattr(gsp, "gsp_build_bvh", lambda *a, **k: {})
    monkeypatch.setattr(gsp, "gsp_sppm_create", lambda *a: 33)
    src = type("Src", (), {})()
    src.verts = src.tris = src.tri_mat = src.mats = None
    src.camera = np.zeros(1, dtype=[("width", "i4"), ("height", "i4")])
    ctx = gsp.Context(0)
    scenes = [gsp.Scene(ctx, src) for _ in range(2)]
    renderers = [gsp.Renderer(scenes[0], {}), gsp.Renderer(scenes[0], {}), gsp.Renderer(scenes[1], {})]
    ctx.close()
    assert calls.count("gsp_sppm_destroy") == 3 and calls.count("gsp_scene_destroy") == 2
    assert calls[-1] == "gsp_context_destroy"
    # every renderer went before its scene
    first_scene = calls.index("gsp_scene_destroy")
    assert calls[:2] == ["gsp_sppm_destroy", "gsp_sppm_destroy"] and first_scene == 2
    n = len(calls)
    for obj in renderers + scenes + [ctx]:  # closing again is a no-op
        obj.close()
    assert len(calls) == n
