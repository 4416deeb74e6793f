"""Handle ownership in the Python binding (no GPU): closing a context first closes the scenes and
renderers made from it, so no C handle is destroyed after the handle it points to."""
import numpy as np

from paper_1505_06022_gb300 import gsp


def test_parents_close_children_first(monkeypatch):
    calls = []
    handles = iter(range(100, 200))

    class FakeLib:
        def __getattr__(self, name):
            return lambda *a: calls.append((name,) + a) or 0

    monkeypatch.setattr(gsp, "_lib", FakeLib())
    monkeypatch.setattr(gsp, "gsp_context_create", lambda d: 11)
    monkeypatch.setattr(gsp, "gsp_scene_upload", lambda *a: next(handles))
    monkeypatch.setattr(gsp, "gsp_build_bvh", lambda *a, **k: {})
    monkeypatch.setattr(gsp, "gsp_sppm_create", lambda *a: next(handles))
    src = type("Src", (), {})()
    src.verts = src.tris = src.tri_mat = src.mats = None
    src.camera = np.zeros(1, dtype=[("width", "i4"), ("height", "i4")])
    ctx = gsp.Context(0)
    scenes = [gsp.Scene(ctx, src) for _ in range(2)]
    renderers = [gsp.Renderer(scenes[0], {}), gsp.Renderer(scenes[0], {}), gsp.Renderer(scenes[1], {})]
    owner = {renderers[0].h: scenes[0].h, renderers[1].h: scenes[0].h, renderers[2].h: scenes[1].h}
    ctx.close()
    names = [c[0] for c in calls]
    assert names.count("gsp_sppm_destroy") == 3 and names.count("gsp_scene_destroy") == 2
    assert names[-1] == "gsp_context_destroy"
    # every renderer went before its own scene
    when = {(c[0], c[1]): i for i, c in enumerate(calls)}
    for r, sc in owner.items():
        assert when[("gsp_sppm_destroy", r)] < when[("gsp_scene_destroy", sc)]
    n = len(calls)
    for obj in renderers + scenes + [ctx]:  # closing again is a no-op
        obj.close()
    assert len(calls) == n
