"""Batched passes (one CUDA graph over many renderers) and the autotuner, against the plain
per-renderer passes."""
import numpy as np
import pytest

from paper_1505_06022_gb300 import gsp, inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gsp.Context(0)
    yield c
    c.close()


def scenes():
    out = [I.cornell_box(width=48, height=40),
           I.full_scene(seed=7, width=64, height=64, plane_quads=32, sphere_n=6),
           I.grad_scene(seed=8, width=40, height=56, plane_quads=24, sphere_n=5),
           I.cornell_box(seed=3, width=16, height=16)]
    kws = [dict(photons_per_pass=9000, seed=1), dict(photons_per_pass=15000, seed=2, r0_frac=0.01),
           dict(photons_per_pass=6000, seed=3, r0_frac=0.02), dict(photons_per_pass=4000, seed=4, photon_mode=1,
                                                                    hash_mode=1)]
    return out, kws


@pytest.mark.parametrize("fused", [False, True])
def test_batch_graph_matches_individual_passes(ctx, fused):
    scs, kws = scenes()
    solo = []
    for sc, kw in zip(scs, kws):
        r = gsp.Renderer(gsp.Scene(ctx, sc), gsp.sppm_params(sc, **kw))
        r.run(3)
        solo.append(r.image().cpu().numpy())
    rs = [gsp.Renderer(gsp.Scene(ctx, sc), gsp.sppm_params(sc, **kw)) for sc, kw in zip(scs, kws)]
    rs[0].run(1)  # a renderer that already ran a pass joins the batch at its own pass index
    rs[1].tune(1, 2)  # per-renderer wavefront settings differ inside one batch
    b = gsp.Batch(rs)
    b.tune(fused)
    b.run(2)      # one captured graph, replayed twice: renderer 0 at 3 passes, the others at 2
    for r in rs[1:]:
        r.run(1)  # plain passes continue from where the graph left off
    torch.cuda.synchronize()
    for r, want in zip(rs, solo):
        r.sync()
        assert np.array_equal(r.image().cpu().numpy(), want)
    b.close()


def test_batch_autotune_keeps_the_estimate(ctx):
    scs, kws = scenes()
    solo = []
    for sc, kw in zip(scs, kws):
        r = gsp.Renderer(gsp.Scene(ctx, sc), gsp.sppm_params(sc, **kw))
        r.run(3)
        solo.append((r.image().cpu().numpy(), r.state()["N"].cpu().numpy()))
    rs = [gsp.Renderer(gsp.Scene(ctx, sc), gsp.sppm_params(sc, **kw)) for sc, kw in zip(scs, kws)]
    b = gsp.Batch(rs)
    res = b.autotune(trial_passes=1)
    assert res["eye_steps"] in (0, 1) and res["photon_steps"] in (0, 1, 2) and res["gather_lanes"] in (4, 8, 16)
    assert 10 <= res["candidates"] <= 20 and res["ms_per_pass"] <= res["first_ms_per_pass"]
    r0 = np.float32(kws[0].get("r0_frac", 0.05) * scs[0].extent())
    assert any(abs(res["cell_h"] - f * r0) <= 1e-6 * r0 for f in (0.75, 1.0, 1.5, 2.0))  # renderer 0 is exact
    assert res["traversal"] in (1, 2) and res["fused"] in (0, 1)
    b.run(3)
    torch.cuda.synchronize()
    for r, (img, n) in zip(rs, solo):
        r.sync()
        st = r.state()
        assert st["passes"] == 3
        assert np.array_equal(st["N"].cpu().numpy(), n)  # the same photons were gathered
        np.testing.assert_allclose(r.image().cpu().numpy(), img, rtol=2e-5, atol=1e-7 * img.max())
    with pytest.raises(gsp.GspError):
        b.autotune(trial_passes=1)  # only before the first pass
    b.close()


def test_batch_rejects_shared_scene(ctx):
    sc = I.cornell_box(width=8, height=8)
    s = gsp.Scene(ctx, sc)
    r1 = gsp.Renderer(s, gsp.sppm_params(sc, 100))
    r2 = gsp.Renderer(s, gsp.sppm_params(sc, 100))
    with pytest.raises(gsp.GspError):
        gsp.Batch([r1, r2])


def test_autotune_keeps_the_estimate(ctx):
    sc = I.full_scene(seed=9, width=96, height=96, plane_quads=48, sphere_n=8)
    kw = dict(photons_per_pass=40000, seed=5, r0_frac=0.01)
    s = gsp.Scene(ctx, sc)
    ref = gsp.Renderer(s, gsp.sppm_params(sc, **kw))
    ref.run(3)
    a = ref.image().cpu().numpy()
    r = gsp.Renderer(s, gsp.sppm_params(sc, **kw))
    res = r.autotune(trial_passes=1)
    assert 12 <= res["candidates"] <= 21 and res["ms_per_pass"] <= res["first_ms_per_pass"]
    assert res["gather_lanes"] in (1, 4, 8, 16) and res["traversal"] in (1, 2)
    assert res["cell_h"] >= np.float32(0.5 * kw["r0_frac"] * sc.extent()) * 0.999
    r.run(3)
    b = r.image().cpu().numpy()
    # the same photons are gathered; only the summation order can differ with the cell size
    np.testing.assert_allclose(b, a, rtol=2e-5, atol=1e-7 * a.max())


def test_full_size_batch_matches_individual_renderers(ctx):
    """The batch configuration: 64 scenes (1k-200k triangles, 64^2-512^2, 2^18 photon paths per
    pass each) as fused graph passes; 8 of the renderers checked bit for bit against the same
    renderers run alone."""
    scs = I.batch_scenes(64, seed=5)
    scenes = [gsp.Scene(ctx, sc) for sc in scs]
    mk = lambda i: gsp.Renderer(scenes[i], gsp.sppm_params(scs[i], 1 << 18, seed=5 + i, r0_frac=0.004, scene_id=i))
    rs = [mk(i) for i in range(64)]
    b = gsp.Batch(rs)
    b.run(2)
    torch.cuda.synchronize()
    pick = np.random.default_rng(3).choice(64, 8, replace=False)
    for i in pick:
        rs[i].sync()
        alone = mk(i)
        alone.run(2)
        assert np.array_equal(rs[i].image().cpu().numpy(), alone.image().cpu().numpy()), i
        alone.close()
    b.close()
    for r in rs:
        r.close()
    for s in scenes:
        s.close()


def test_two_pass_graphs_match_individual_passes(ctx):
    """Fused batches with exact hashing run pairs of passes as two-pass graphs (the second pass
    traced beside the first, into the other trace sets) and an odd pass as a one-pass graph; with
    one-bounce-per-pass photon paths the second pass's photon front follows the first's. Five
    passes, then two more, must equal the renderers run alone."""
    scs = [I.full_scene(seed=11, width=48, height=40, plane_quads=24, sphere_n=5),
           I.cornell_box(seed=4, width=32, height=24),
           I.grad_scene(seed=12, width=40, height=32, plane_quads=16, sphere_n=4)]
    kws = [dict(photons_per_pass=12000, seed=7, r0_frac=0.01, scene_id=0),
           dict(photons_per_pass=6000, seed=8, photon_mode=1, scene_id=1),
           dict(photons_per_pass=9000, seed=9, r0_frac=0.02, scene_id=2)]
    solo = []
    for sc, kw in zip(scs, kws):
        r = gsp.Renderer(gsp.Scene(ctx, sc), gsp.sppm_params(sc, **kw))
        r.run(7)
        solo.append((r.image().cpu().numpy(), r.state()["N"].cpu().numpy()))
    rs = [gsp.Renderer(gsp.Scene(ctx, sc), gsp.sppm_params(sc, **kw)) for sc, kw in zip(scs, kws)]
    b = gsp.Batch(rs)
    b.tune(True)
    b.run(5)
    b.run(2)
    torch.cuda.synchronize()
    for r, (img, n) in zip(rs, solo):
        r.sync()
        st = r.state()
        assert st["passes"] == 7
        assert np.array_equal(st["N"].cpu().numpy(), n)
        assert np.array_equal(r.image().cpu().numpy(), img)
    b.close()


@pytest.mark.parametrize("fused", [False, True])
def test_batch_recaptures_after_a_scene_changes(ctx, fused):
    """A new BVH (host SAH with one link set, then the device build) and new shading data move a
    scene's device buffers; the next batch pass captures its graphs again instead of replaying
    ones that point at the old buffers. Closest hits, and so images, do not depend on the tree."""
    scs = [I.shaded_scene(seed=16, width=40, height=32, plane_quads=16, sphere_n=4, tex_size=16),
           I.full_scene(seed=17, width=32, height=32, plane_quads=16, sphere_n=4)]
    kws = [dict(photons_per_pass=8000, seed=2, r0_frac=0.02, scene_id=0),
           dict(photons_per_pass=8000, seed=3, r0_frac=0.02, scene_id=1)]
    solo = []
    for sc, kw in zip(scs, kws):
        r = gsp.Renderer(gsp.Scene(ctx, sc), gsp.sppm_params(sc, **kw))
        r.run(6)
        solo.append(r.image().cpu().numpy())
    scenes = [gsp.Scene(ctx, sc) for sc in scs]
    rs = [gsp.Renderer(s, gsp.sppm_params(sc, **kw)) for s, sc, kw in zip(scenes, scs, kws)]
    b = gsp.Batch(rs)
    b.tune(fused)
    b.run(2)
    gsp.gsp_build_bvh(scenes[0].h, link_sets=1)
    gsp.gsp_scene_set_attributes(scenes[0].h, scs[0].normals, scs[0].texcoords)  # same data, new buffer
    for m, rgb in scs[0].textures.items():
        gsp.gsp_scene_set_texture(scenes[0].h, m, rgb)
    b.run(2)
    gsp.gsp_build_bvh_device(scenes[1].h)
    b.run(2)
    torch.cuda.synchronize()
    for r, want in zip(rs, solo):
        r.sync()
        assert r.state()["passes"] == 6
        assert np.array_equal(r.image().cpu().numpy(), want)
    b.close()


def test_batch_scenes_against_the_oracle(ctx):
    """The four cheapest of the 64-scene batch workload (1-4k triangles, 64^2-128^2 pixels,
    2^18 photon paths per pass, r0 = 0.004 * diagonal, scene ids from their place in the batch)
    rendered by one fused batch (one persistent path launch, a two-pass graph) for 2 passes,
    each image against the FP64 oracle at the plain bar."""
    import oracle as O
    from gpu_util import image_parity
    scs = I.batch_scenes(64, seed=5)
    cost = [sc.ntris * int(sc.camera[0]["width"]) * int(sc.camera[0]["height"]) for sc in scs]
    sel = [int(i) for i in np.argsort(cost)[:4]]
    kw = [dict(photons_per_pass=1 << 18, seed=5 + i, r0_frac=0.004, scene_id=i) for i in sel]
    rs = [gsp.Renderer(gsp.Scene(ctx, scs[i]), gsp.sppm_params(scs[i], **k)) for i, k in zip(sel, kw)]
    b = gsp.Batch(rs)
    b.tune(True)
    b.run(2)
    torch.cuda.synchronize()
    for r, i, k in zip(rs, sel, kw):
        r.sync()
        orc = O.Sppm(scs[i], O.default_params(scs[i], **k))
        orc.run(2)
        assert r.state()["Ne"] == orc.state()["Ne"]
        image_parity(r.image().cpu().numpy(), orc.image())
    b.close()
