"""GPU path-replay adjoint (gsp_render_grad) against the oracle's FP64 forward-mode gradient,
central finite differences of the GPU forward, and the torch autograd wrapper."""
import numpy as np
import pytest

import oracle as O
from paper_1505_06022_gb300 import gsp, inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KW = dict(photons_per_pass=20000, seed=4, r0_frac=0.02)
PASSES = 3


@pytest.fixture(scope="module")
def ctx():
    c = gsp.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def case():
    sc = I.grad_scene(width=64, height=64, plane_quads=48, sphere_n=8)
    orc = O.Sppm(sc, O.default_params(sc, **KW))
    orc.enable_grad()
    orc.run(PASSES)
    L = orc.image()
    g = L - 0.9 * L.mean() - 0.05 * np.random.default_rng(7).standard_normal(L.shape)
    ga, gl = orc.grad(g)
    return sc, g, ga, gl


def gpu_grad(ctx, sc, g, **tune):
    s = gsp.Scene(ctx, sc)
    r = gsp.Renderer(s, gsp.sppm_params(sc, **KW))
    if tune:
        r.tune(**tune)
    r.enable_grad(PASSES)
    r.run(PASSES)
    before = r.image().clone()
    ga, gl = r.grad(torch.from_numpy(g.astype(np.float32)).cuda())
    after = r.image()
    torch.cuda.synchronize()
    r.sync()
    assert torch.equal(before, after)  # the replay leaves the forward state alone
    return ga.cpu().numpy(), gl.cpu().numpy(), r, s


def assert_per_component(ga, ga_o, rtol=1e-3):
    """Every component within rtol of the FP64 gradient, relative to its own size or, for
    components far below the rest, to 1e-3 of the gradient's norm."""
    floor = 1e-3 * np.linalg.norm(ga_o)
    assert floor > 0
    err = np.abs(ga - ga_o)
    bound = rtol * np.maximum(np.abs(ga_o), floor)
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), f"component {worst}: {ga.flat[worst]:.6g} vs {ga_o.flat[worst]:.6g}"


def test_adjoint_matches_oracle_gradient(ctx, case):
    sc, g, ga_o, gl_o = case
    ga, gl, _, _ = gpu_grad(ctx, sc, g)
    diffuse = sc.mats["type"] == I.DIFFUSE
    assert_per_component(ga[diffuse], ga_o[diffuse])
    assert_per_component(gl, gl_o)
    assert np.all(ga[~diffuse] == 0)


def test_adjoint_matches_gpu_central_differences(ctx, case):
    sc, g, _, _ = case
    ga, gl, r, s = gpu_grad(ctx, sc, g)

    def objective(mats):
        gsp.gsp_scene_set_materials(s.h, mats)
        rr = gsp.Renderer(s, gsp.sppm_params(sc, **KW))
        rr.run(PASSES)
        img = rr.image().cpu().numpy().astype(np.float64)
        return float(np.sum(g * img))

    scale = np.abs(ga).max()
    for m, c in [(1, 0), (6, 2), (13, 1)]:
        mp, mm = sc.mats.copy(), sc.mats.copy()
        mp["albedo"][m, c] += 1e-2
        mm["albedo"][m, c] -= 1e-2
        dh = float(mp["albedo"][m, c]) - float(mm["albedo"][m, c])
        fd = (objective(mp) - objective(mm)) / dh
        assert abs(fd - ga[m, c]) <= 2e-3 * scale, (m, c, fd, ga[m, c])
    gsp.gsp_scene_set_materials(s.h, sc.mats)


def test_autograd_function(ctx):
    sc = I.grad_scene(width=32, height=32, plane_quads=24, sphere_n=4)
    s = gsp.Scene(ctx, sc)
    params = gsp.sppm_params(sc, photons_per_pass=8000, seed=9, r0_frac=0.03)
    em = gsp.emitting_material(sc.mats)
    albedo = torch.tensor(sc.mats["albedo"], device="cuda", requires_grad=True)
    emission = torch.tensor(sc.mats["emission"][em], device="cuda", requires_grad=True)
    target = torch.zeros((32, 32, 3), device="cuda")
    img = gsp.render(albedo, emission, s, params, 2)
    loss = 0.5 * ((img - target) ** 2).sum()
    loss.backward()
    r = gsp.Renderer(s, params)
    r.enable_grad(2)
    r.run(2)
    ga, gl = r.grad((r.image() - target).contiguous())
    torch.testing.assert_close(albedo.grad, ga, rtol=1e-4, atol=1e-6)
    torch.testing.assert_close(emission.grad, gl, rtol=1e-4, atol=1e-6)


def test_call_order_is_checked(ctx):
    sc = I.grad_scene(width=16, height=16, plane_quads=16, sphere_n=3)
    s = gsp.Scene(ctx, sc)
    params = gsp.sppm_params(sc, photons_per_pass=1000, seed=1)
    r = gsp.Renderer(s, params)
    g = torch.zeros((16, 16, 3), device="cuda")
    with pytest.raises(gsp.GspError) as e:
        r.grad(g)  # no enable_grad
    assert e.value.code == -7
    r.run(1)
    with pytest.raises(gsp.GspError):
        r.enable_grad(4)  # after a pass
    r2 = gsp.Renderer(s, params)
    r2.enable_grad(1)
    r2.run(1)
    with pytest.raises(gsp.GspError) as e:
        r2.run(1)  # radius history full
    assert e.value.code == -9


def test_adjoint_does_not_depend_on_execution_settings(ctx, case):
    """Wavefront steps and the path kernel's traversal give the same hits, hence the same
    forward records and the same gradient up to the order of its atomic per-material sums."""
    sc, g, _, _ = case
    base = gpu_grad(ctx, sc, g)
    for tune in (dict(traversal=gsp.TRAVERSAL_STACK), dict(eye_steps=1, photon_steps=2),
                 dict(eye_steps=2, photon_steps=1, traversal=gsp.TRAVERSAL_STACK)):
        ga, gl, _, _ = gpu_grad(ctx, sc, g, **tune)
        np.testing.assert_allclose(ga, base[0], rtol=1e-5, atol=1e-6 * np.abs(base[0]).max())
        np.testing.assert_allclose(gl, base[1], rtol=1e-5, atol=1e-6 * np.abs(base[1]).max())


def test_full_size_gradient_configuration(ctx):
    """The gradient configuration itself: 256x256, 50,770 triangles, 16 diffuse materials + a
    light, 262,144 photon paths per pass, 8 passes, L2 loss against a render at perturbed
    albedos. The adjoint against the FP64 oracle's gradient, and against central differences
    of the GPU forward with h = 1e-3 on three albedo components."""
    sc = I.grad_scene(seed=4)
    kw = dict(photons_per_pass=1 << 18, seed=4, r0_frac=0.004)
    passes = 8
    s = gsp.Scene(ctx, sc)
    tgt = sc.mats.copy()
    tgt["albedo"] = np.clip(tgt["albedo"] * np.random.default_rng(40).uniform(0.8, 1.2, tgt["albedo"].shape), 0.05, 0.95)
    gsp.gsp_scene_set_materials(s.h, tgt)
    rt = gsp.Renderer(s, gsp.sppm_params(sc, **kw))
    rt.run(passes)
    target = rt.image()
    gsp.gsp_scene_set_materials(s.h, sc.mats)
    r = gsp.Renderer(s, gsp.sppm_params(sc, **kw))
    r.enable_grad(passes)
    r.run(passes)
    g = (r.image() - target).contiguous()
    ga, gl = (x.cpu().numpy() for x in r.grad(g))
    g_np = g.cpu().numpy().astype(np.float64)
    orc = O.Sppm(sc, O.default_params(sc, **kw))
    orc.enable_grad()
    orc.run(passes)
    ga_o, gl_o = orc.grad(g_np)
    diffuse = sc.mats["type"] == I.DIFFUSE
    scale = np.abs(ga_o[diffuse]).max()
    assert_per_component(ga[diffuse], ga_o[diffuse])
    assert_per_component(gl, gl_o)

    def objective(mats):
        gsp.gsp_scene_set_materials(s.h, mats)
        rr = gsp.Renderer(s, gsp.sppm_params(sc, **kw))
        rr.run(passes)
        val = float(np.sum(g_np * rr.image().cpu().numpy().astype(np.float64)))
        rr.close()
        return val

    h = 1e-3
    for m, c in [(0, 0), (7, 1), (15, 2)]:
        mp, mm = sc.mats.copy(), sc.mats.copy()
        mp["albedo"][m, c] += h
        mm["albedo"][m, c] -= h
        dh = float(mp["albedo"][m, c]) - float(mm["albedo"][m, c])
        fd = (objective(mp) - objective(mm)) / dh
        assert abs(fd - ga[m, c]) <= 2e-3 * scale, (m, c, fd, ga[m, c])
    gsp.gsp_scene_set_materials(s.h, sc.mats)


def test_gradient_after_batched_passes(ctx):
    """Passes run through a fused batch (two-pass graphs, the pass index read from the device)
    record the same radius history as plain passes, so the replayed gradient is the same."""
    scs = [I.grad_scene(seed=13, width=32, height=24, plane_quads=16, sphere_n=3),
           I.full_scene(seed=14, width=24, height=24, plane_quads=12, sphere_n=3)]
    params = [gsp.sppm_params(scs[0], 6000, seed=3, r0_frac=0.03, scene_id=0),
              gsp.sppm_params(scs[1], 5000, seed=4, r0_frac=0.03, scene_id=1)]
    scenes = [gsp.Scene(ctx, sc) for sc in scs]
    alone = gsp.Renderer(scenes[0], params[0])
    alone.enable_grad(4)
    alone.run(4)
    img = alone.image()
    g = (img - img.mean()).contiguous()
    ga, gl = (x.cpu().numpy() for x in alone.grad(g))
    rs = [gsp.Renderer(s, p) for s, p in zip(scenes, params)]
    rs[0].enable_grad(4)
    b = gsp.Batch(rs)
    b.tune(True)
    b.run(4)
    torch.cuda.synchronize()
    rs[0].sync()
    assert torch.equal(rs[0].image(), img)
    gb, glb = (x.cpu().numpy() for x in rs[0].grad(g))
    np.testing.assert_allclose(gb, ga, rtol=1e-5, atol=1e-6 * np.abs(ga).max())
    np.testing.assert_allclose(glb, gl, rtol=1e-5, atol=1e-6 * np.abs(gl).max())
    with pytest.raises(gsp.GspError):
        b.run(1)  # radius history full
    b.close()
