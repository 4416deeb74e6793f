"""Work counters of an SPPM pass (gsp_sppm_count_work): what the roofline of a pass is computed
from. Counting leaves the estimate unchanged, is deterministic, agrees with quantities known
independently (one primary ray per pixel, the deposits the pass reports, the oracle's hit
points), and refuses the settings it does not cover."""
import numpy as np
import pytest

import oracle as O
from paper_1505_06022_gb300 import gsp, inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gsp.Context(0)
    yield c
    c.close()


def test_counting_leaves_the_image_unchanged_and_repeats(ctx):
    sc = I.cornell_box(seed=1)
    s = gsp.Scene(ctx, sc)
    params = gsp.sppm_params(sc, 16384, seed=1)
    plain = gsp.Renderer(s, params)
    plain.run(4)
    want = plain.image()
    counts = []
    for _ in range(2):
        r = gsp.Renderer(s, params)
        r.count_work(True)
        r.run(4)
        got = r.image()
        counts.append(r.count_work(False))
        assert torch.equal(got, want)
        r.close()
    # rays, deposits and gathers repeat exactly; box and triangle tests within 0.1 % (which lanes
    # share a warp decides when a postponed leaf is tested, and so how soon the best t culls)
    c, c2 = counts
    for k in ("eye_rays", "photon_rays", "deposits", "hit_points", "photons_scanned"):
        assert c[k] == c2[k], k
    for k in ("node_visits", "tri_tests"):
        assert abs(c[k] - c2[k]) <= 1e-3 * c[k], k
    # the Cornell box has no specular surface: exactly one eye ray per pixel and pass
    assert c["eye_rays"] == 4 * 64 * 64
    assert c["deposits"] <= c["photon_rays"] <= 4 * 16384 * 32
    assert c["node_visits"] >= c["eye_rays"] + c["photon_rays"]
    assert c["tri_tests"] > 0 and c["photons_scanned"] > 0 and c["hit_points_scanned"] == 0
    # counting was switched off: nothing more is counted
    r = gsp.Renderer(s, params)
    r.run(1)
    assert all(v == 0 for v in r.count_work(False).values())


@pytest.mark.parametrize("hash_mode", [gsp.EXACT, gsp.STOCHASTIC])
def test_one_pass_counts_against_independent_quantities(ctx, hash_mode):
    sc = I.cornell_box(seed=1)
    s = gsp.Scene(ctx, sc)
    kw = dict(photons_per_pass=16384, seed=3, hash_mode=hash_mode)
    r = gsp.Renderer(s, gsp.sppm_params(sc, **kw))
    r.count_work(True)
    r.run(1)
    c = r.count_work(False)
    assert c["deposits"] == len(r.last_deposits())
    orc = O.Sppm(sc, O.default_params(sc, **kw))
    orc.run(1)
    valid = int(orc.last_gather()["valid"].sum())
    assert abs(c["hit_points"] - valid) <= 2  # a grazing eye ray may end on the other side
    if hash_mode == gsp.EXACT:
        assert c["photons_scanned"] >= c["deposits"] // 8  # every hit point reads its cells' photons
    else:
        assert c["photons_scanned"] <= 27 * c["hit_points"]  # at most one survivor per query bucket


def test_gradient_counts_the_replay_and_the_adjoint_gather(ctx):
    sc = I.grad_scene(width=32, height=32, plane_quads=16, sphere_n=3)
    s = gsp.Scene(ctx, sc)
    r = gsp.Renderer(s, gsp.sppm_params(sc, 4000, seed=2, r0_frac=0.03))
    r.enable_grad(2)
    r.count_work(True)
    r.run(2)
    img = r.image()
    fwd = r.count_work(True)
    r.grad(torch.ones_like(img))
    bwd = r.count_work(False)
    # the replay traces the same rays and deposits the same photons as the forward passes
    for k in ("eye_rays", "photon_rays", "deposits"):
        assert bwd[k] == fwd[k], k
    for k in ("node_visits", "tri_tests"):
        assert abs(bwd[k] - fwd[k]) <= 1e-3 * fwd[k], k
    assert bwd["hit_points_scanned"] > 0 and fwd["hit_points_scanned"] == 0


def test_counting_refuses_what_it_does_not_cover(ctx):
    sc = I.cornell_box(width=16, height=16)
    s = gsp.Scene(ctx, sc)
    params = gsp.sppm_params(sc, 1000, seed=1)
    r = gsp.Renderer(s, params)
    r.tune(eye_steps=1)
    with pytest.raises(gsp.GspError) as e:
        r.count_work(True)
    assert e.value.code == -7  # GSP_ERR_BAD_STATE
    r.tune(eye_steps=0)
    r.count_work(True)
    for kw in (dict(photon_steps=1), dict(traversal=gsp.TRAVERSAL_STACK)):
        with pytest.raises(gsp.GspError):
            r.tune(**kw)
    with pytest.raises(gsp.GspError):
        r.autotune(trial_passes=1)
    other = gsp.Renderer(gsp.Scene(ctx, sc), params)  # a batch's renderers have scenes of their own
    b = gsp.Batch([r, other])
    with pytest.raises(gsp.GspError):
        b.run(1)
    r.count_work(False)
    b.run(1)  # counting off: the batch runs
    b.close()
