"""Pins for the specular branches of the oracle's eye and photon paths (Sec. 2: eye paths follow
specular bounces to the first non-specular hit; photons are traced through specular surfaces and
stored at diffuse ones), against closed forms.

* A furnace of emitting walls with albedo 0 holding a mirror sphere (albedo 1) and a glass
  box: every eye path ends on a wall with weight 1, so every pixel is exactly Le (the specular
  depth caps are raised so that no rare long chain of Fresnel reflections is cut). Catches a
  glass that scales the weight by its albedo, a wrong reflection or refraction that loses the
  path, a chain cut short.
* The same furnace with albedo 0.5: lossless specular surfaces leave the uniform radiance field
  uniform, L = Le / (1 - rho). Catches photons lost or gained at the mirror and the glass.
* Camera -> mirror (albedo rho_m) -> emitter: direct / P is exactly rho_m * Le per channel.
  Catches a mirror that forgets its albedo in the eye weight, or a channel mix-up.
* A mirror corridor with 16 and 17 reflections: the eye path follows at most 16 specular
  bounces, so the first sees rho_m^16 Le and the second nothing.
* One photon reflected by a mirror floor onto a ceiling: its stored flux is exactly
  rho_m * pi * A * Le, it is the path's second vertex, and its direction obeys the reflection law.
* One photon through a glass slab: its flux is exactly pi * A * Le whatever the glass albedo.
"""
import numpy as np
import pytest

import oracle as O
from paper_1505_06022_gb300 import inputs as I


def quad_area(sc, mat):
    v = sc.verts.astype(np.float64)
    t = sc.tris[sc.tri_mat == mat]
    return 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1).sum()


def test_specular_furnace_without_albedo_is_exactly_le():
    sc = I.specular_furnace_scene(albedo=0.0, le=1.25, width=16, height=16)
    r = O.Sppm(sc, O.default_params(sc, 2000, r0=0.15, max_eye_depth=256))
    r.run(2)
    st = r.state()
    g = r.last_gather()
    assert g["valid"].all()  # every pixel ends on a wall, through the glass or off the mirror or not
    np.testing.assert_allclose(st["direct"] / st["passes"], 1.25, rtol=1e-12)
    np.testing.assert_allclose(r.image(), 1.25, rtol=1e-12)
    # both specular objects are in view
    d = np.array([[-0.3, -0.05, -0.45], [0.3, 0.05, -0.45]])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.zeros((2, 8), np.float32)
    rays[:, 4:7], rays[:, 7] = d, np.inf
    hit = r.surface(rays)
    assert list(sc.tri_mat[hit["id"]]) == [1, 2]


@pytest.mark.slow
def test_specular_furnace_keeps_the_uniform_field():
    rho = 0.5
    sc = I.specular_furnace_scene(albedo=rho, le=1.0, width=12, height=12)
    r = O.Sppm(sc, O.default_params(sc, 120000, r0=0.15, max_eye_depth=256, max_photon_depth=256))
    r.run(4)
    img = r.image()
    want = 1.0 / (1.0 - rho)
    assert img.mean() == pytest.approx(want, rel=0.01)
    assert np.all(np.abs(img / want - 1) < 0.05)


def test_mirror_scales_the_eye_weight_by_its_albedo():
    rho_m, le = (0.9, 0.6, 0.3), (4.0, 5.0, 6.0)
    sc = I.mirror_view_scene(rho_m, le)
    r = O.Sppm(sc, O.default_params(sc, 16, r0=0.01))
    r.run(3)
    st = r.state()
    want = np.array(rho_m, np.float32).astype(np.float64) * np.array(le, np.float32)
    np.testing.assert_allclose(st["direct"] / 3, np.broadcast_to(want, st["direct"].shape), rtol=1e-12)
    np.testing.assert_allclose(r.image(), np.broadcast_to(want, st["direct"].shape), rtol=1e-12)
    assert not r.last_gather()["valid"].any()  # no diffuse surface: no hit point


@pytest.mark.parametrize("length,reaches", [(16, True), (17, False)])
def test_eye_path_follows_at_most_16_specular_bounces(length, reaches):
    rho_m, le = (0.95, 0.9, 0.85), 3.0
    sc = I.mirror_corridor_scene(length, rho_m, (le,) * 3)
    r = O.Sppm(sc, O.default_params(sc, 4, r0=0.01, max_eye_depth=16))
    r.run(1)
    direct = r.state()["direct"][0, 0]
    if reaches:
        want = np.array(rho_m, np.float32).astype(np.float64) ** 16 * le
        np.testing.assert_allclose(direct, want, rtol=1e-12)
    else:
        assert np.all(direct == 0.0)


def first_deposit(sc, seed):
    params = O.default_params(sc, 1, seed=seed, r0=50.0, rr_continue=1e-30)
    r = O.Sppm(sc, params)
    r.run(1)
    return r.last_photons()


def test_photon_reflected_by_a_mirror_keeps_its_albedo_scaled_flux():
    rho_m, le, light = (0.9, 0.6, 0.3), 5.0, 0.2
    sc = I.photon_mirror_scene(rho_m, le, light, mirror=True)
    phi0 = le * np.pi * quad_area(sc, 2)  # flux of a one-sided Lambertian emitter, pi A Le
    landed = 0
    for seed in range(1, 9):
        ph = first_deposit(sc, seed)
        if len(ph["ids"]) == 0:  # the reflected photon met the back of the light
            continue
        assert len(ph["ids"]) == 1 and ph["ids"][0] == 1  # path k = 0, second vertex
        np.testing.assert_allclose(ph["phi"][0], np.array(rho_m, np.float32).astype(np.float64) * phi0, rtol=1e-12)
        x, din = ph["x"][0], ph["din"][0]
        assert x[1] == pytest.approx(2.0, abs=1e-9) and din[1] > 0
        # reflection law: unfolded at the mirror, the path is a straight line of vertical length
        # 1 + 2 from a point of the light to the deposit
        start = x[[0, 2]] - 3.0 * din[[0, 2]] / din[1]
        assert np.all(np.abs(start) <= light / 2 + 1e-9)
        landed += 1
    assert landed >= 6


def test_photon_through_glass_keeps_its_flux():
    le, light = 5.0, 0.2
    sc = I.photon_mirror_scene(le=le, light=light, mirror=False, glass_albedo=(0.3, 0.3, 0.3))
    phi0 = le * np.pi * quad_area(sc, 2)
    through = 0
    for seed in range(1, 13):
        ph = first_deposit(sc, seed)
        for x, phi, pid in zip(ph["x"], ph["phi"], ph["ids"]):
            np.testing.assert_allclose(phi, phi0, rtol=1e-12)  # glass neither absorbs nor tints
            if x[1] < 0.3:  # landed on the floor below the slab: in at the top, out at the bottom
                assert pid == 2 or pid >= 4
                through += 1 if pid == 2 else 0
    assert through >= 8
