"""Pins for the oracle's gradient of an L2 image loss (forward-mode derivatives through the
photon paths and the progressive update): central finite differences of the oracle's own FP64
forward, and the closed form of the emission gradient (one light: the image is linear in Le)."""
import copy

import numpy as np
import pytest

import oracle as O
from paper_1505_06022_gb300 import inputs as I


@pytest.fixture(scope="module")
def setup():
    sc = I.grad_scene(width=24, height=24, plane_quads=24, sphere_n=4)
    kw = dict(photons_per_pass=3000, seed=4, r0_frac=0.02)
    passes = 2

    def render(mats):
        s2 = copy.copy(sc)
        s2.mats = mats
        r = O.Sppm(s2, O.default_params(s2, **kw))
        r.run(passes)
        return r.image()

    target = sc.mats.copy()
    target["albedo"] = np.clip(target["albedo"] * np.random.default_rng(40).uniform(0.8, 1.2, target["albedo"].shape),
                               0.05, 0.95)
    T = render(target)
    r = O.Sppm(sc, O.default_params(sc, **kw))
    r.enable_grad()
    r.run(passes)
    L = r.image()
    ga, gl = r.grad(L - T)
    return sc, render, T, L, ga, gl


def test_albedo_gradient_matches_central_differences(setup):
    sc, render, T, L, ga, gl = setup
    loss = lambda img: 0.5 * np.sum((img - T) ** 2)
    scale = np.abs(ga).max()
    assert scale > 0
    for m, c in [(0, 0), (3, 1), (7, 2), (12, 0), (15, 1)]:
        mp, mm = sc.mats.copy(), sc.mats.copy()
        mp["albedo"][m, c] += 1e-3
        mm["albedo"][m, c] -= 1e-3
        dh = float(mp["albedo"][m, c]) - float(mm["albedo"][m, c])  # float32-rounded step
        fd = (loss(render(mp)) - loss(render(mm))) / dh
        assert abs(fd - ga[m, c]) <= 1e-5 * scale, (m, c, fd, ga[m, c])
    assert np.all(ga[16] == 0)  # the emitter's albedo enters nothing


def test_emission_gradient_matches_closed_form_and_differences(setup):
    sc, render, T, L, ga, gl = setup
    le = sc.mats["emission"][16].astype(np.float64)
    g = L - T
    np.testing.assert_allclose(gl, (g * L).sum(axis=(0, 1)) / le, rtol=1e-10)
    loss = lambda img: 0.5 * np.sum((img - T) ** 2)
    mp, mm = sc.mats.copy(), sc.mats.copy()
    mp["emission"][16, 1] += 1e-2
    mm["emission"][16, 1] -= 1e-2
    dh = float(mp["emission"][16, 1]) - float(mm["emission"][16, 1])
    assert (loss(render(mp)) - loss(render(mm))) / dh == pytest.approx(gl[1], rel=1e-6)


def test_gradient_mode_does_not_change_the_image():
    sc = I.grad_scene(width=16, height=16, plane_quads=16, sphere_n=3)
    kw = dict(photons_per_pass=2000, seed=5, r0_frac=0.02)
    a = O.Sppm(sc, O.default_params(sc, **kw))
    a.run(2)
    b = O.Sppm(sc, O.default_params(sc, **kw))
    b.enable_grad()
    b.run(2)
    assert np.array_equal(a.image(), b.image())
