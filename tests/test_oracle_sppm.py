"""Pins for the oracle's SPPM (Sec. 2 three-stage iteration, Sec. 3.3 path regeneration,
Sec. 3.4 stochastic hashing; progressive update of Hachisuka & Jensen 2009).

Each test checks the oracle against something fixed outside it: closed forms of the
progressive recurrence, hand-computable one-photon renders, the white-furnace closed form
L = Le / (1 - rho), brute-force range queries, and sampling identities.
"""
import numpy as np
import pytest

import oracle as O
from paper_1505_06022_gb300 import inputs as I


# ------------------------------------------------------------------------ progressive update
def test_update_recurrence_closed_forms():
    rng = np.random.default_rng(3)
    n, P, alpha, r0 = 64, 12, 0.7, 0.3
    M = rng.poisson(rng.uniform(0, 20, n)[None, :], size=(P, n)).astype(np.float64)
    M[rng.random((P, n)) < 0.2] = 0.0
    Phi = rng.uniform(0, 2, (P, n, 3)) * (M[..., None] > 0)
    N, R, tau = np.zeros(n), np.full(n, r0), np.zeros((n, 3))
    radii = []
    for i in range(P):
        radii.append(R.copy())
        O.sppm_update(alpha, M[i], Phi[i], N, R, tau)
    # N_P = alpha * sum M ;  R_P^2 = r0^2 prod_i (N_i + alpha M_i) / (N_i + M_i)
    Ncum = np.concatenate([np.zeros((1, n)), np.cumsum(alpha * M, axis=0)])[:-1]
    with np.errstate(invalid="ignore", divide="ignore"):
        fac = np.where(M > 0, (Ncum + alpha * M) / (Ncum + M), 1.0)
    np.testing.assert_allclose(N, alpha * M.sum(0), rtol=1e-12)
    np.testing.assert_allclose(R ** 2, r0 ** 2 * np.prod(fac, axis=0), rtol=1e-12)
    # telescoping: tau_P / R_P^2 = sum_i Phi_i / R_i^2
    want = sum(Phi[i] / radii[i][:, None] ** 2 for i in range(P))
    np.testing.assert_allclose(tau / R[:, None] ** 2, want, rtol=1e-12)


def one_photon_scene(rho=0.6, le=5.0, light=0.2):
    """Huge diffuse floor, a small downward light, one-pixel camera looking straight down."""
    S = 500.0
    verts = np.array([[-S, 0, -S], [-S, 0, S], [S, 0, S], [S, 0, -S],
                      [-light / 2, 1, -light / 2], [light / 2, 1, -light / 2],
                      [light / 2, 1, light / 2], [-light / 2, 1, light / 2]], np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]], np.int32)
    mats = np.concatenate([I.material(I.DIFFUSE, (rho,) * 3), I.material(I.EMITTER, emission=(le,) * 3)])
    cam = I.camera((0.3, 2, 0.1), (0.3, 0, 0.1001), (0, 0, 1), 1.0, 1, 1)
    return I.Scene(verts, tris, np.array([0, 0, 1, 1], np.int32), mats, cam)


def test_one_photon_hand_case():
    rho, le, light = 0.6, 5.0, 0.2
    sc = one_photon_scene(rho, le, light)
    r0, alpha = 2000.0, 0.7  # the ball covers the whole floor
    params = O.default_params(sc, 1, r0=r0, alpha=alpha, rr_continue=1e-30)
    rnd = O.Sppm(sc, params)
    phi0 = le * np.pi * light * light  # flux of a Lambertian emitter, pi * A * Le
    rnd.run(1)
    ph = rnd.last_photons()
    assert len(ph["ids"]) == 1 and ph["ids"][0] == 0
    np.testing.assert_allclose(ph["phi"][0], phi0, rtol=1e-6)
    # after one pass: N = alpha, R^2 = alpha r0^2, tau = alpha * Phi_1  ->  L = Phi_1 / (pi r0^2)
    img = rnd.image()[0, 0]
    want1 = (rho / np.pi) * phi0 / (np.pi * r0 ** 2)
    np.testing.assert_allclose(img, want1, rtol=1e-6)
    st = rnd.state()
    np.testing.assert_allclose(st["N"][0, 0], alpha, rtol=1e-7)
    np.testing.assert_allclose(st["R"][0, 0] ** 2, alpha * r0 ** 2, rtol=1e-6)
    # second pass, another single photon: N = 2 alpha, ratio = 2 alpha / (alpha + 1)
    rnd.run(1)
    img2 = rnd.image()[0, 0]
    f = (rho / np.pi) * phi0
    want2 = (alpha * f + f) / (np.pi * alpha * r0 ** 2 * 2)
    np.testing.assert_allclose(img2, want2, rtol=1e-6)


@pytest.fixture(scope="module")
def cornell_pass():
    sc = I.cornell_box(width=32, height=32)
    params = O.default_params(sc, 4096)
    rnd = O.Sppm(sc, params)
    rnd.run(3)
    return sc, params, rnd


def test_first_deposit_flux_and_direct_term(cornell_pass):
    sc, params, rnd = cornell_pass
    ph = rnd.last_photons()
    first = ph["ids"] % 32 == 0
    assert first.sum() > 1000
    le = float(sc.mats["emission"][-1][0])
    np.testing.assert_allclose(ph["phi"][first], le * np.pi * 0.25 * 0.25, rtol=1e-6)
    st = rnd.state()
    # pixels whose jittered rays always land on the light see exactly Le per pass
    assert np.max(st["direct"]) / st["passes"] == pytest.approx(le, rel=1e-12)
    assert st["Ne"] == 3 * 4096


def test_exact_gather_is_the_brute_force_range_query(cornell_pass):
    sc, params, _ = cornell_pass
    rnd = O.Sppm(sc, params)
    rnd.run(1)  # the first pass gathers with R = r0 everywhere
    ph = rnd.last_photons()
    g = rnd.last_gather()
    r0 = params["r0"]
    albedo = sc.mats["albedo"].astype(np.float64)
    valid = np.nonzero(g["valid"])[0]
    assert len(valid) > 900
    for p in valid:
        d2 = np.sum((ph["x"] - g["x"][p]) ** 2, axis=1)
        sel = (d2 < r0 * r0) & (ph["din"] @ g["n"][p] < 0)
        assert g["M"][p] == sel.sum()
        want = (g["w"][p] * albedo[g["mat"][p]] / np.pi) * ph["phi"][sel].sum(axis=0)
        np.testing.assert_allclose(g["Phi"][p], want, rtol=1e-10, atol=1e-300)


def test_exact_gather_does_not_depend_on_cell_size():
    sc = I.cornell_box(width=24, height=24)
    base = O.default_params(sc, 2048)
    imgs = []
    for f in (2.0, 1.0, 0.5, 4.0):
        p = dict(base, cell_h=float(np.float32(f * base["r0"])))
        r = O.Sppm(sc, p)
        r.run(2)
        imgs.append(r.image())
    for im in imgs[1:]:
        assert np.array_equal(im, imgs[0])


def test_stochastic_hashing_is_unbiased():
    # After one pass L = Phi_1 / (pi r0^2 N_e) in both modes, so the means over seeds agree.
    sc = I.cornell_box(width=12, height=12)
    K = 48
    out = {0: [], 1: []}
    for mode in (0, 1):
        for seed in range(K):
            p = O.default_params(sc, 2048, seed=100 + seed, hash_mode=mode)
            r = O.Sppm(sc, p)
            r.run(1)
            out[mode].append(r.image().mean(axis=2))
    a, b = np.array(out[0]), np.array(out[1])
    diff = b.mean(0) - a.mean(0)
    se = np.sqrt(a.var(0, ddof=1) / K + b.var(0, ddof=1) / K) + 1e-12
    z = diff / se
    assert abs(diff.mean()) < 3 * np.sqrt(np.mean(se ** 2) / z.size) * 3
    assert np.mean(np.abs(z) > 3.5) < 0.02
    assert b.std(0).mean() > a.std(0).mean()  # hashing adds variance, never removes it


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.8])
def test_white_furnace(rho):
    sc = I.furnace_scene(n=32, albedo=rho, le=1.0, width=12, height=12)
    p = O.default_params(sc, 120000, r0=0.15)
    r = O.Sppm(sc, p)
    r.run(4)
    img = r.image()
    assert img.mean() == pytest.approx(1.0 / (1.0 - rho), rel=0.01)
    assert np.all(np.abs(img / (1.0 / (1.0 - rho)) - 1) < 0.05)


def test_regeneration_mode_bookkeeping():
    sc = I.cornell_box(width=16, height=16)
    np_ = 3000
    p = O.default_params(sc, np_, photon_mode=1)
    r = O.Sppm(sc, p)
    r.run(1)
    assert r.state()["Ne"] == np_  # every thread starts a path in the first pass
    ph = r.last_photons()
    assert len(np.unique(ph["ids"])) == len(ph["ids"]) and ph["ids"].max() < np_
    ne_prev = np_
    for _ in range(5):
        r.run(1)
        ne = r.state()["Ne"]
        new = ne - ne_prev
        assert 0 < new < np_  # only finished paths restart
        assert len(r.last_photons()["ids"]) <= np_
        ne_prev = ne


def test_regeneration_and_full_paths_converge_to_the_same_image():
    # Compare the photon-density part tau / (pi R^2 N_e): the direct term of a tiny image is
    # a handful of jitter samples of the light and says nothing about the photon modes.
    # Regeneration counts paths still in flight in N_e, a bias that shrinks with passes.
    sc = I.cornell_box(width=8, height=8)

    def indirect(mode, passes):
        r = O.Sppm(sc, O.default_params(sc, 20000, photon_mode=mode))
        r.run(passes)
        st = r.state()
        return float((st["tau"].sum(-1) / (np.pi * st["R"] ** 2)).mean() / st["Ne"])

    full = indirect(0, 8)
    early, late = indirect(1, 16), indirect(1, 160)
    assert abs(late / full - 1) < 0.03
    assert abs(late / full - 1) < abs(early / full - 1)


# ------------------------------------------------------------------------ sampling identities
def test_cosine_directions():
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    g = (np.arange(64) + 0.5) / 64
    d = np.array([O.cosine_dir(n, np.float32(a), np.float32(b)) for a in g for b in g])
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, rtol=1e-12)
    c = d @ n
    assert np.all(c > 0)
    assert c.mean() == pytest.approx(2 / 3, abs=2e-3)     # E[cos] for a cosine density
    assert (c ** 2).mean() == pytest.approx(1 / 2, abs=2e-3)
    assert np.abs(d.mean(0) - c.mean() * n).max() < 2e-3  # no tangential bias


def test_dielectric_fresnel_and_snell():
    nrm = np.array([0.0, 0.0, 1.0])
    us = (np.arange(100000) + 0.5) / 100000
    # normal incidence: F = ((1 - 1.5) / (1 + 1.5))^2 = 0.04
    dn = np.array([0.0, 0.0, -1.0])
    refl = np.mean([O.dielectric(dn, nrm, 1.5, np.float32(u))[2] > 0 for u in us[::10]])
    assert refl == pytest.approx(0.04, abs=2e-4)
    # Brewster's angle: p-polarised reflectance vanishes, F = R_s / 2 = 0.1479 / 2
    th = np.arctan(1.5)
    d = np.array([np.sin(th), 0.0, -np.cos(th)])
    refl = np.mean([O.dielectric(d, nrm, 1.5, np.float32(u))[2] > 0 for u in us[::10]])
    assert refl == pytest.approx(0.1479 / 2, abs=3e-4)
    # Snell: sin(theta_t) = sin(theta_i) / 1.5 for the refracted branch
    t = O.dielectric(d, nrm, 1.5, np.float32(0.999))
    assert t[2] < 0 and np.hypot(t[0], t[1]) == pytest.approx(np.sin(th) / 1.5, rel=1e-12)
    # from inside beyond the critical angle: total internal reflection for every u
    th2 = np.arcsin(1 / 1.5) + 0.05
    d2 = np.array([np.sin(th2), 0.0, np.cos(th2)])  # travelling outwards through the back
    assert all(O.dielectric(d2, nrm, 1.5, np.float32(u))[2] < 0 for u in (0.0, 0.5, 0.999))
