"""Checkpoint / resume: passes after gsp_sppm_load reproduce an uninterrupted run bit for bit
(the PRNG is keyed by the pass index), in both photon modes; mismatched renderers are refused."""
import ctypes as C

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


@pytest.mark.parametrize("photon_mode,hash_mode", [(0, 0), (1, 1)])
def test_resume_is_bit_identical(ctx, tmp_path, photon_mode, hash_mode):
    sc = I.cornell_box(width=40, height=32)
    s = gsp.Scene(ctx, sc)
    params = gsp.sppm_params(sc, 6000, seed=11, photon_mode=photon_mode, hash_mode=hash_mode)
    whole = gsp.Renderer(s, params)
    whole.run(5)
    want = whole.image().cpu().numpy()
    first = gsp.Renderer(s, params)
    first.run(2)
    path = str(tmp_path / "ck.bin")
    first.save(path)
    first.close()
    resumed = gsp.Renderer(s, params)
    resumed.load(path)
    resumed.run(3)
    got = resumed.image().cpu().numpy()
    assert resumed.state()["passes"] == 5
    assert np.array_equal(got, want)


def test_resume_keeps_gradients(ctx, tmp_path):
    sc = I.grad_scene(width=24, height=24, plane_quads=16, sphere_n=3)
    s = gsp.Scene(ctx, sc)
    params = gsp.sppm_params(sc, 3000, seed=12, r0_frac=0.03)
    g = torch.ones((24, 24, 3), device="cuda")
    a = gsp.Renderer(s, params)
    a.enable_grad(4)
    a.run(4)
    want = a.grad(g)
    b = gsp.Renderer(s, params)
    b.enable_grad(4)
    b.run(2)
    b.save(str(tmp_path / "g.bin"))
    c = gsp.Renderer(s, params)
    c.enable_grad(4)
    c.load(str(tmp_path / "g.bin"))
    c.run(2)
    got = c.grad(g)
    torch.testing.assert_close(got[0], want[0], rtol=1e-5, atol=1e-7)
    torch.testing.assert_close(got[1], want[1], rtol=1e-5, atol=1e-7)


def test_mismatched_checkpoint_is_refused(ctx, tmp_path):
    sc = I.cornell_box(width=16, height=16)
    s = gsp.Scene(ctx, sc)
    r = gsp.Renderer(s, gsp.sppm_params(sc, 1000, seed=1))
    r.run(1)
    path = str(tmp_path / "ck.bin")
    r.save(path)
    other = gsp.Renderer(s, gsp.sppm_params(sc, 1000, seed=2))
    with pytest.raises(gsp.GspError) as e:
        other.load(path)
    assert e.value.code == -7
    with pytest.raises(gsp.GspError) as e:
        other.load(str(tmp_path / "missing.bin"))
    assert e.value.code == -8


def test_short_or_padded_checkpoint_leaves_the_renderer_unchanged(ctx, tmp_path):
    sc = I.cornell_box(width=24, height=16)
    s = gsp.Scene(ctx, sc)
    params = gsp.sppm_params(sc, 2000, seed=5)
    src = gsp.Renderer(s, params)
    src.run(3)
    path = tmp_path / "ck.bin"
    src.save(str(path))
    data = path.read_bytes()
    r = gsp.Renderer(s, params)
    r.run(1)
    before = {k: (v.clone() if hasattr(v, "clone") else v) for k, v in r.state().items()}
    # a radius above r0 or a NaN count in the pixel state (a gather would visit cells without bound)
    npix = 24 * 16
    st0 = 8 + 7 * 8 + C.sizeof(gsp.SppmParams)  # magic, header, parameters, then st0 and st1
    big_r = bytearray(data)
    big_r[st0 + npix * 16 + 5 * 16 + 12: st0 + npix * 16 + 5 * 16 + 16] = np.float32(2 * params["r0"]).tobytes()
    nan_n = bytearray(data)
    nan_n[st0 + 7 * 16 + 12: st0 + 7 * 16 + 16] = np.float32("nan").tobytes()
    for bad in (data[: len(data) - 20], data + b"\0" * 16, bytes(big_r), bytes(nan_n)):
        bp = tmp_path / "bad.bin"
        bp.write_bytes(bad)
        with pytest.raises(gsp.GspError) as e:
            r.load(str(bp))
        assert e.value.code == -8
        after = r.state()
        assert after["passes"] == 1
        for k, v in before.items():
            if hasattr(v, "clone"):
                assert torch.equal(after[k], v), k
    r.load(str(path))  # the intact file still loads
    assert r.state()["passes"] == 3
