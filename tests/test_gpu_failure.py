"""Failure detection without a GPU fault: a traversal that reaches its step bound ends early and
records GSP_ERR_TRAVERSAL_LIMIT in the context's status word; the host reads it at the next
sync, and the context keeps working. The bound is lowered through the API (the default one is
only reachable with corrupt links)."""
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


def trace(scene, rays, method):
    tri, t = scene.trace(torch.from_numpy(rays).cuda(), method=method)
    torch.cuda.synchronize()
    return tri.cpu().numpy(), t.cpu().numpy()


@pytest.mark.parametrize("method", ["mtbvh", "stack"])
def test_step_limit_is_reported_and_the_context_recovers(ctx, method):
    sc = I.traversal_sphere(n=24, seed=3)
    rays = I.traversal_rays(64, 32, n_random=2000, seed=51)
    s = gsp.Scene(ctx, sc)
    want = trace(s, rays, method)
    ctx.sync()
    gsp.gsp_scene_set_step_limit(s.h, 3)
    trace(s, rays, method)
    with pytest.raises(gsp.GspError) as e:
        ctx.sync()
    assert e.value.code == -4
    ctx.sync()  # the status word was cleared by the read
    gsp.gsp_scene_set_step_limit(s.h, 0)
    got = trace(s, rays, method)
    ctx.sync()
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1].view(np.int32), want[1].view(np.int32))


def test_step_limit_in_an_sppm_pass(ctx):
    sc = I.cornell_box(width=24, height=24)
    s = gsp.Scene(ctx, sc)
    params = gsp.sppm_params(sc, 4000, seed=2)
    gsp.gsp_scene_set_step_limit(s.h, 2)
    r = gsp.Renderer(s, params)
    r.run(2)
    with pytest.raises(gsp.GspError) as e:
        r.sync()
    assert e.value.code == -4
    gsp.gsp_scene_set_step_limit(s.h, 0)
    a = gsp.Renderer(s, params)
    a.run(2)
    a.sync()
    b = gsp.Renderer(s, params)
    b.run(2)
    b.sync()
    assert np.array_equal(a.image().cpu().numpy(), b.image().cpu().numpy())


def test_step_limit_rejects_negative(ctx):
    s = gsp.Scene(ctx, I.cornell_box(width=8, height=8))
    with pytest.raises(gsp.GspError):
        gsp.gsp_scene_set_step_limit(s.h, -1)


def _cudart():
    """The CUDA runtime this process has loaded (the one the library and torch share)."""
    import ctypes
    rt = ctypes.CDLL("libcudart.so.13")
    rt.cudaMalloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]
    return rt


def test_an_error_left_pending_by_the_caller_is_reported_and_consumed(ctx):
    """An error that the caller's own CUDA work left pending (here a 1 PB allocation request, which
    fails at once and allocates nothing) is reported by the next call that launches work, before it
    launches anything, and consumed: the call after it runs normally."""
    import ctypes
    rt = _cudart()
    ids = torch.arange(256, dtype=torch.int64, device="cuda")
    want = gsp.gsp_rng_fill(ctx.h, 7, 0, 1, 2, ids, 4).cpu()
    out = torch.zeros((256, 4), dtype=torch.float32, device="cuda")  # no torch work while the error is pending
    torch.cuda.synchronize()
    p = ctypes.c_void_p()
    try:
        assert rt.cudaMalloc(ctypes.byref(p), 1 << 50) == 2  # cudaErrorMemoryAllocation
        assert rt.cudaPeekAtLastError() == 2
        with pytest.raises(gsp.GspError) as e:
            gsp.gsp_rng_fill(ctx.h, 7, 0, 1, 2, ids, 4, out=out)
        assert e.value.code == -3 and "pending before the call" in str(e.value)
        assert rt.cudaPeekAtLastError() == 0
    finally:
        rt.cudaGetLastError()
    got = gsp.gsp_rng_fill(ctx.h, 7, 0, 1, 2, ids, 4).cpu()
    assert torch.equal(got, want)


def test_a_failing_call_consumes_the_error_it_reports(ctx):
    """The library's own CUDA failure (an allocation of 1 PB for the bandwidth probe) is returned
    as GSP_ERR_OOM and leaves no error pending for the caller's next CUDA call."""
    rt = _cudart()
    try:
        with pytest.raises(gsp.GspError) as e:
            gsp.gsp_measure_read_bandwidth(ctx.h, 1 << 50, 1)
        assert e.value.code == -2
        assert rt.cudaPeekAtLastError() == 0
    finally:
        rt.cudaGetLastError()
    ids = torch.arange(64, dtype=torch.int64, device="cuda")
    gsp.gsp_rng_fill(ctx.h, 1, 0, 0, 0, ids, 2)
    torch.cuda.synchronize()
