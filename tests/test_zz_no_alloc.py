"""The allocation-free hash-grid build (for callers that cannot allocate device memory, such as
hosts whose device memory belongs to another allocator, or loops that must not block on
cudaMalloc) gives the same grid as the allocating entry point, on consecutive calls that reuse its
static scratch, up to its largest point count and table size, and allocates nothing.

Kept in a file that pytest collects last, so a run that stops at the first failure has run
every other test before this one."""
import numpy as np
import pytest

from paper_1505_06022_gb300 import gsp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cloud(n, seed):
    rng = np.random.default_rng(seed)
    x = np.concatenate([rng.normal(scale=1.0, size=(n // 2, 3)), rng.normal(scale=0.03, size=(n - n // 2, 3))])
    pos = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    pos[:, :3] = torch.from_numpy(x.astype(np.float32)).cuda()
    return pos


def test_static_build_matches_allocating_build_twice():
    ctx = gsp.Context(0)
    torch.cuda.set_device(0)
    cases = [(cloud(300_001, 1), 0.02, 1 << 19),          # first call: scratch as loaded
             (cloud(gsp.GRID_STATIC_MAX_POINTS, 2), 0.005, 1 << 20)]  # second: reuses it, at the limit
    for pos, h, T in cases:
        n = pos.shape[0]
        want_order, want_starts = gsp.gsp_hash_grid_build(ctx.h, pos, h, T)
        order = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        starts = torch.full((T + 1,), -7, dtype=torch.int32, device="cuda")
        gsp.gsp_hash_grid_build_static(pos, h, T, order, starts)
        torch.cuda.synchronize()
        assert torch.equal(order, want_order)
        assert torch.equal(starts, want_starts)
        assert int(starts[-1]) == n
    ctx.close()


def test_static_build_at_its_largest_sizes_on_a_side_stream_allocates_nothing():
    ctx = gsp.Context(0)
    torch.cuda.set_device(0)
    n, T = gsp.GRID_STATIC_MAX_POINTS, gsp.GRID_STATIC_MAX_TABLE
    pos = cloud(n, 3)
    want_order, want_starts = gsp.gsp_hash_grid_build(ctx.h, pos, 0.003, T)
    order = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    starts = torch.full((T + 1,), -7, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    gsp.gsp_hash_grid_build_static(pos, 0.003, T, order, starts, side)  # loads and looks up once
    side.synchronize()
    assert torch.equal(order, want_order) and torch.equal(starts, want_starts)
    # a second call on the same stream: neither torch nor the driver sees an allocation
    order.fill_(-7)
    starts.fill_(-7)
    torch.cuda.synchronize()
    allocs = torch.cuda.memory_stats()["allocation.all.allocated"]
    free0, _ = torch.cuda.mem_get_info()
    gsp.gsp_hash_grid_build_static(pos, 0.003, T, order, starts, side)
    side.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_stats()["allocation.all.allocated"] == allocs
    assert free1 == free0
    assert torch.equal(order, want_order) and torch.equal(starts, want_starts)
    ctx.close()


def test_static_build_rejects_sizes_beyond_its_scratch():
    n = gsp.GRID_STATIC_MAX_POINTS + 1
    pos = torch.zeros((n, 4), device="cuda")
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    starts = torch.empty(65, dtype=torch.int32, device="cuda")
    with pytest.raises(gsp.GspError, match="static scratch"):
        gsp.gsp_hash_grid_build_static(pos, 0.1, 64, order, starts)
    small = torch.zeros((16, 4), device="cuda")
    big_table = gsp.GRID_STATIC_MAX_TABLE * 2
    # the binding refuses a bucket-start buffer shorter than the table before calling the library
    with pytest.raises(ValueError, match="bstart"):
        gsp.gsp_hash_grid_build_static(small, 0.1, big_table, order[:16], torch.empty(2, dtype=torch.int32, device="cuda"))
    # the library itself refuses the table size (called directly, past the binding's checks)
    import ctypes as C
    rc = gsp.lib().gsp_hash_grid_build_static(C.c_void_p(small.data_ptr()), 16, C.c_float(0.1), big_table,
                                              C.c_void_p(order.data_ptr()), C.c_void_p(starts.data_ptr()),
                                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1 and "static scratch" in gsp.lib().gsp_last_error_message().decode()
