"""GPU exact hash grid (the exact deposit's index) against the oracle, bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_1505_06022_gb300 import gsp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def points(n, seed, spread=1.5):
    rng = np.random.default_rng(seed)
    x = np.concatenate([rng.normal(scale=spread, size=(n // 2, 3)),        # diffuse cloud
                        rng.normal(scale=0.02, size=(n - n // 2, 3))])      # a dense caustic-like clump
    return x.astype(np.float32)


@pytest.mark.parametrize("n,T,h", [(0, 64, 0.1), (1, 1, 0.1), (777, 256, 0.05), (200_003, 1 << 18, 0.01),
                                   (1_000_000, 1 << 21, 0.004)])
def test_hash_grid_matches_oracle(n, T, h):
    x = points(n, seed=n + 3)
    _, _, _, near = O.hash_grid(x, h, T)
    x = x[near == 0]  # coordinates on a cell face may round to either cell; keep the rest
    b, order, starts, _ = O.hash_grid(x, h, T)
    ctx = gsp.Context(0)
    pos = torch.zeros((len(x), 4), dtype=torch.float32, device="cuda")
    pos[:, :3] = torch.from_numpy(x).cuda()
    got_order, got_starts = gsp.gsp_hash_grid_build(ctx.h, pos, h, T)
    torch.cuda.synchronize()
    ctx.sync()
    np.testing.assert_array_equal(got_order.cpu().numpy().view(np.uint32), order)
    np.testing.assert_array_equal(got_starts.cpu().numpy().view(np.uint32), starts)
    ctx.close()


def test_rejects_bad_arguments():
    ctx = gsp.Context(0)
    pos = torch.zeros((8, 4), device="cuda")
    for h, T in [(0.0, 64), (0.1, 63), (0.1, 0), (float("nan"), 64)]:
        with pytest.raises(gsp.GspError):
            gsp.gsp_hash_grid_build(ctx.h, pos, h, T)
    ctx.close()
