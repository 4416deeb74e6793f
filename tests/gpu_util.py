"""Helpers shared by the GPU parity tests."""
import numpy as np


def parity_hits(tri, t, ids, tt, nd, max_excluded=0.02):
    """Closest-hit parity: ids bit-exact on non-degenerate rays, t within 1e-5 relative."""
    sel = nd.astype(bool)
    assert 1.0 - sel.mean() <= max_excluded, f"degenerate fraction {1 - sel.mean():.4f}"
    bad = np.nonzero(sel & (tri != ids))[0]
    assert len(bad) == 0, f"{len(bad)} id mismatches, e.g. {bad[:5]} gpu {tri[bad[:5]]} oracle {ids[bad[:5]]}"
    hit = sel & (ids >= 0)
    rel = np.abs(t[hit].astype(np.float64) - tt[hit]) / np.abs(tt[hit])
    assert rel.max(initial=0) <= 1e-5, f"max rel t error {rel.max():.3g}"
    assert np.all(np.isinf(t[sel & (ids < 0)]))


def image_parity(gpu, ref, rtol=1e-3, min_frac=0.999):
    """Per-pixel relative error <= rtol on at least min_frac of the pixels (floor 1e-6 * mean)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    floor = 1e-6 * max(ref.mean(), 1e-30)
    rel = np.abs(gpu - ref) / np.maximum(np.abs(ref), floor)
    per_pixel = rel.reshape(-1, rel.shape[-1]).max(axis=1)
    frac = float(np.mean(per_pixel <= rtol))
    assert frac >= min_frac, f"only {frac:.5f} of pixels within {rtol} (worst {per_pixel.max():.3g})"
    return frac


def image_parity_boundary(gpu, ref, n_gpu, n_ref, alpha, rtol=1e-3, min_frac=0.998, max_unexplained=2e-4):
    """Full-size form of image_parity for renders whose FP32 photon positions (GPU) and FP64 ones
    (oracle) differ by a few 1e-7 of the scene: a photon that close to a pixel's gather radius
    is counted on one side only, moving that pixel by one photon (N by alpha, the image by
    several percent). At least min_frac of the pixels must be within rtol, and every pixel
    outside it but at most max_unexplained of them must differ by that single photon."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    floor = 1e-6 * max(ref.mean(), 1e-30)
    rel = (np.abs(gpu - ref) / np.maximum(np.abs(ref), floor)).reshape(-1, gpu.shape[-1]).max(axis=1)
    within = rel <= rtol
    one_photon = np.abs(np.asarray(n_gpu, np.float64) - np.asarray(n_ref, np.float64)).reshape(-1) <= alpha * (1 + 1e-4)
    frac = float(within.mean())
    unexplained = float(np.mean(~within & ~one_photon))
    assert frac >= min_frac, f"only {frac:.5f} of pixels within {rtol} (worst {rel.max():.3g})"
    assert unexplained <= max_unexplained, f"{unexplained:.5f} of pixels off by more than one boundary photon"
    return frac, unexplained


# the hash grid's lattice shift (cell = floor(x / h + 0.381966)), the same on both sides
CELL_OFFSET = 0.381966


def _cell_buckets(cells, h, T):
    """Buckets of integer cells [n, 3], through the oracle's hash of their centres."""
    import oracle as O
    centres = ((np.asarray(cells, np.float64) + 0.5 - CELL_OFFSET) * h).astype(np.float32)
    return O.hash_grid(centres, h, T)[0]


def stochastic_uncertain_pixels(deposits_x, hit_x, valid, R, h, T):
    """Pixels whose stochastic-hashing gather may differ between FP32 and FP64 for want of a
    rounding: a deposit within rounding of a cell face (the oracle's near flag) may fall into
    either cell, changing the survivor and the count of both cells' buckets; every pixel whose
    query cells (those overlapping x +- R) hash to such a bucket is uncertain. Returns a bool mask
    over pixels and the number of deposits near a face."""
    import oracle as O
    x = np.asarray(deposits_x, np.float64)
    near = O.hash_grid(x.astype(np.float32), h, T)[3].astype(bool)
    flagged = np.zeros(len(hit_x), bool)
    if not near.any():
        return flagged, 0
    q = x[near] / h + CELL_OFFSET
    tol = 1e-5 + 1e-6 * np.abs(q)  # the near flag's band, in cells
    lo, hi = np.floor(q - tol).astype(np.int64), np.floor(q + tol).astype(np.int64)
    cells = {tuple(int(c) for c in (cx, cy, cz))
             for a, b in zip(lo, hi)
             for cx in range(a[0], b[0] + 1) for cy in range(a[1], b[1] + 1) for cz in range(a[2], b[2] + 1)}
    bad = set(_cell_buckets(np.array(sorted(cells)), h, T).tolist())
    hx = np.asarray(hit_x, np.float64)
    Rv = np.asarray(R, np.float64)[:, None]
    qlo = np.floor((hx - Rv) / h + CELL_OFFSET).astype(np.int64)
    qhi = np.floor((hx + Rv) / h + CELL_OFFSET).astype(np.int64)
    assert np.all(qhi - qlo <= 1), "query ranges of more than two cells per axis (cell edge below 2 R)"
    corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)])
    cand = np.minimum(qlo[:, None, :] + corners[None], qhi[:, None, :])  # [npix, 8, 3]
    b = _cell_buckets(cand.reshape(-1, 3), h, T).reshape(len(hx), 8)
    flagged = np.isin(b, np.array(sorted(bad))).any(axis=1) & np.asarray(valid, bool)
    return flagged, int(near.sum())
