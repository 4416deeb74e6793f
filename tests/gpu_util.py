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
