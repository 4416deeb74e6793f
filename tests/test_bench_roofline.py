"""The benchmark's roofline blocks, recomputed by hand from the work model they state: a
closest-hit query costs 32 bytes per node box test, 48 per triangle test and 40 per ray (in and
out), and 12 and 30 FP32 operations per box and triangle test; an SPPM pass adds 3 x 32 bytes per
deposit, 32 bytes per photon a gather reads and 72 bytes per pixel (the adjoint 20 bytes per hit
point it reads and 96 per pixel); the FP32 peak is SMs x 128 lanes x 2 (FMA) x the maximum SM
clock. No GPU: the helpers are plain arithmetic."""
import pytest

import bench

PEAKS = {"hbm_gbs": 6789.0, "sm_max_mhz": 2070.0}
TIERS = {"l2_peak_gbs": 19412.5}


def test_traversal_roofline_by_hand():
    v_node, v_tri, n, ms = 18.853, 1.827, 4_194_304, 0.745
    r = bench.traversal_roofline(v_node, v_tri, n, ms, 0.7596, 152, PEAKS, TIERS)
    bytes_ray = 32 * 18.853 + 48 * 1.827 + 40  # 730.992
    achieved = bytes_ray * n / (ms * 1e-3) / 1e9  # GB/s
    assert r["algorithmic_bytes_per_ray"] == pytest.approx(731.0, abs=0.05)
    assert r["algorithmic_bytes_per_launch"] == round(bytes_ray * n)
    assert r["achieved"] == pytest.approx(achieved, abs=0.05)
    assert r["frac"] == pytest.approx(achieved / 6789.0, abs=1e-4)
    assert r["peak"] == 6789.0 and r["unit"] == "GB/s"
    assert r["l2"]["frac"] == pytest.approx(achieved / 19412.5, abs=1e-4)
    fp32_peak = 152 * 128 * 2 * 2070e6 / 1e12  # 80.55 TFLOP/s
    flops_ray = 12 * 18.853 + 30 * 1.827
    assert r["fp32"]["peak"] == pytest.approx(fp32_peak, abs=0.01)
    assert r["fp32"]["frac"] == pytest.approx(flops_ray * n / (ms * 1e-3) / 1e12 / fp32_peak, abs=1e-4)
    # the byte term binds: bytes / HBM peak is far above flops / FP32 peak
    assert r["bound"] == "hbm"
    assert r["roofline_ms"] == pytest.approx(bytes_ray * n / 6789e9 * 1e3, abs=1e-4)
    assert r["kernel_ms"] == 0.745 and r["call_ms"] == 0.7596


def test_traversal_roofline_without_measured_peaks_uses_the_fallback():
    r = bench.traversal_roofline(18.0, 2.0, 1 << 20, 0.2, 0.21, 152, None, TIERS)
    assert r["peak"] == 6800.0 and "fallback" in r["peak_source"]
    assert r["fp32"]["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12, abs=0.01)


def test_sppm_work_model_by_hand():
    c = {"eye_rays": 1000, "photon_rays": 5000, "node_visits": 100_000, "tri_tests": 9000, "deposits": 700,
         "photons_scanned": 40_000, "hit_points": 900, "hit_points_scanned": 3000}
    nbytes, flops, parts = bench.sppm_work(c, 64 * 64, 4)
    assert parts == {"traversal": 32 * 100_000 + 48 * 9000 + 40 * 6000,
                     "deposit": 96 * 700,
                     "gather": 32 * 40_000 + 72 * 4096 * 4}
    assert nbytes == sum(parts.values())
    assert flops == 12 * 100_000 + 30 * 9000
    nb2, _, p2 = bench.sppm_work(c, 4096, 4, adjoint=True)
    assert p2["adjoint_gather"] == 20 * 3000 + 96 * 4096 * 4 and nb2 == nbytes + p2["adjoint_gather"]
    rl = {"peaks": PEAKS, "tiers": TIERS, "sm_count": 152}
    w = bench.work_roofline(nbytes, flops, 1e-3, rl)
    assert w["achieved"] == pytest.approx(nbytes / 1e-3 / 1e9, abs=0.05)
    assert w["frac"] == pytest.approx(nbytes / 1e-3 / 1e9 / 6789.0, abs=1e-4)
    assert w["l2"]["frac"] == pytest.approx(nbytes / 1e-3 / 1e9 / 19412.5, abs=1e-4)
    assert w["algorithmic_bytes"] == nbytes and w["flops"] == flops
