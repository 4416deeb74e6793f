#!/usr/bin/env python3
"""Benchmark: closest-hit ray casting through the multiple-threaded BVH, plus the SPPM workloads.

Default workload (one line of JSON on rank 0):
  * step = one gsp_trace_closest_hit call over 4,194,304 rays (2,097,152 coherent pinhole rays
    + 2,097,152 uniform random rays) against a 1,003,520-triangle displaced icosphere
    (SAH BVH, 16 bins, six hit/miss link sets). metric: closest-hit Mrays/s.
  * "e2e": the same rays through gsp_trace_closest_hit_host from pinned host memory (the
    host->device transfer of the rays and the device->host copy of the hits inside the timed
    region).
  * "traversal_fig4": MTBVH vs TBVH vs stack traversal (Fig. 4) and the device BVH build.
  * "sppm_512": SPPM passes/s at 512x512 on a 247,234-triangle scene with 1M photon paths/pass
    (a 64-pass render; default and autotuned settings).
  * "sppm_512_shaded": the 512x512 render with per-vertex normals, texture coordinates and albedo
    textures, against the same geometry without them.
  * "grad_256": backward/forward time of the path-replay adjoint (256x256, 8 passes).
  * "batch_64": 64 scenes as one graph per pass vs one renderer after another.
  * "sppm_modes": the paper's photon-pass / hashing variants at equal image error.
Multi-GPU: every rank casts its own 4M rays (independent work, no collective on the data
path); the value is all rays of all ranks over the slowest rank's time.

--impl reference times the CPU oracle (FP64, all host cores) on a bounded sample of the same
workload and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Work model of a closest-hit query (the measurement plan's cost model): per node visit a 32-byte
# node and 12 FP32 operations (the slab test), per triangle test a 48-byte triangle and 30 FP32
# operations (Moller-Trumbore), per ray a 32-byte ray in and an 8-byte hit out. Roofline time =
# max(bytes / memory bandwidth, flops / FP32 peak), FP32 peak = SMs x 128 lanes x 2 x clock.
FLOPS_PER_NODE = 12
FLOPS_PER_TRI = 30
BYTES_PER_NODE = 32
BYTES_PER_TRI = 48
BYTES_PER_RAY_IO = 32 + 8
FALLBACK_HBM_GBS = 6800.0


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks and throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_ranks(world, dev):
    """One process per GPU: NCCL between GPUs, gloo for host-only ranks. None when world == 1."""
    if world <= 1:
        return None
    import torch.distributed as dist
    if dev.type == "cuda":
        dist.init_process_group("nccl", device_id=dev)
    else:
        dist.init_process_group("gloo")
    return dist


def max_over_ranks(x, pg, dev):
    """The largest x over all ranks: the slowest replica sets the job's time."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_mrays(world, rays_per_rank, ms_per_step):
    """Whole-job throughput: every replica traces its own batch each step."""
    return world * rays_per_rank / (ms_per_step / 1000.0) / 1e6


def traversal_workload():
    from paper_1505_06022_gb300 import inputs as I
    sc = I.traversal_sphere(n=224, seed=2)
    rays = I.traversal_rays(2048, 1024, seed=2)
    return sc, rays


def stratified(n, k, seed=11):
    rng = np.random.default_rng(seed)
    half = n // 2
    return np.sort(np.concatenate([rng.choice(half, k // 2, replace=False),
                                   half + rng.choice(n - half, k - k // 2, replace=False)]))


def cpu_oracle_rays(sc, rays, sample_rays, steps=1, warmup=0, min_seconds=0.0):
    """Times the FP64 oracle's closest-hit query on `sample_rays` rays per step, all cores;
    with min_seconds, repeats the step until that much time has passed. Returns (Mrays/s,
    cores, seconds, steps run)."""
    import oracle as O
    mesh = O.Mesh(sc.verts, sc.tris)
    idx = stratified(len(rays), sample_rays) if sample_rays < len(rays) else np.arange(len(rays))
    sub = np.ascontiguousarray(rays[idx])
    cores = O.nthreads_default()
    for _ in range(warmup):
        mesh.closest_hit(sub, classify=False, nthreads=cores)
    t0 = time.perf_counter()
    done = 0
    while done < steps or time.perf_counter() - t0 < min_seconds:
        mesh.closest_hit(sub, classify=False, nthreads=cores)
        done += 1
    dt = time.perf_counter() - t0
    return len(sub) * done / dt / 1e6, cores, dt, done


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    sc, rays = traversal_workload()
    sample = args.ref_rays
    mrays, cores, dt, _ = cpu_oracle_rays(sc, rays, sample, steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": "closest-hit Mrays/s", "value": round(mrays, 4), "unit": "Mrays/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1000 * dt / args.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "closest-hit traversal: 1,003,520-triangle displaced icosphere, 4,194,304 rays "
                               "(half coherent pinhole, half uniform random)",
                   "sample_rays_per_step": sample, "parallelism": "host threads"},
        "cpu_baseline": {"value": round(mrays, 4), "unit": "Mrays/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} stratified rays of the 4,194,304 per step, FP64 oracle BVH"},
        "e2e": {"value": round(mrays, 4), "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, world, rank, local):
    import torch
    from paper_1505_06022_gb300 import gsp, inputs as I

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = init_ranks(world, dev)
    gsp.lib()
    ctx = gsp.Context(local)
    sc, rays_h = traversal_workload()
    scene = gsp.Scene(ctx, sc, bins=16, leaf_threshold=4, max_leaf=7, link_sets=6)
    n = len(rays_h)
    rays = torch.from_numpy(rays_h).to(dev)
    tri = torch.empty(n, dtype=torch.int32, device=dev)
    tt = torch.empty(n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        gsp.gsp_trace_closest_hit(scene.h, rays, tri, tt, None, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.sync()
    # the library brackets each timed step's k_trace launch with a pair of events made here
    gsp.gsp_trace_time_launches(scene.h, args.steps)
    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    ev[1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    ms_total = max_over_ranks(ev[0].elapsed_time(ev[1]), pg, dev)
    ctx.sync()
    ms_step = ms_total / args.steps
    launch_ms = gsp.gsp_trace_launch_times(scene.h, args.steps)
    gsp.gsp_trace_time_launches(scene.h, 0)
    assert len(launch_ms) == args.steps
    ms_kernel = max_over_ranks(float(launch_ms.mean()), pg, dev)
    mrays = job_mrays(world, n, ms_step)

    # ---- end to end through the C ABI with host buffers: each step copies the rays from pinned
    # host memory to the device, traces them and copies ids and t back (one synchronous call) ----
    rays_pin = torch.from_numpy(rays_h).pin_memory()
    tri_pin = torch.empty(n, dtype=torch.int32).pin_memory()
    t_pin = torch.empty(n, dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 50))

    def e2e_step():
        gsp.gsp_trace_closest_hit_host(scene.h, rays_pin, tri_pin, t_pin)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(1000.0 * (time.perf_counter() - t0) / e2e_steps, pg, dev)
    # correctness of the timed results on a few rays (host walk of the same BVH)
    chk = stratified(n, 4096, seed=5)
    htri, _, vis, tests = scene.host_walk(rays_h[chk])
    agree = float(np.mean(htri == tri_pin.numpy()[chk]))

    # ---- roofline of the traversal: max(bytes / bandwidth, flops / FP32 peak) ----
    peaks = load_peaks()
    tiers = measure_tiers(ctx)
    wk = stratified(n, 65536, seed=6)
    _, _, visw, testw = scene.host_walk(rays_h[wk])
    v_node, v_tri = float(visw.mean()), float(testw.mean())
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    roofline = traversal_roofline(v_node, v_tri, n, ms_kernel, ms_step, sm_count, peaks, tiers)
    rl = {"peaks": peaks, "tiers": tiers, "sm_count": sm_count}
    traffic_file = os.path.join(ROOT, "profiles", "trace_traffic.json")
    if os.path.exists(traffic_file):
        try:
            tf = json.load(open(traffic_file))
            if tf.get("kernel_digest") == gsp_kernel_digest():
                roofline["traffic"] = tf.get("dram_bytes_per_launch")
        except Exception:
            pass

    # ---- Fig. 4's traversal comparison, SPPM pass at 512x512, the gradient workload, the batch ----
    fig4 = bench_traversals(args, ctx, dev, stream, sc, scene, rays) if not args.skip_fig4 else None
    cornell = bench_cornell(args, ctx, dev, stream, with_cpu(args, world, rank)) if not args.skip_sppm else None
    sppm = bench_sppm(args, ctx, dev, stream, pg, rl) if not args.skip_sppm else None
    shaded = bench_shaded(args, ctx, dev, stream, pg) if not (args.skip_sppm or args.skip_shaded) else None
    grad = bench_grad(args, ctx, dev, stream, rl) if not args.skip_grad else None
    batch = bench_batch(args, ctx, dev, stream, rl) if not args.skip_batch else None
    modes = bench_modes(args, ctx, dev, stream) if not args.skip_modes else None

    # ---- CPU baseline: the oracle on the same workload ----
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        mr, cores, dt, reps = cpu_oracle_rays(sc, rays_h, n, warmup=1, min_seconds=10.0)
        cpu = {"value": round(mr, 4), "unit": "Mrays/s", "cores": cores, "kind": "oracle",
               "sample": f"the whole 4,194,304-ray batch (half coherent, half random) traced {reps} times by "
                         f"the FP64 oracle BVH, {dt:.1f} s"}
    if rank == 0:
        line = {
            "metric": "closest-hit Mrays/s", "value": round(mrays, 2), "unit": "Mrays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "closest-hit traversal: 1,003,520-triangle displaced icosphere (SAH 16 bins, "
                                   "6 link sets), 4,194,304 rays (2,097,152 coherent pinhole + 2,097,152 "
                                   "uniform random)", "rays_per_rank": n, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (rays 134 MB per step); BVH resident",
                       "bvh": scene.stats},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": round(job_mrays(world, n, e2e_ms), 2), "unit": "Mrays/s",
                    "h2d_bytes_per_step": int(rays_h.nbytes), "d2h_bytes_per_step": int(n * 8)},
            "gpu_launches": 3 * args.steps,
            "clocks": clk,
            "wall_s_timed": round(wall, 4),
            "check": {"host_walk_agreement": round(agree, 5)},
            "traversal_fig4": fig4,
            "sppm_cornell_64": cornell,
            "sppm_512": sppm,
            "sppm_512_shaded": shaded,
            "grad_256": grad,
            "batch_64": batch,
            "sppm_modes": modes,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


def measure_tiers(ctx):
    """Read bandwidth of L2 (streaming over 32 and 48 MB buffers, resident after a warm-up pass;
    the larger rate is the L2 peak) and of HBM (4 GiB), from the library's microbenchmark."""
    from paper_1505_06022_gb300 import gsp
    l2 = {f"{mb}MB": round(gsp.gsp_measure_read_bandwidth(ctx.h, mb << 20, 300), 1) for mb in (32, 48)}
    hbm = round(gsp.gsp_measure_read_bandwidth(ctx.h, 4 << 30, 3), 1)
    return {"l2_read_gbs": l2, "l2_peak_gbs": max(l2.values()), "hbm_read_gbs": hbm}


def fp32_peak_tflops(sm_count, peaks):
    sm_max = (peaks or {}).get("sm_max_mhz", 2070.0)
    return sm_count * 128 * 2 * sm_max * 1e6 / 1e12, sm_max


def traversal_roofline(v_node, v_tri, n, ms, call_ms, sm_count, peaks, tiers):
    """The bench line's roofline block for closest hit: algorithmic bytes and flops of n rays with
    v_node node visits and v_tri triangle tests per ray, against the traversal kernel's mean launch
    time `ms` (call_ms: the whole call, with the counter reset and the refinement of flagged hits)."""
    bytes_ray = BYTES_PER_NODE * v_node + BYTES_PER_TRI * v_tri + BYTES_PER_RAY_IO
    flops_ray = FLOPS_PER_NODE * v_node + FLOPS_PER_TRI * v_tri
    hbm = (peaks or {}).get("hbm_gbs")
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (copy), of measured"
    if not hbm:
        hbm, hbm_src = FALLBACK_HBM_GBS, "fallback 6.8 TB/s"
    fp32, sm_max = fp32_peak_tflops(sm_count, peaks)
    s = ms / 1000.0
    t_hbm = bytes_ray * n / (hbm * 1e9)
    t_flop = flops_ray * n / (fp32 * 1e12)
    achieved = bytes_ray * n / s / 1e9
    l2 = tiers["l2_peak_gbs"]
    return {"bound": "hbm" if t_hbm >= t_flop else "alu", "achieved": round(achieved, 1), "peak": hbm,
            "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": None, "peak_source": hbm_src,
            "roofline_ms": round(1000 * max(t_hbm, t_flop), 4), "kernel_ms": round(ms, 4),
            "call_ms": round(call_ms, 4),
            "kernel_timing": "mean over the timed steps of k_trace's own launch: CUDA events that the library "
                             "records on the call's stream right before and after it (gsp_trace_time_launches)",
            "l2": {"peak": l2, "frac": round(achieved / l2, 4), "unit": "GB/s",
                   "source": "gsp_measure_read_bandwidth, buffers of 32 and 48 MB resident in L2"},
            "fp32": {"achieved": round(flops_ray * n / s / 1e12, 3), "peak": round(fp32, 2), "unit": "TFLOP/s",
                     "frac": round(flops_ray * n / s / 1e12 / fp32, 4),
                     "source": f"{sm_count} SMs x 128 FP32 lanes x 2 (FMA) x {sm_max:.0f} MHz"},
            "node_visits_per_ray": round(v_node, 3), "tri_tests_per_ray": round(v_tri, 3),
            "algorithmic_bytes_per_ray": round(bytes_ray, 1), "flops_per_ray": round(flops_ray, 1),
            "algorithmic_bytes_per_launch": int(round(bytes_ray * n)), "tiers": tiers}


# Work model of an SPPM pass (the measurement plan's per-pass figures): every traced ray as a
# closest-hit query above; 3 x 32 bytes per deposit (written, sorted, read back); 32 bytes per
# photon a gather reads and 72 bytes per pixel (hit point and progressive state). The adjoint adds
# 20 bytes per hit point its photon-centric gather reads and 96 bytes per pixel (hit-point grid,
# radius and flux history, loss gradient).
def sppm_work(c, npix, passes, adjoint=False):
    npix, passes = int(npix), int(passes)
    rays = c["eye_rays"] + c["photon_rays"]
    parts = {"traversal": BYTES_PER_NODE * c["node_visits"] + BYTES_PER_TRI * c["tri_tests"] + BYTES_PER_RAY_IO * rays,
             "deposit": 3 * 32 * c["deposits"],
             "gather": 32 * c["photons_scanned"] + 72 * npix * passes}
    if adjoint:
        parts["adjoint_gather"] = 20 * c["hit_points_scanned"] + 96 * npix * passes
    flops = FLOPS_PER_NODE * c["node_visits"] + FLOPS_PER_TRI * c["tri_tests"]
    return sum(parts.values()), flops, parts


def work_roofline(nbytes, flops, seconds, rl, counts=None, parts=None, per=None):
    """Roofline block of a whole workload: algorithmic bytes and flops over its measured time."""
    peaks, tiers, sm_count = rl["peaks"], rl["tiers"], rl["sm_count"]
    hbm = (peaks or {}).get("hbm_gbs") or FALLBACK_HBM_GBS
    fp32, _ = fp32_peak_tflops(sm_count, peaks)
    achieved = nbytes / seconds / 1e9
    t_hbm, t_flop = nbytes / (hbm * 1e9), flops / (fp32 * 1e12)
    out = {"bound": "hbm" if t_hbm >= t_flop else "alu", "achieved": round(achieved, 1), "peak": hbm,
           "unit": "GB/s", "frac": round(achieved / hbm, 4),
           "l2": {"peak": tiers["l2_peak_gbs"], "frac": round(achieved / tiers["l2_peak_gbs"], 4)},
           "fp32": {"achieved": round(flops / seconds / 1e12, 3), "peak": round(fp32, 2), "unit": "TFLOP/s",
                    "frac": round(flops / seconds / 1e12 / fp32, 4)},
           "algorithmic_bytes": int(nbytes), "flops": int(flops)}
    if per:
        out["per"] = per
    if parts:
        out["bytes_by_stage"] = {k: int(v) for k, v in parts.items()}
    if counts:
        out["work_counts"] = counts
    return out


def counted_passes(r, k, warm=0):
    """Work counts of k passes of renderer r (after `warm` uncounted passes)."""
    if warm:
        r.run(warm)
    r.count_work(True)
    r.run(k)
    return r.count_work(False)


def gsp_kernel_digest():
    from paper_1505_06022_gb300 import build
    return build.trace_digest()


def timed_passes(r, k, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r.run(k, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    r.sync()
    return e0.elapsed_time(e1) / k


def oracle_sppm(sc, kw, passes, grad=False):
    """The FP64 CPU oracle rendering `passes` passes of a configuration on all host cores (with
    forward-mode derivatives when grad): (ms per pass, cores)."""
    import oracle as O
    o = O.Sppm(sc, O.default_params(sc, **kw))
    if grad:
        o.enable_grad()
    t0 = time.perf_counter()
    o.run(passes)
    dt = time.perf_counter() - t0
    return 1000.0 * dt / passes, O.nthreads_default()


def with_cpu(args, world, rank):
    return rank == 0 and world == 1 and not args.skip_cpu


def bench_cornell(args, ctx, dev, stream, cpu):
    """The small configuration (Cornell box, 64x64, 16,384 photons/pass, 4 passes, alpha 0.7,
    r0 = 0.05 * diagonal, seed 1): a render of 4 passes on the GPU, and the oracle beside it."""
    import torch
    from paper_1505_06022_gb300 import gsp, inputs as I
    sc = I.cornell_box(seed=1)
    s = gsp.Scene(ctx, sc)
    kw = dict(photons_per_pass=16384, seed=1)
    warm = gsp.Renderer(s, gsp.sppm_params(sc, **kw))
    warm.run(4, stream)
    torch.cuda.synchronize()
    warm.close()
    ms = []
    for _ in range(5):
        r = gsp.Renderer(s, gsp.sppm_params(sc, **kw))
        ms.append(timed_passes(r, 4, stream))
        r.close()
    out = {"ms_per_pass": round(statistics.median(ms), 4), "passes_per_s": round(1000.0 / statistics.median(ms), 1),
           "config": "Cornell box 36 triangles, 64x64, 16,384 photons/pass, 4 passes, alpha 0.7, r0 = 0.05 * diagonal"}
    if cpu:
        oms, cores = oracle_sppm(sc, kw, 4)
        out["cpu_oracle"] = {"ms_per_pass": round(oms, 2), "cores": cores, "passes": 4}
    s.close()
    return out


def bench_sppm(args, ctx, dev, stream, pg, rl):
    import torch
    from paper_1505_06022_gb300 import gsp, inputs as I
    side = args.sppm_side  # 512 for the benchmark; smaller sides only for profiling captures
    sc = I.full_scene(seed=3, width=side, height=side)
    s = gsp.Scene(ctx, sc)
    nphot = (1 << 20) * side * side // (512 * 512)
    params = gsp.sppm_params(sc, nphot, seed=3, r0_frac=0.004)
    warm = gsp.Renderer(s, params)
    warm.run(3, stream)
    torch.cuda.synchronize()
    warm.close()
    # a render of k passes from its first pass (the radii shrink as it goes)
    k = args.sppm_passes
    r = gsp.Renderer(s, params)
    ms = max_over_ranks(timed_passes(r, k, stream), pg, dev)
    img = r.image(stream)
    torch.cuda.synchronize()
    # autotune times its candidates on a temporary renderer: `tuned` itself is still at pass 0
    tuned = gsp.Renderer(s, params)
    t0 = time.perf_counter()
    choice = tuned.autotune(trial_passes=6)
    tune_s = time.perf_counter() - t0
    ms_tuned = timed_passes(tuned, k, stream)
    img_tuned = tuned.image(stream)
    same = bool(torch.equal(img, img_tuned))
    npix = side * side
    out = {"passes_per_s": round(1000.0 / ms, 2), "ms_per_pass": round(ms, 3), "passes_timed": k,
           # the paper's readout is complete paths per second (eye paths + photon paths)
           "paths_per_s": round((npix + nphot) * 1000.0 / ms, 0),
           "autotuned": {"passes_per_s": round(1000.0 / ms_tuned, 2), "ms_per_pass": round(ms_tuned, 3),
                         "choice": {kk: (round(v, 5) if isinstance(v, float) else v) for kk, v in choice.items()},
                         "tuning_s": round(tune_s, 2)},
           "config": f"{side}x{side}, 247,234 triangles (displaced plane, glass/mirror/diffuse icospheres, area light), "
                     f"{nphot:,} photon paths/pass, alpha 0.7, r0 = 0.004 * diagonal, full paths + exact hash grid",
           "image_mean": round(float(img.mean()), 5), "autotuned_image_identical": same}
    # the same k passes once more with the work counted (untimed): the roofline of the timed render
    cr = gsp.Renderer(s, params)
    counts = counted_passes(cr, k)
    cr.close()
    nbytes, flops, parts = sppm_work(counts, npix, k)
    out["roofline"] = work_roofline(nbytes, flops, k * ms / 1000.0, rl, counts, parts,
                                    per="the 64-pass render at the default settings")
    out["autotuned"]["roofline_frac"] = round(nbytes / (k * ms_tuned / 1000.0) / 1e9 / out["roofline"]["peak"], 4)
    if with_cpu(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))):
        oms, cores = oracle_sppm(sc, dict(photons_per_pass=nphot, seed=3, r0_frac=0.004), 2)
        out["cpu_oracle"] = {"ms_per_pass": round(oms, 1), "passes_per_s": round(1000.0 / oms, 3), "cores": cores,
                             "passes": 2, "sample": "the first 2 passes of the same render, FP64 oracle"}
    tuned.close()
    r.close()
    s.close()
    return out


def bench_shaded(args, ctx, dev, stream, pg):
    """The 512^2 SPPM render with per-vertex shading data (smooth normals on every surface,
    texture coordinates, two 256^2 albedo textures) against the same geometry without it."""
    import copy
    import torch
    from paper_1505_06022_gb300 import gsp, inputs as I
    sc = I.shaded_scene(seed=6)
    flat = copy.copy(sc)
    flat.normals, flat.texcoords, flat.textures = None, None, {}
    kw = dict(photons_per_pass=1 << 20, seed=6, r0_frac=0.004)
    k = args.sppm_passes
    out = {}
    for name, scene in (("shaded", sc), ("no_shading_data", flat)):
        s = gsp.Scene(ctx, scene)
        params = gsp.sppm_params(scene, **kw)
        warm = gsp.Renderer(s, params)
        warm.run(3, stream)
        torch.cuda.synchronize()
        warm.close()
        r = gsp.Renderer(s, params)
        ms = max_over_ranks(timed_passes(r, k, stream), pg, dev)
        out[name] = {"ms_per_pass": round(ms, 3), "passes_per_s": round(1000.0 / ms, 2)}
        r.close()
        s.close()
    out["passes_timed"] = k
    out["shading_cost"] = round(out["shaded"]["ms_per_pass"] / out["no_shading_data"]["ms_per_pass"], 3)
    out["config"] = ("512x512, 247,234 triangles, smooth vertex normals (radial on the spheres, area-weighted on the "
                     "plane), texture coordinates, 256^2 albedo textures on the plane and the diffuse sphere, "
                     "1,048,576 photon paths/pass, r0 = 0.004 * diagonal, full paths + exact hash grid")
    if with_cpu(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))):
        oms, cores = oracle_sppm(sc, kw, 2)
        out["cpu_oracle"] = {"ms_per_pass": round(oms, 1), "passes_per_s": round(1000.0 / oms, 3), "cores": cores,
                             "passes": 2, "sample": "the first 2 passes of the shaded render, FP64 oracle"}
    return out


def bench_grad(args, ctx, dev, stream, rl):
    """Backward/forward time of the path-replay adjoint: 256x256, 50,770 triangles, 16 diffuse
    materials, 262,144 photon paths/pass, 8 passes, L2 loss against a render at perturbed albedos."""
    import torch
    from paper_1505_06022_gb300 import gsp, inputs as I
    sc = I.grad_scene(seed=4)
    s = gsp.Scene(ctx, sc)
    params = gsp.sppm_params(sc, 1 << 18, seed=4, r0_frac=0.004)
    passes = 8
    tgt = sc.mats.copy()
    tgt["albedo"] = np.clip(tgt["albedo"] * np.random.default_rng(40).uniform(0.8, 1.2, tgt["albedo"].shape), 0.05, 0.95)
    gsp.gsp_scene_set_materials(s.h, tgt)
    rt = gsp.Renderer(s, params)
    rt.run(passes, stream)
    target = rt.image(stream)
    gsp.gsp_scene_set_materials(s.h, sc.mats)
    # execution settings for this scene (they leave the estimate unchanged; the replay uses them too)
    probe = gsp.Renderer(s, params)
    choice = probe.autotune(trial_passes=2)
    probe.close()
    params = dict(params, cell_h=float(choice["cell_h"]))
    fwd, bwd = [], []
    for rep in range(7):  # medians of 6 timed repetitions (the first warms up)
        r = gsp.Renderer(s, params)
        r.tune(choice["eye_steps"], choice["photon_steps"], 0.0, choice["gather_lanes"], choice["traversal"])
        r.enable_grad(passes)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        r.run(passes, stream)
        img = r.image(stream)
        e[1].record(stream)
        g = (img - target).contiguous()
        ga, gl = r.grad(g, stream)
        e[2].record(stream)
        torch.cuda.synchronize()
        r.sync()
        if rep > 0:  # the first repetition warms up
            fwd.append(e[0].elapsed_time(e[1]))
            bwd.append(e[1].elapsed_time(e[2]))
        r.close()
    # work of the forward and of the backward (the replay and the adjoint gathers), counted untimed
    r = gsp.Renderer(s, params)
    r.tune(0, 0, 0.0, choice["gather_lanes"], 1)
    r.enable_grad(passes)
    r.count_work(True)
    r.run(passes, stream)
    img = r.image(stream)
    cf = r.count_work(True)
    r.grad((img - target).contiguous(), stream)
    cb = r.count_work(False)
    r.close()
    f, b = statistics.median(fwd), statistics.median(bwd)
    npix = 256 * 256
    fb, ff, fparts = sppm_work(cf, npix, passes)
    bb, bf, bparts = sppm_work(cb, npix, passes, adjoint=True)
    out = {"forward_ms": round(f, 3), "backward_ms": round(b, 3), "backward_over_forward": round(b / f, 3),
           "grad_norm": round(float(ga.norm()), 6),
           "roofline": {"forward": work_roofline(fb, ff, f / 1000.0, rl, cf, fparts),
                        "backward": work_roofline(bb, bf, b / 1000.0, rl, cb, bparts)},
           "settings": {k: (round(v, 5) if isinstance(v, float) else v) for k, v in choice.items()
                        if k in ("eye_steps", "photon_steps", "cell_h", "gather_lanes", "traversal")},
           "config": "256x256, 50,770 triangles (displaced plane in 12 material regions + 4 icospheres), "
                     "16 diffuse materials + light, 262,144 photon paths/pass, 8 passes, L2 loss vs a render "
                     "at perturbed albedos; gradient w.r.t. 16 RGB albedos and the light's emission"}
    if with_cpu(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))):
        # the oracle's gradient: FP64 forward-mode derivatives carried through the 8 passes
        oms, cores = oracle_sppm(sc, dict(photons_per_pass=1 << 18, seed=4, r0_frac=0.004), passes, grad=True)
        out["cpu_oracle"] = {"forward_with_gradient_ms": round(oms * passes, 1), "cores": cores,
                             "sample": "the same 8 passes, FP64 forward-mode derivatives"}
    return out


def bench_traversals(args, ctx, dev, stream, sc, scene, rays):
    """Fig. 4's comparison on the closest-hit workload: the multiple-threaded BVH (6 link sets),
    the original threaded BVH (1 link set, one fixed order) and a stack-based near-first
    traversal of the same SAH tree, each on all rays and on the coherent and random halves."""
    import torch
    from paper_1505_06022_gb300 import gsp
    n = rays.shape[0]
    tbvh = gsp.Scene(ctx, sc, bins=16, leaf_threshold=4, max_leaf=7, link_sets=1)
    t0 = time.perf_counter()
    lbvh = gsp.Scene(ctx, sc, builder="device", link_sets=6, max_leaf=4)
    lbvh_wall_ms = 1000.0 * (time.perf_counter() - t0)
    tri = torch.empty(n, dtype=torch.int32, device=dev)
    tt = torch.empty(n, dtype=torch.float32, device=dev)
    parts = {"all": (0, n), "coherent": (0, n // 2), "random": (n // 2, n)}
    kinds = {"mtbvh": (scene, gsp.gsp_trace_closest_hit), "tbvh": (tbvh, gsp.gsp_trace_closest_hit),
             "stack": (scene, gsp.gsp_trace_closest_hit_stack),
             "mtbvh_on_device_lbvh": (lbvh, gsp.gsp_trace_closest_hit),
             "stack_on_device_lbvh": (lbvh, gsp.gsp_trace_closest_hit_stack)}
    reps = max(3, min(args.steps, 30))
    out = {}
    for kind, (scn, fn) in kinds.items():
        out[kind] = {}
        for part, (a, b) in parts.items():
            r, o1, o2 = rays[a:b], tri[a:b], tt[a:b]
            for _ in range(2):
                fn(scn.h, r, o1, o2, None, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn(scn.h, r, o1, o2, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out[kind][part] = round((b - a) / (ms / 1000.0) / 1e6, 1)
    ctx.sync()
    tbvh.close()
    out["mtbvh_over_tbvh"] = {p: round(out["mtbvh"][p] / out["tbvh"][p], 3) for p in parts}
    out["unit"] = "Mrays/s"
    out["bvh_build"] = {
        "host_sah_ms": round(scene.stats["build_ms"], 1), "host_threading_ms": round(scene.stats["thread_ms"], 1),
        "device_lbvh_ms": round(lbvh.stats["build_ms"], 2), "device_threading_ms": round(lbvh.stats["thread_ms"], 2),
        "device_lbvh_call_ms": round(lbvh_wall_ms, 1),
        "nodes": {"host_sah": scene.stats["nodes"], "device_lbvh": lbvh.stats["nodes"]}}
    lbvh.close()
    return out


def bench_modes(args, ctx, dev, stream):
    """The paper's photon-pass and hashing variants at equal image error (512x512 full scene,
    2^20 photon paths or threads per pass): RMSE against a 256-pass full-path exact-grid render
    of another seed, after 16, 32 and 64 passes, time per pass, and the time each mode needs to
    reach the error of 64 full-path exact-grid passes (log-log interpolation in passes)."""
    import torch
    from paper_1505_06022_gb300 import gsp, inputs as I
    sc = I.full_scene(seed=3)
    s = gsp.Scene(ctx, sc)
    ref = gsp.Renderer(s, gsp.sppm_params(sc, 1 << 20, seed=99, r0_frac=0.004))
    ref.run(256, stream)
    want = ref.image(stream).double()
    ref.close()
    norm = float(want.pow(2).mean().sqrt())
    modes = {"full_path+exact": (gsp.FULL_PATH, gsp.EXACT), "full_path+stochastic": (gsp.FULL_PATH, gsp.STOCHASTIC),
             "regen+exact": (gsp.REGEN, gsp.EXACT), "regen+stochastic": (gsp.REGEN, gsp.STOCHASTIC)}
    marks = [16, 32, 64]
    out = {}
    for name, (pm, hm) in modes.items():
        r = gsp.Renderer(s, gsp.sppm_params(sc, 1 << 20, seed=3, r0_frac=0.004, photon_mode=pm, hash_mode=hm))
        rmse, ms, done = [], 0.0, 0
        for k in marks:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r.run(k - done, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            done = k
            img = r.image(stream).double()
            rmse.append(float((img - want).pow(2).mean().sqrt()) / norm)
        out[name] = {"ms_per_pass": round(ms / marks[-1], 3), "relative_rmse": dict(zip(map(str, marks),
                                                                                   [round(v, 5) for v in rmse]))}
        r.close()
    target = out["full_path+exact"]["relative_rmse"]["64"]
    for name, o in out.items():
        e = [o["relative_rmse"][str(k)] for k in marks]
        slope = (np.log(e[-1]) - np.log(e[0])) / (np.log(marks[-1]) - np.log(marks[0]))
        passes = marks[-1] * np.exp((np.log(target) - np.log(e[-1])) / slope) if slope < 0 else float("nan")
        o["passes_to_reference_error"] = round(float(passes), 1)
        o["ms_to_reference_error"] = round(float(passes) * o["ms_per_pass"], 1)
    s.close()
    return {"modes": out, "reference": "256 passes, full paths + exact grid, seed 99",
            "error_target": f"relative RMSE {target} (64 passes of full paths + exact grid)"}


def bench_batch(args, ctx, dev, stream, rl):
    """64 scenes (1k-200k triangles log-uniform, 64^2-512^2): scene-passes per second as one CUDA
    graph per pass (settings from the batch autotuner) vs the same renderers run one after
    another, k passes each (the same photons gathered)."""
    import torch
    from paper_1505_06022_gb300 import gsp, inputs as I
    scs = I.batch_scenes(args.batch_scenes, seed=5)
    scenes = [gsp.Scene(ctx, sc) for sc in scs]
    mk = lambda: [gsp.Renderer(s, gsp.sppm_params(sc, 1 << 18, seed=5 + i, r0_frac=0.004, scene_id=i))
                  for i, (s, sc) in enumerate(zip(scenes, scs))]
    k = args.batch_passes + args.batch_passes % 2  # whole two-pass graphs
    seq = mk()
    for r in seq:
        r.run(2, stream)  # untimed: allocates the second trace set that several passes use
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the plain path: one renderer after another, each running its k passes in one call
    e0.record(stream)
    for r in seq:
        r.run(k, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / k
    for r in seq:
        r.close()
    bat = mk()
    b = gsp.Batch(bat)
    t0 = time.perf_counter()
    choice = b.autotune(trial_passes=2)
    tune_s = time.perf_counter() - t0
    b.run(2, stream)  # untimed: captures the graphs the timed passes replay
    torch.cuda.synchronize()
    e0.record(stream)
    b.run(k, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    bat_ms = e0.elapsed_time(e1) / k
    for r in bat:
        r.sync()
    n = len(scs)
    # work of the timed passes (passes 2 .. k + 1 of every scene), counted on renderers run alone
    # (a batched pass does the same work; batched passes are not counted)
    tot = None
    npix_sum = 0
    for i, (sc_, scn) in enumerate(zip(scs, scenes)):
        cr = gsp.Renderer(scn, gsp.sppm_params(sc_, 1 << 18, seed=5 + i, r0_frac=0.004, scene_id=i))
        c = counted_passes(cr, k, warm=2)
        cr.close()
        tot = c if tot is None else {kk: tot[kk] + c[kk] for kk in c}
        npix_sum += int(sc_.camera[0]["width"]) * int(sc_.camera[0]["height"])
    nbytes, flops, parts = sppm_work(tot, npix_sum, k)
    out = {"scenes": n, "triangles": [int(min(sc.ntris for sc in scs)), int(max(sc.ntris for sc in scs))],
           "sequential_scene_passes_per_s": round(1000.0 * n / seq_ms, 1),
           "graph_scene_passes_per_s": round(1000.0 * n / bat_ms, 1),
           "speedup": round(seq_ms / bat_ms, 3), "ms_per_batch_pass": round(bat_ms, 3), "passes_timed": k,
           "roofline": work_roofline(nbytes, flops, k * bat_ms / 1000.0, rl, tot, parts, per="the timed batch passes"),
           "sequential_roofline_frac": round(nbytes / (k * seq_ms / 1000.0) / 1e9 /
                                             ((rl["peaks"] or {}).get("hbm_gbs") or FALLBACK_HBM_GBS), 4),
           "batch_autotune": {"choice": {kk: v for kk, v in choice.items()
                                         if kk in ("eye_steps", "photon_steps", "gather_lanes", "traversal",
                                                   "fused", "cell_h")},
                              "tuning_s": round(tune_s, 2)},
           "config": f"{n} scenes, 1e3-2e5 triangles log-uniform, image side in {{64,128,256,512}}, "
                     "262,144 photon paths/pass each, full paths + exact hash grid"}
    if with_cpu(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))):
        t = []
        for i, sc in enumerate(scs[:4]):
            oms, cores = oracle_sppm(sc, dict(photons_per_pass=1 << 18, seed=5 + i, r0_frac=0.004, scene_id=i), 1)
            t.append(oms)
        out["cpu_oracle"] = {"scene_passes_per_s": round(1000.0 * len(t) / sum(t), 2), "cores": cores,
                             "sample": "one pass of each of the first 4 scenes, FP64 oracle"}
    b.close()
    for r in bat:
        r.close()
    for s in scenes:
        s.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sppm-passes", type=int, default=64)
    ap.add_argument("--sppm-side", type=int, default=512,
                    help="image side of the full-scene SPPM section (512 = the benchmark; smaller sides, with "
                         "photons scaled by the pixel count, only for profiling captures)")
    ap.add_argument("--skip-sppm", action="store_true")
    ap.add_argument("--skip-shaded", action="store_true")
    ap.add_argument("--skip-grad", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-fig4", action="store_true")
    ap.add_argument("--skip-modes", action="store_true")
    ap.add_argument("--batch-scenes", type=int, default=64)
    ap.add_argument("--batch-passes", type=int, default=4)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--ref-rays", type=int, default=1 << 19,
                    help="rays per step of the CPU reference arm (a stratified sample of the batch)")
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
