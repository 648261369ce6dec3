"""Benchmark: Mpaths/s and ms/frame of the tet-grid path tracer at 1024^2, 32 spp.

Workload: the production scene -- a 1024 x 1024 x 512 sparse fBm x Worley
cloud (synthetic, seeded), adaptive LEB grid for the 1024^2 view at a 1-pixel
footprint, BF16 densities, albedo 0.95, HG g = 0.7, up to 128 bounces, sun and
environment light.  A step renders one 1024^2 x 32 spp frame (33.5 M paths)
on the grid, which is built once before timing (its build time is reported
separately and is part of the end-to-end number).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--scene NAME]

Under torchrun each rank renders the frame with its own range of samples
(no data-path collective): weak scaling.  --impl reference times the CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpaths/s & ms/frame @1024² 32spp; time-to-equal-RMSE cached vs plain"
BYTES_PER_STEP = 32          # one 32-byte record (one DRAM sector) per tet step, shadow steps included


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--scene", default="production")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-dda", action="store_true", help="skip the regular-grid comparator frame")
    p.add_argument("--cpu-sample-px", type=int, default=0, help="side of the oracle's pixel window (0: auto)")
    p.add_argument("--no-cache", action="store_true", help="skip the radiance-cache time-to-equal-RMSE leg")
    p.add_argument("--no-ext", action="store_true", help="skip the extra-channel / voxel-medium frames")
    p.add_argument("--no-rebuild", action="store_true", help="skip the moved-camera rebuild leg")
    p.add_argument("--no-batch", action="store_true", help="skip the batched heterogeneous leg")
    p.add_argument("--no-precision", action="store_true", help="skip the FP32 / FP16 density-storage frames")
    p.add_argument("--batch-jobs", type=int, default=64)
    p.add_argument("--cache-train-rounds", default="2,4,8,32,128", help="training budgets (rounds of 2^16 samples)")
    p.add_argument("--cache-train-bounces", default="16,32",
                   help="collision limits of training paths tried besides the medium's (empty: none)")
    p.add_argument("--cache-ref-pixels", type=int, default=4096)
    p.add_argument("--cache-ref-spp", type=int, default=4096)
    p.add_argument("--mlp-kernels-only", action="store_true",
                   help="only time the radiance cache's MLP kernels (no grid, no frame) and print their rates")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    for path in (os.path.join(ROOT, "MEASURED_PEAKS.json"),):
        if os.path.exists(path):
            with open(path) as fh:
                d = json.load(fh)
            return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = open(os.path.join("/tmp", "tetvol_clocks_%d.csv" % os.getpid()), "w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        self.out.close()
        try:
            os.remove(self.out.name)
        except OSError:
            pass
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                s, m = float(r[1]), float(r[2])
            except (ValueError, IndexError):
                continue
            sm.append(s)
            mx = max(mx, m)
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2506_11510_gb300", "csrc")
    for f in ("estimator.cuh", "walk_tet.cuh", "common.cuh", "render.cu"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(scene_name):
    """DRAM bytes per render launch from the committed ncu summary, if it was taken
    on the current kernel source; otherwise None."""
    path = os.path.join(ROOT, "profiles", "k_estimate_%s_traffic.json" % scene_name)
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    if d.get("kernel_digest") != kernel_source_digest():
        return None
    return d.get("dram_bytes_per_launch")


def workload_name(s):
    """The workload, named by the scene's recipe and sizes (the same for both arms)."""
    nx, ny, nz = s.dims
    vol = {"sphere": "fBm-perturbed sphere", "cloud": "fBm cloud", "wispy": "fBm x Worley cloud"}.get(s.recipe,
                                                                                                  s.recipe)
    uniform = s.variation_threshold < 0 and s.footprint_px <= 0
    grid = ("uniform LEB grid, depth %d" % s.max_depth) if uniform else "adaptive LEB grid"
    return ("%s: %dx%dx%d %s, %s (%s density), %dx%d @ %d spp, albedo %.2f, g %.1f, <= %d bounces"
            % (s.name, nx, ny, nz, vol, grid, {0: "FP32", 1: "BF16", 2: "FP16"}[s.density_format],
               s.camera.width, s.camera.height, s.spp, s.medium.albedo, s.medium.g, s.medium.max_bounces))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import _build, sharding, workloads as W

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    dev = torch.device("cuda", local if ws > 1 else torch.cuda.current_device())
    s = W.scene(args.scene)
    st = torch.cuda.current_stream()

    vol = W.make_volume(s, device=dev)
    torch.cuda.synchronize()
    t0 = time.time()
    grid = tv.build_scene_grid(s, vol)
    torch.cuda.synchronize()
    build_ms = (time.time() - t0) * 1e3
    ntets = grid.info.num_tets
    grid_depth = grid.info.max_depth

    W_, H_ = s.camera.width, s.camera.height
    img = torch.zeros((H_, W_), dtype=torch.float32, device=dev)
    img2 = torch.zeros_like(img)
    stats = tv.new_stats(dev)
    spp = s.spp
    offset, _ = sharding.sample_range(rank, ws, spp)      # each rank its own samples

    for _ in range(args.warmup):
        tv.tet_render(grid, s.camera, s.medium, spp, s.render_seed, offset, img, img2)
    torch.cuda.synchronize()

    # counters of one frame (identical every frame: same paths)
    stats.zero_()
    tv.tet_render(grid, s.camera, s.medium, spp, s.render_seed, offset, img, img2, stats=stats)
    torch.cuda.synchronize()
    counters = tv.stats_dict(stats)
    steps_per_frame = counters["tet_steps"] + counters["shadow_steps"]

    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    e_all0, e_all1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_all0.record(st)
    for i in range(args.steps):
        ev[i][0].record(st)
        tv.tet_render(grid, s.camera, s.medium, spp, s.render_seed, offset, img, img2)
        ev[i][1].record(st)
    e_all1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = e_all0.elapsed_time(e_all1)
    per_launch = [a.elapsed_time(b) for a, b in ev]
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    ms_per_step = total_ms / args.steps
    paths = float(W_ * H_ * spp)
    value = paths * ws * args.steps / (total_ms * 1e-3) / 1e6

    # the regular-grid comparator (3D DDA, same estimator) on the same volume, camera and medium
    comparator = None
    if not args.no_dda:
        dsum = torch.zeros_like(img)
        dst = tv.new_stats(dev)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(st)
        tv.grid_render(vol, s.box_min, s.voxel_size, s.camera, s.medium, spp, s.render_seed, offset, dsum, None, dst,
                       want_sq=False)
        a1.record(st)
        torch.cuda.synchronize()
        dda_ms = a0.elapsed_time(a1)
        dcount = tv.stats_dict(dst)
        comparator = {"method": "regular voxel grid, 3D DDA, same estimator", "voxels": int(vol.numel()),
                      "ms_per_frame": round(dda_ms, 2), "mpaths_s": round(paths / dda_ms / 1e3, 3),
                      "voxel_steps_per_path": round((dcount["tet_steps"] + dcount["shadow_steps"]) / paths, 1),
                      "tet_speedup": round(dda_ms / (total_ms / args.steps), 3)}
        if rank == 0 and args.scene == "production":
            comparator["adaptive_256"] = adaptive_comparator_leg(dev)

    precision = None
    if not args.no_precision and rank == 0:
        precision = precision_leg(s, grid, vol, dev)

    cache = None
    if not args.no_cache and rank == 0:
        cache = cache_leg(args, s, grid, dev, ms_per_step)
    ext = None
    if not args.no_ext and rank == 0:
        ext = ext_leg(s, grid, vol, dev, comparator)
    rebuild = None
    if not args.no_rebuild and rank == 0:
        rebuild = rebuild_leg(s, grid, vol)
    batch = None
    if not args.no_batch and rank == 0:
        batch = batch_leg(args, dev)

    # end to end through the public API: host volume -> device, build, render, image -> host
    e2e = None
    if args.e2e_steps > 0:
        host_vol = vol.cpu().pin_memory()
        out_sum = torch.empty((H_, W_), dtype=torch.float32).pin_memory()
        out_sq = torch.empty_like(out_sum).pin_memory()
        del grid
        torch.cuda.empty_cache()
        # the build reads the pinned host volume in place (each value once, in its quantisation
        # kernel): no separate upload.  For comparison, one step that first copies it to the device.
        torch.cuda.synchronize()
        c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        c0.record(st)
        dvol = host_vol.to(dev, non_blocking=True)
        c1.record(st)
        g2 = tv.build_scene_grid(s, dvol)
        c2.record(st)
        torch.cuda.synchronize()
        copy_path = {"upload_ms": round(c0.elapsed_time(c1), 2), "build_ms": round(c1.elapsed_time(c2), 2)}
        del g2, dvol
        times, phases = [], None
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.time()
            ev4 = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev4[0].record(st)
            g2 = tv.build_scene_grid(s, host_vol)
            ev4[1].record(st)
            a, b = tv.tet_render(g2, s.camera, s.medium, spp, s.render_seed, offset)
            ev4[2].record(st)
            out_sum.copy_(a, non_blocking=True)
            out_sq.copy_(b, non_blocking=True)
            ev4[3].record(st)
            torch.cuda.synchronize()
            times.append(time.time() - t0)
            phases = {k: round(ev4[i].elapsed_time(ev4[i + 1]), 2)
                      for i, k in enumerate(("build_from_pinned_host", "render", "download"))}
            del g2
        e2e_s = sum(times) / len(times)
        if ws > 1:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": round(paths * ws / e2e_s / 1e6, 3), "unit": "Mpaths/s",
               "h2d_bytes_per_step": int(host_vol.numel() * 4), "d2h_bytes_per_step": int(2 * out_sum.numel() * 4),
               "ms_per_step": round(e2e_s * 1e3, 2),
               "includes": "LEB build reading the pinned host volume in place, frame render, image download",
               "last_step_phases_ms": phases, "copy_then_build": copy_path}

    peak, peak_kind = load_peaks()
    mean_launch_ms = sum(per_launch) / len(per_launch)
    achieved = steps_per_frame * BYTES_PER_STEP / (mean_launch_ms * 1e-3) / 1e9
    traffic = profiled_traffic(args.scene)
    dram_frac = None if traffic is None else round(traffic / (mean_launch_ms * 1e-3) / 1e9 / peak, 4)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "dram_frac": dram_frac,
                "dram_frac_note": "measured DRAM bytes per launch (profiles/k_estimate_production_traffic.json) "
                                  "over this run's mean launch time, against the same peak",
                "kernel": "k_estimate<TetWalker> (persistent path tracer)",
                "algorithmic_bytes": "32 B per tet step x %d steps per launch" % steps_per_frame,
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured" else
                "fallback 6.8 TB/s"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, s, vol, dev)
        checks = cpu.pop("oracle_checks", None)
        if checks is not None:
            if precision is not None:
                precision["vs_fp64_oracle"] = checks
            if cache is not None:
                cache["reference_check"] = checks["cache_reference_check"]

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "Mpaths/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded procedural volume; stands in for the paper's OpenVDB assets)",
                "config": {"workload": workload_name(s), "ms_per_frame": round(ms_per_step, 3),
                           "tets": ntets, "grid_depth": grid_depth, "build_ms": round(build_ms, 1),
                           "width": W_, "height": H_, "spp": spp, "paths_per_frame": int(paths),
                           "tet_steps_per_path": round(steps_per_frame / paths, 2),
                           "g_tet_steps_per_s": round(steps_per_frame / (mean_launch_ms * 1e-3) / 1e9, 3),
                           "collisions_per_path": round(counters["collisions"] / paths, 3),
                           "density_storage": {0: "fp32", 1: "bf16", 2: "fp16"}[s.density_format],
                           "l2": "inputs larger than L2: grid records %.2f GB" % (ntets * 32 / 1e9),
                           "parallelism": "one frame per rank, disjoint sample ranges"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
                "clocks": clk, "comparator": comparator, "precision": precision, "cache": cache, "ext": ext,
                "rebuild": rebuild,
                "batch": batch}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# density storage: FP32 and FP16 beside the benchmark's BF16
# ---------------------------------------------------------------------------
def precision_leg(s, grid, vol, dev):
    """The frame on grids whose densities are stored as FP32, BF16 and FP16 (the
    same cells: the criteria use exact integer statistics, not the stored
    value): frame time, and each image's difference from the FP32-density
    image over the same paths.  Every format fills the same 32-byte record, so
    BF16 and FP16 save no bytes per cell step; what they change is the density
    value.  The comparison against the fp64 oracle is added by the CPU-baseline
    leg (vs_fp64_oracle)."""
    import dataclasses
    import torch
    import paper_2506_11510_gb300 as tv
    st = torch.cuda.current_stream()
    H_, W_ = s.camera.height, s.camera.width
    out = {"record_bytes": 32, "note": "density sits in the record's last word in every format (no bytes saved)"}
    imgs = {}
    for fmt, name in ((0, "fp32"), (1, "bf16"), (2, "fp16")):
        g = grid if fmt == s.density_format else tv.build_scene_grid(dataclasses.replace(s, density_format=fmt), vol)
        a = torch.zeros((H_, W_), dtype=torch.float32, device=dev)
        a2 = torch.zeros_like(a)
        tv.tet_render(g, s.camera, s.medium, s.spp, s.render_seed, 0, a, a2)          # image (and warm-up)
        ms = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b = torch.zeros_like(a)
            e0.record(st)
            tv.tet_render(g, s.camera, s.medium, s.spp, s.render_seed, 0, b, None, want_sq=False)
            e1.record(st)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        imgs[name] = (a.double() / s.spp, a2.double() / s.spp)
        out[name] = {"tets": g.info.num_tets, "ms_per_frame": round(min(ms), 2)}
        if g is not grid:
            del g
        torch.cuda.empty_cache()
    ref, ref2 = imgs["fp32"]
    rms = float(torch.sqrt(torch.mean(ref ** 2)))
    se = float(torch.sqrt(torch.mean(torch.clamp(ref2 - ref ** 2, min=0) / s.spp)))
    out["frame"] = ("1024^2 at 32 spp, the same paths in every format; errors relative to the FP32-density "
                    "image's RMS %.5f; Monte Carlo standard error of a pixel %.5f of it" % (rms, se / rms))
    for name in ("bf16", "fp16"):
        m = imgs[name][0]
        out[name].update({"pixel_rms_rel": round(float(torch.sqrt(torch.mean((m - ref) ** 2))) / rms, 6),
                          "pixel_max_rel": round(float(torch.max(torch.abs(m - ref))) / rms, 6),
                          "image_mean_rel": round(float((m.mean() - ref.mean()) / ref.mean()), 6)})
    return out


# ---------------------------------------------------------------------------
# the regular-grid comparator on the 256^3 adaptive scene
# ---------------------------------------------------------------------------
def adaptive_comparator_leg(dev):
    """Tet frame and DDA frame on the 256^3 cloud (512^2 at 32 spp, ~4 M tets):
    the speed-up over the regular grid at the second configuration."""
    import torch
    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import workloads as W
    s = W.scene("adaptive")
    vol = W.make_volume(s, device=dev)
    g = tv.build_scene_grid(s, vol)
    st = torch.cuda.current_stream()
    a = torch.zeros((s.camera.height, s.camera.width), dtype=torch.float32, device=dev)

    def timed(fn, reps=3):
        fn()
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return min(ms)
    tet_ms = timed(lambda: tv.tet_render(g, s.camera, s.medium, s.spp, s.render_seed, 0, a, None, want_sq=False))
    dda_ms = timed(lambda: tv.grid_render(vol, s.box_min, s.voxel_size, s.camera, s.medium, s.spp, s.render_seed, 0,
                                          a, None, want_sq=False))
    res = {"workload": workload_name(s), "tets": g.info.num_tets, "voxels": int(vol.numel()),
           "tet_ms_per_frame": round(tet_ms, 2), "dda_ms_per_frame": round(dda_ms, 2),
           "tet_speedup": round(dda_ms / tet_ms, 3)}
    del g, vol
    torch.cuda.empty_cache()
    return res


# ---------------------------------------------------------------------------
# batched heterogeneous rendering
# ---------------------------------------------------------------------------
def batch_leg(args, dev):
    """64 clouds of uneven size (64^3..384^3 voxels, 128^2..1024^2 views, 4..64 spp,
    g in [-0.3, 0.8]) rendered by one persistent CUDA-graph launch (autotuned),
    against the same jobs rendered one tet_render after another."""
    import statistics as stt
    import torch
    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import workloads as W
    st = torch.cuda.current_stream()
    scenes = W.batch_scenes(args.batch_jobs, seed=100)
    jobs, tets = [], []
    t0 = time.time()
    for sc in scenes:
        v = W.make_volume(sc, device=dev)
        g = tv.build_scene_grid(sc, v)
        del v
        a = torch.zeros((sc.camera.height, sc.camera.width), dtype=torch.float32, device=dev)
        jobs.append((g, sc.camera, sc.medium, sc.spp, sc.render_seed, a, None))
        tets.append(g.info.num_tets)
    torch.cuda.synchronize()
    prep_s = time.time() - t0
    paths = sum(sc.camera.width * sc.camera.height * sc.spp for sc in scenes)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # one job after another
    for (g, cam, med, spp, seed, a, _) in jobs[:4]:
        tv.tet_render(g, cam, med, spp, seed, 0, a, None, want_sq=False)
    marks = [ev() for _ in range(len(jobs) + 1)]
    marks[0].record(st)
    for k, (g, cam, med, spp, seed, a, _) in enumerate(jobs):
        tv.tet_render(g, cam, med, spp, seed, 0, a, None, want_sq=False)
        marks[k + 1].record(st)
    torch.cuda.synchronize()
    seq_done = [marks[0].elapsed_time(m) for m in marks[1:]]
    seq_ms = seq_done[-1]
    # one launch
    t0 = time.time()
    b = tv.Batch(jobs, autotune=True)
    torch.cuda.synchronize()
    tune_s = time.time() - t0
    b.render()
    e0, e1 = ev(), ev()
    reps = 3
    e0.record(st)
    for _ in range(reps):
        b.render()
    e1.record(st)
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1) / reps
    knobs, job_ms = b.info()

    def pct(xs, q):
        xs = sorted(xs)
        return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))]
    res = {"jobs": len(jobs), "paths": paths, "tets_min": min(tets), "tets_max": max(tets),
           "tets_median": int(stt.median(tets)), "setup_s": round(prep_s, 1),
           "one_launch": {"ms": round(batch_ms, 2), "mpaths_s": round(paths / batch_ms / 1e3, 3),
                          "job_latency_ms_p50": round(pct(job_ms, 0.5), 2),
                          "job_latency_ms_p99": round(pct(job_ms, 0.99), 2), "knobs": knobs,
                          "autotune_s": round(tune_s, 2), "graph": True},
           "one_after_another": {"ms": round(seq_ms, 2), "mpaths_s": round(paths / seq_ms / 1e3, 3),
                                 "job_latency_ms_p50": round(pct(seq_done, 0.5), 2),
                                 "job_latency_ms_p99": round(pct(seq_done, 0.99), 2)},
           "speedup": round(seq_ms / batch_ms, 3)}
    b.free()
    return res


# ---------------------------------------------------------------------------
# rebuilds for a moved camera (animated camera)
# ---------------------------------------------------------------------------
def rebuild_leg(s, grid, vol):
    """leb_rebuild from the frame's grid for moved cameras, against a fresh
    leb_build for the same camera: time, whether the two grids are identical,
    and the fraction of the new grid's cells the previous grid did not have.
    The first two moves (a small orbit and a zoom) leave this grid unchanged;
    the camera moved close to the cloud and the pan that sweeps the frustum's
    edge across it change it."""
    import torch
    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import workloads as W
    c = s.camera
    tgt = c.target
    prev_codes = grid.export(("codes",))["codes"]
    moves = []
    for name, deg, zoom in (("orbit 5 deg", 5.0, 1.0), ("zoom 10%", 0.0, 0.9)):
        a = math.radians(deg)
        vx, vz = c.pos[0] - tgt[0], c.pos[2] - tgt[2]
        pos = (tgt[0] + zoom * (vx * math.cos(a) - vz * math.sin(a)), tgt[1] + zoom * (c.pos[1] - tgt[1]),
               tgt[2] + zoom * (vx * math.sin(a) + vz * math.cos(a)))
        moves.append((name, dict(pos=pos)))
    moves.append(("camera moved close (eye 0.6 in front of the box)", dict(pos=(1.0, 1.0, -0.6))))
    moves.append(("pan: eye and target 0.8 along x (frustum edge across the cloud)",
                  dict(pos=(c.pos[0] + 0.8, c.pos[1], c.pos[2]), target=(tgt[0] + 0.8, tgt[1], tgt[2]))))
    res = []
    for name, cam in moves:
        s1 = W.with_camera(s, **cam)
        torch.cuda.synchronize()
        t0 = time.time()
        g1 = tv.rebuild_scene_grid(grid, s1, vol)
        torch.cuda.synchronize()
        t_re = (time.time() - t0) * 1e3
        t0 = time.time()
        g2 = tv.build_scene_grid(s1, vol)
        torch.cuda.synchronize()
        t_full = (time.time() - t0) * 1e3
        e1, e2 = g1.export(("codes", "nbr")), g2.export(("codes", "nbr"))
        same = g1.info.num_tets == g2.info.num_tets and all(torch.equal(e1[k], e2[k]) for k in e1)
        new_frac = float((~torch.isin(e1["codes"], prev_codes)).double().mean())
        res.append({"move": name, "tets": g1.info.num_tets, "new_cells_frac": round(new_frac, 4),
                    "rebuild_ms": round(t_re, 1), "fresh_build_ms": round(t_full, 1),
                    "speedup": round(t_full / t_re, 3), "identical": bool(same)})
        del g1, g2, e1, e2
    return res


# ---------------------------------------------------------------------------
# extra channels (temperature -> emission, albedo, g) and the voxel medium
# ---------------------------------------------------------------------------
def ext_leg(s, grid, vol, dev, comparator):
    """Frames of the extended medium on the same grid: per-cell channels with
    emission, and the voxel medium tracked against the cells' voxel majorants
    (the medium the regular-grid comparator renders)."""
    import torch
    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import workloads as W
    st = torch.cuda.current_stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        out = fn()
        b.record(st)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    t, a, g = W.make_channels(s, device=dev)
    torch.cuda.synchronize()
    t0 = time.time()
    grid.channels(vol, t, a, g)
    chan_ms = (time.time() - t0) * 1e3
    del t, a, g
    paths = s.camera.width * s.camera.height * s.spp
    res = {"channels_ms": round(chan_ms, 1), "variants": []}
    for name, flags in (("emission+albedo+g channels", 7), ("voxel medium, delta tracking on tet majorants", 8),
                        ("voxel medium + channels", 15)):
        tv.tet_render_ext(grid, s.camera, s.medium, flags, s.spp, s.render_seed, emission_scale=2.0, density=vol)
        stats = tv.new_stats(dev)
        _, ms = timed(lambda: tv.tet_render_ext(grid, s.camera, s.medium, flags, s.spp, s.render_seed,
                                                emission_scale=2.0, density=vol, stats=stats))
        c = tv.stats_dict(stats)
        v = {"flags": flags, "name": name, "ms_per_frame": round(ms, 2), "mpaths_s": round(paths / ms / 1e3, 3),
             "tet_steps_per_path": round((c["tet_steps"] + c["shadow_steps"]) / paths, 1),
             "collisions_per_path": round(c["collisions"] / paths, 3)}
        if flags & 8 and comparator is not None:
            v["speedup_vs_dda_same_medium"] = round(comparator["ms_per_frame"] / ms, 3)
        res["variants"].append(v)
    return res


# ---------------------------------------------------------------------------
# the learned radiance cache: time to equal RMSE, cached vs plain
# ---------------------------------------------------------------------------
def cache_leg(args, s, grid, dev, plain_ms):
    """RMSE over random pixels against a high-spp plain reference: the plain
    tracer's at the frame's spp (one frame, plain_ms), and the cached tracer's
    after online training, at increasing spp; the time to equal RMSE is the
    training time plus the first cached frame whose RMSE is at most the plain one."""
    import torch
    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import cache as RC, workloads as W
    st = torch.cuda.current_stream()
    W_, H_ = s.camera.width, s.camera.height
    npx, ref_spp = args.cache_ref_pixels, args.cache_ref_spp
    gen = torch.Generator().manual_seed(1234)
    pix = torch.randperm(W_ * H_, generator=gen)[:npx].to(dev)
    px, py = (pix % W_).int(), (pix // W_).int()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        out = fn()
        b.record(st)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    # reference: ref_spp samples per pixel from a sample range the frames do not use
    ref = torch.zeros(npx, dtype=torch.float64, device=dev)
    chunk = max(1, min(ref_spp, (1 << 24) // npx))
    ref_base = 1 << 20
    ref_ms = 0.0
    for s0 in range(0, ref_spp, chunk):
        k = min(chunk, ref_spp - s0)
        rx, ry = px.repeat_interleave(k), py.repeat_interleave(k)
        rs = (ref_base + s0 + torch.arange(k, device=dev, dtype=torch.int32)).repeat(npx)
        out, ms = timed(lambda: tv.tet_trace_paths(grid, s.camera, s.medium, s.render_seed, rx, ry, rs))
        ref += out["L"].view(npx, k).double().sum(1)
        ref_ms += ms
        del out, rx, ry, rs
    ref /= ref_spp

    def rmse(img, spp):
        m = img[py.long(), px.long()].double() / spp
        return float(torch.sqrt(torch.mean((m - ref) ** 2)))

    plain, _ = tv.tet_render(grid, s.camera, s.medium, s.spp, s.render_seed, 0)
    target = rmse(plain, s.spp)
    rel = float(torch.sqrt(torch.mean(ref ** 2)))
    res = {"reference": "%d spp at %d random pixels (plain tracer, samples from %d)" % (ref_spp, npx, ref_base),
           "reference_ms": round(ref_ms, 1), "rms_radiance": round(rel, 6),
           "plain": {"spp": s.spp, "ms": round(plain_ms, 2), "rmse": round(target, 6)}, "variants": []}

    def variant(rounds, depth, train_bounces=None, seed_k=0, survive=0.0, rfrom=0):
        # seed_k selects the initial weights and the training paths (their pixels and random streams)
        rc = RC.RadianceCache(W.mlp_init_params(1 + seed_k, b4=0.1), device=dev, lr=3e-3)
        _, train_ms = timed(lambda: rc.train(grid, s.camera, s.medium, s.render_seed + 7919 * seed_k, rounds=rounds,
                                             max_bounces=train_bounces, survive=survive, roulette_from=rfrom))
        curve, reached = [], None
        for spp in (1, 2, 4, 8, 16, 32):
            (img, _), ms = timed(lambda: rc.render(grid, s.camera, s.medium, spp, s.render_seed, depth))
            e = rmse(img, spp)
            curve.append({"spp": spp, "ms": round(ms, 2), "rmse": round(e, 6)})
            if reached is None and e <= target:
                reached = train_ms + ms
        return {"seed": seed_k, "train_ms": round(train_ms, 2), "adam_steps": rc.step,
                "final_train_loss": round(float(rc.loss[2]), 6), "curve": curve,
                "time_to_equal_rmse_ms": None if reached is None else round(reached, 2)}

    def seeds(rounds, depth, train_bounces=None, n=3, survive=0.0, rfrom=0):
        runs = [variant(rounds, depth, train_bounces, k, survive, rfrom) for k in range(n)]
        t = [r["time_to_equal_rmse_ms"] for r in runs]
        ok = sorted(x for x in t if x is not None)
        med = statistics.median(t) if len(ok) == len(t) else None
        return {"cache_depth": depth, "train_rounds": rounds, "train_samples_per_round": (1 << 14) * 4,
                "train_max_bounces": train_bounces or s.medium.max_bounces, "train_survive": survive,
                "train_roulette_from": rfrom,
                "seeds": len(runs),
                "reached": len(ok), "time_to_equal_rmse_ms_median": None if med is None else round(med, 2),
                "time_to_equal_rmse_ms_min": ok[0] if ok else None,
                "time_to_equal_rmse_ms_max": ok[-1] if len(ok) == len(t) else None,
                "speedup_vs_plain_median": None if med is None else round(plain_ms / med, 3), "runs": runs}

    # the headline: one configuration fixed before it was measured -- 8 training rounds of 2^16
    # vertex samples, paths ending into the cache at their first collision -- as the median of
    # 3 seeds.  The same with the training paths ended by Russian roulette (survival 1/2) after
    # their last training vertex was measured next, as a second fixed configuration: it trains
    # about 3x faster but its cache does not reach the plain frame's RMSE (reported, not the headline)
    def summary(v):
        out = {k: val for k, val in v.items() if k != "runs"}
        out["runs"] = [{"seed": r["seed"], "train_ms": r["train_ms"], "time_to_equal_rmse_ms": r["time_to_equal_rmse_ms"],
                        "rmse_at_32spp": r["curve"][-1]["rmse"]} for r in v["runs"]]
        return out
    fixed = seeds(8, 1)
    res["fixed_configuration"] = summary(fixed)
    fixed_rr = seeds(8, 1, survive=0.5)
    res["fixed_configuration_roulette"] = summary(fixed_rr)
    # A third configuration, fixed before its first measurement: the same roulette (survival 1/2)
    # played only from collision 16 (0-based) on, so that it cuts only the long tail of training
    # paths (3.1 collisions per path on average), which sets the training trace's time
    res["fixed_configuration_late_roulette"] = summary(seeds(8, 1, survive=0.5, rfrom=16))
    res["roulette_variants"] = [summary(seeds(8, 1, survive=0.75)), summary(seeds(32, 1, survive=0.5))]
    # the other training budgets and depths, for context (each the median of 3 seeds as well)
    for rounds in [int(r) for r in str(args.cache_train_rounds).split(",") if r]:
        for depth in (1, 2):
            v = fixed if (rounds, depth) == (8, 1) else seeds(rounds, depth)
            res["variants"].append({k: val for k, val in v.items() if k != "runs"})
    for tb in [int(b) for b in str(args.cache_train_bounces).split(",") if b]:
        for rounds in (4, 8):
            try:
                v = seeds(rounds, 1, tb)
            except Exception as exc:                      # noqa: BLE001
                res["variants"].append({"cache_depth": 1, "train_rounds": rounds, "train_max_bounces": tb,
                                        "error": str(exc)[:200]})
                continue
            res["variants"].append({k: val for k, val in v.items() if k != "runs"})
    # where training time goes: tracing the training paths, and the grad + Adam steps
    rc = RC.RadianceCache(W.mlp_init_params(1, b4=0.1), device=dev, lr=3e-3)
    n_tr = 32 << 14
    tx, ty, ts = RC.random_paths(77, n_tr, W_, H_, 1 << 24)
    buf, trace_ms = timed(lambda: RC.cache_samples(grid, s.camera, s.medium, s.render_seed, tx, ty, ts, 4))

    def steps():
        per = buf.shape[0] // 128
        for i in range(128):
            RC.mlp_grad(rc.params, buf[i * per:(i + 1) * per], rc.grad, rc.loss)
            rc.step += 1
            RC.adam(rc.params, rc.m, rc.v, rc.grad, rc.loss, rc.step, rc.lr)
    _, steps_ms = timed(steps)
    res["train_phases"] = {"trace_paths": n_tr, "trace_ms": round(trace_ms, 2), "steps": 128,
                           "samples_per_step": buf.shape[0] // 128, "steps_ms": round(steps_ms, 2)}
    res["mlp_kernels"] = mlp_kernel_rates(dev)
    med = fixed["time_to_equal_rmse_ms_median"]
    res["time_to_equal_rmse_ms"] = med
    res["speedup_vs_plain"] = None if med is None else round(plain_ms / med, 3)
    res["headline"] = "fixed configuration (8 rounds, cache depth 1), median of 3 training seeds"
    res["timeouts"] = RC.timeouts()
    return res


def mlp_kernel_rates(dev):
    """The fused tensor-core MLP kernels alone (CUDA events, through the public API) at
    the cache leg's sizes: one training step of 2^14 samples (and 2^18), and inference
    over 2^20 records (one 1024^2 cached frame at 1 spp) and 2^22; FLOPs per record
    2 (128*64 + 2*64*64) forward, three times that with the backward pass."""
    import torch
    from paper_2506_11510_gb300 import cache as RC, workloads as W
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak = float(json.load(fh)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        peak = 1900.0
    st = torch.cuda.current_stream()
    p = torch.from_numpy(W.mlp_init_params(1, b4=0.1)).to(dev)
    fwd = 2 * (128 * 64 + 2 * 64 * 64)
    out = {"bf16_peak_tflops": peak, "grad": [], "infer": []}

    def timed(fn, reps):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e3 / reps

    for n in (1 << 14, 1 << 18):
        rec = torch.from_numpy(W.mlp_random_records(n, 3)).to(dev)
        rec[:, 7] = 1.0
        g = torch.zeros_like(p)
        loss = torch.zeros(3, dtype=torch.float32, device=dev)
        us = timed(lambda: RC.mlp_grad(p, rec, g, loss), 20)
        tf = n * 3 * fwd / (us * 1e-6) / 1e12
        out["grad"].append({"samples": n, "us": round(us, 1), "tflops": round(tf, 1), "frac": round(tf / peak, 4)})
    for n in (1 << 20, 1 << 22):
        rec = torch.from_numpy(W.mlp_random_records(n, 4)).to(dev)
        y = torch.empty(n, dtype=torch.float32, device=dev)
        us = timed(lambda: RC.mlp_infer(p, rec, y), 10)
        tf = n * fwd / (us * 1e-6) / 1e12
        out["infer"].append({"records": n, "us": round(us, 1), "tflops": round(tf, 1), "frac": round(tf / peak, 4)})
    return out


# ---------------------------------------------------------------------------
# the oracle (CPU) on a bounded sample of the workload
# ---------------------------------------------------------------------------
def oracle_window(s, vol_np, side, nthreads=0):
    """The oracle's grid for a side x side pixel window at the centre of the frame:
    the camera criterion refines the window's sub-frustum only, so outside it the
    grid stays coarse (cheaper paths than the full frame's).  Returns the grid,
    the window camera and the build time."""
    import oracle as O
    from paper_2506_11510_gb300 import workloads as W
    cam = s.camera
    frac = side / cam.height
    fov = 2 * math.degrees(math.atan(math.tan(math.radians(cam.fov_y_deg) / 2) * frac))
    wcam = W.Camera(cam.pos, cam.target, cam.up, fov, side, side)
    t0 = time.time()
    g = O.Grid.for_scene(s, vol_np, camera=wcam, nthreads=nthreads)
    return g, wcam, time.time() - t0


def oracle_window_render(s, g, wcam, min_seconds=10.0, nthreads=0):
    """The window's paths at the frame's spp, repeated over further sample ranges
    until at least min_seconds have passed (at most 256 frames); returns (paths, seconds)."""
    import numpy as np
    side = wcam.width
    py, px, sm = np.meshgrid(np.arange(side), np.arange(side), np.arange(s.spp), indexing="ij")
    px, py, sm = px.ravel(), py.ravel(), sm.ravel()
    t0 = time.time()
    paths, k, steps = 0, 0, 0
    while k < 256:
        r = g.render_paths(wcam, s.medium, s.render_seed, px, py, sm + k * s.spp, nthreads=nthreads)
        paths += len(px)
        steps += int(r["steps"].sum())
        k += 1
        if time.time() - t0 >= min_seconds:
            break
    oracle_window_render.steps = steps
    return paths, time.time() - t0


def cpu_sample_text(side, s, paths, tb):
    grid = ("on the oracle's grid refined for the window's sub-frustum only (coarse elsewhere, so paths are "
            "cheaper than the full frame's" if s.footprint_px > 0 else
            "on the oracle's grid (the same grid as the full frame's: no camera criterion")
    return ("%dx%d-pixel window at the frame centre, %d spp per frame, %d paths over successive sample ranges, "
            "%s; built once in %.0f s, not timed); fp64 C++, OpenMP over paths"
            % (side, side, s.spp, paths, grid, tb))


def cpu_baseline(args, s, vol, dev=None):
    """The oracle on a bounded sample: the frame's central window on the oracle's
    grid for that window, timed on all host cores and on one core.  This leg is
    also where the GPU path's results on that window are compared with the fp64
    oracle (the oracle runs nowhere else in the benchmark): the GPU grid of the
    window against the oracle's, per-path estimates, the storage error of BF16
    and FP16 densities against FP32 densities, and the 4096-spp reference
    procedure of the cache leg."""
    vol_np = vol.cpu().numpy() if hasattr(vol, "cpu") else vol
    cores = os.cpu_count() or 1
    side = args.cpu_sample_px or 64
    g, wcam, tb = oracle_window(s, vol_np, side)
    paths, tr = oracle_window_render(s, g, wcam)
    steps = oracle_window_render.steps
    p1, t1 = oracle_window_render(s, g, wcam, min_seconds=5.0, nthreads=1)
    steps1 = oracle_window_render.steps
    out = {"value": round(paths / tr / 1e6, 5), "unit": "Mpaths/s", "cores": cores, "kind": "oracle",
           "sample": cpu_sample_text(side, s, paths, tb), "render_s": round(tr, 2),
           "tet_steps_per_path": round(steps / paths, 1), "g_tet_steps_per_s": round(steps / tr / 1e9, 4),
           "single_thread": {"value": round(p1 / t1 / 1e6, 5), "unit": "Mpaths/s", "cores": 1, "paths": p1,
                             "render_s": round(t1, 2), "g_tet_steps_per_s": round(steps1 / t1 / 1e9, 4)},
           "window_build_s": round(tb, 1)}
    if dev is not None:
        out["oracle_checks"] = oracle_checks(s, vol, vol_np, g, wcam)
    return out


def oracle_checks(s, vol, vol_np, g_orc, wcam):
    """GPU against the fp64 oracle on the central window of the production frame."""
    import dataclasses
    import numpy as np
    import torch
    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import workloads as W
    import oracle as O
    side = wcam.width
    ws = W.with_camera(s, fov_y_deg=wcam.fov_y_deg, width=side, height=side)
    res = {"window": "central %dx%d pixels of the frame (the frame's camera, field of view narrowed)" % (side, side)}
    # the GPU build of the window grid against the oracle's
    gw = tv.build_scene_grid(ws, vol)
    a = g_orc.export()
    e = gw.export(("codes", "nbr", "density", "plane"))
    same = (len(a.codes) == e["codes"].shape[0]
            and np.array_equal(e["codes"].cpu().numpy().view(np.uint64), a.codes)
            and np.array_equal(e["nbr"].cpu().numpy(), a.nbr) and np.array_equal(e["density"].cpu().numpy(), a.density)
            and np.array_equal(e["plane"].cpu().numpy(), a.plane))
    res["grid"] = {"tets": int(len(a.codes)), "depth": int(a.max_depth), "gpu_equals_oracle": bool(same)}
    # per-path estimates, BF16 grid, the frame's medium
    rng = np.random.default_rng(77)
    n = 8192
    px = rng.integers(0, side, n).astype(np.int32)
    py = rng.integers(0, side, n).astype(np.int32)
    sm = rng.integers(0, s.spp, n).astype(np.int32)
    got = tv.tet_trace_paths(gw, ws.camera, ws.medium, ws.render_seed, px, py, sm)
    want = g_orc.render_paths(ws.camera, ws.medium, ws.render_seed, px, py, sm)
    Lg, Lo = got["L"].cpu().numpy().astype(np.float64), want["L"]
    rel = np.abs(Lg - Lo) / np.maximum(np.abs(Lo), 1e-6)
    d = Lg - Lo
    res["paths"] = {"n": n, "frac_within_1e-4": round(float(np.mean(rel <= 1e-4)), 5),
                    "rel_err_p50": float(np.percentile(rel, 50)), "rel_err_p99_9": float(np.percentile(rel, 99.9)),
                    "rel_err_max": float(rel.max()),
                    "collisions_equal_frac": round(float(np.mean(got["collisions"].cpu().numpy() ==
                                                                 want["collisions"])), 5),
                    "mean_diff_over_3se": round(float(abs(d.mean()) / (3 * d.std() / math.sqrt(n) + 1e-30)), 4)}
    # storage error: BF16 and FP16 densities against FP32 densities, all on the fp64 oracle
    py2, px2, sm2 = np.meshgrid(np.arange(side), np.arange(side), np.arange(s.spp), indexing="ij")
    px2, py2, sm2 = px2.ravel().astype(np.int32), py2.ravel().astype(np.int32), sm2.ravel().astype(np.int32)
    imgs = {}
    for fmt, name in ((0, "fp32"), (1, "bf16"), (2, "fp16")):
        gf = g_orc if fmt == s.density_format else O.Grid.for_scene(dataclasses.replace(ws, density_format=fmt),
                                                                    vol_np)
        imgs[name] = gf.render_paths(ws.camera, ws.medium, ws.render_seed, px2, py2, sm2)["L"]
        del gf
    ref = imgs["fp32"].reshape(side * side, s.spp).mean(1)
    rms = float(np.sqrt(np.mean(ref ** 2)))
    se = float(np.sqrt(np.mean(imgs["fp32"].reshape(side * side, s.spp).var(1, ddof=1) / s.spp)))
    st = {"image": "%dx%d window at %d spp, fp64 oracle; errors relative to the FP32-density image's RMS %.5f"
                   % (side, side, s.spp, rms), "monte_carlo_se_rel": round(se / rms, 5)}
    for name in ("bf16", "fp16"):
        img = imgs[name].reshape(side * side, s.spp).mean(1)
        dd = imgs[name] - imgs["fp32"]
        st[name] = {"pixel_rms_rel": round(float(np.sqrt(np.mean((img - ref) ** 2)) / rms), 6),
                    "pixel_max_rel": round(float(np.max(np.abs(img - ref)) / rms), 6),
                    "image_mean_rel": round(float((img.mean() - ref.mean()) / ref.mean()), 6),
                    "image_mean_diff_over_3se": round(float(abs(dd.mean()) / (3 * dd.std() / math.sqrt(dd.size)
                                                                               + 1e-30)), 4),
                    "paths_equal_frac": round(float(np.mean(imgs[name] == imgs["fp32"])), 5)}
    res["storage_vs_fp32"] = st
    # the cache leg's reference procedure (GPU trace of 4096 samples from 2^20 on) at 64 window pixels
    npx, rspp, base = 64, 4096, 1 << 20
    pix = rng.choice(side * side, npx, replace=False)
    rx = np.repeat(pix % side, rspp).astype(np.int32)
    ry = np.repeat(pix // side, rspp).astype(np.int32)
    rs = np.tile(base + np.arange(rspp), npx).astype(np.int32)
    gm = tv.tet_trace_paths(gw, ws.camera, ws.medium, ws.render_seed, rx, ry, rs)["L"].cpu().numpy()
    om = g_orc.render_paths(ws.camera, ws.medium, ws.render_seed, rx, ry, rs)["L"]
    gmean, omean = gm.astype(np.float64).reshape(npx, rspp).mean(1), om.reshape(npx, rspp).mean(1)
    rr = np.abs(gmean - omean) / np.maximum(np.abs(omean), 1e-6)
    res["cache_reference_check"] = {"pixels": npx, "spp": rspp,
                                    "frac_within_1e-4": round(float(np.mean(rr <= 1e-4)), 4),
                                    "rel_err_max": float(rr.max())}
    del gw
    torch.cuda.empty_cache()
    return res


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2506_11510_gb300 import workloads as W
    s = W.scene(args.scene)
    try:
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
    except Exception:
        dev = "cpu"
    vol = W.make_volume(s, device=dev).cpu().numpy()
    side = args.cpu_sample_px or 64
    g, wcam, tb = oracle_window(s, vol, side)
    for _ in range(args.warmup):
        oracle_window_render(s, g, wcam, min_seconds=0.0)
    times, counts, nsteps = [], [], 0
    for _ in range(max(1, args.steps)):
        paths, tr = oracle_window_render(s, g, wcam, min_seconds=5.0)
        times.append(tr)
        counts.append(paths)
        nsteps += oracle_window_render.steps
    mean = sum(times) / len(times)
    value = sum(counts) / sum(times) / 1e6
    cores = os.cpu_count() or 1
    line = {"metric": METRIC, "value": round(value, 5), "unit": "Mpaths/s", "n_gpus": ws, "steps": len(times),
            "warmup": args.warmup, "ms_per_step": round(mean * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_name(s),
                       "ms_per_frame_extrapolated": round(s.camera.width * s.camera.height * s.spp / value / 1e3, 1),
                       "sample": "the CPU oracle on a %dx%d-pixel window of the frame" % (side, side)},
            "cpu_baseline": {"value": round(value, 5), "unit": "Mpaths/s", "cores": cores, "kind": "oracle",
                             "sample": cpu_sample_text(side, s, paths, tb),
                             "tet_steps_per_path": round(nsteps / sum(counts), 1),
                             "g_tet_steps_per_s": round(nsteps / sum(times) / 1e9, 4)},
            "e2e": {"value": round(value, 5), "unit": "Mpaths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mlp_kernels_only:
        import torch
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        torch.cuda.set_device(dev)
        print(json.dumps({"mlp_kernels": mlp_kernel_rates(dev)}))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
