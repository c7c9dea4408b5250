#!/usr/bin/env python3
"""Benchmark of multi-depth ray casting + sensor model (Sec. 3.2.2, Algorithm 1, Appendix A.2).

Variants (``--variant``):
  plain      4096 envs x 2 cameras x 64x48 px, 20.48M-triangle terrain, 30 links of 512 triangles,
             sensor on (0.01 m noise, 2 % dropout, latency 0-3), binary BVH, FP32 depth (default);
  precision  the same with the eight-wide BVH of 8-bit quantised boxes and FP16 depth;
  batching   4096 envs x 4 uneven cameras (80x60, 80x60, 48x36, 48x36) in one launch, replayed as a
             CUDA graph of the whole path;
  perception the paper's perception settings: 4096 envs x 2 cameras ray cast at 240x135 and averaged
             to 48x27 (101 x 69 deg FOV), per-env camera pose and FOV randomisation, side masking by
             terrain kind, sensor preset sigma = 0.1 depth, 5 % dropout, latency 0-3;
  serving    Poisson request streams from 4 trainers through the continuous-batching server;
  table1     the paper's Table 1 setting (1024 envs, 240x135, 1 / 2 / 4 cameras): time per render
             and device memory per camera count.
One step = the whole path over all envs with the next resident pose set: rpl_render (prep, tile-prep and render
kernels), or one graph replay for ``batching``.  The launch shape is chosen by the library's
autotuner before timing.  Rank 0 prints one JSON line.  ``--impl reference`` times the FP64 CPU
oracle instead on a bounded sample of the same workload.

Multi-GPU (torchrun): each rank renders its own 4096 envs (env_offset = rank * envs) with no
data-path collective; the barrier and the max-over-ranks time only bracket the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Grays/s and depth frames/s at 4096 envs; serve p50/p99 latency vs plain FP32"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# ncu counters of single render_kernel launches of the bench's own workloads (full size, no scaling)
COUNTERS = os.path.join(ROOT, "profiles", "render_kernel_counters.json")
SMSP_PER_SM = 4   # warp schedulers per SM, each issuing at most one warp instruction per cycle
TRI_BYTES, BOX_BYTES = 48, 32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default="plain",
                    choices=["plain", "precision", "batching", "perception", "serving", "table1"])
    ap.add_argument("--envs", type=int, default=4096)
    ap.add_argument("--tiles", type=int, default=20)
    ap.add_argument("--pose-sets", type=int, default=8)
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch shape")
    ap.add_argument("--autotune", action="store_true",
                    help="plain variant: run the library's autotuner instead of its default launch shape")
    ap.add_argument("--no-serve", action="store_true", help="leave out the serving measurement")
    ap.add_argument("--serve-requests", type=int, default=400, help="requests per form in the serve object")
    ap.add_argument("--tuning", default=None,
                    help="fixed launch shape tile_w,tile_h,persistent,terrain_first,min_blocks[,env_order,chunk_tiles] "
                         "(skips the autotuner)")
    ap.add_argument("--bvh", type=int, default=None, choices=[2, 4, 8],
                    help="terrain BVH layout: 2 binary, 4 four-wide FP32, 8 eight-wide quantised "
                         "(default: 8 for precision, else 2)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU work of the oracle sample")
    return ap.parse_args()


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload(args, rank):
    from paper_2602_03002_gb300 import workloads as W
    if args.variant == "batching":
        return W.config_uneven(n_steps=args.pose_sets, n_envs=args.envs, tiles=args.tiles, seed=rank)
    if args.variant == "perception":
        return W.config_perception(n_steps=args.pose_sets, n_envs=args.envs, tiles=args.tiles, seed=rank)
    if args.variant == "table1":
        return W.config_perception(n_steps=args.pose_sets, n_envs=1024, tiles=args.tiles, seed=rank)
    w = W.config_scale(n_steps=args.pose_sets, n_envs=args.envs, tiles=args.tiles, seed=rank)
    if args.variant == "precision":
        w.sensor.out_dtype = 1
    return w


def bvh_number(args):
    if args.bvh is not None:
        return args.bvh
    return 8 if args.variant == "precision" else 2


def bvh_kind(args, rpl):
    return {2: rpl.RPL_BVH2, 4: rpl.RPL_BVH4, 8: rpl.RPL_BVH8Q8}[bvh_number(args)]


BVH_NAMES = {2: "binary BVH", 4: "four-wide FP32 BVH", 8: "eight-wide BVH with 8-bit quantised boxes"}


def workload_name(w, variant, bvh):
    cams = " + ".join("%dx%d" % (c.width, c.height) + ("->%dx%d" % (c.out_width, c.out_height) if c.downsample > 1 else "")
                      for c in w.cameras)
    s = w.sensor
    sensor = ("sensor sigma %.2f m + %.2f depth, %.0f%% dropout, latency 0-%d steps"
              % (s.sigma_abs, s.sigma_rel, 100 * s.p_drop, s.max_latency) if s.enabled else "no sensor model")
    form = BVH_NAMES[bvh] + ", " + {
        "plain": "FP32 depth", "precision": "FP16 depth",
        "batching": "FP32 depth, one CUDA-graph replay per step",
        "perception": "FP32 depth, raw images block-averaged before the sensor, per-env camera pose/FOV "
                      "randomisation, side masking (cols %s by mode)" % (tuple(w.rsm_cols),),
        "table1": "FP32 depth, the paper's Table 1 setting (1024 envs, 240x135 averaged to 48x27)",
        "serving": "FP32 depth, requests served by the continuous-batching server"}[variant]
    return ("%s: %d envs x cams (%s px); terrain %d tris (tiles of 8x8 m at 0.05 m: stairs 0.22/0.25/0.30 m run, "
            "20 deg slopes, stepping stones); %d links x %d-tri meshes; %s; %s"
            % (variant, w.n_envs, cams, len(w.terrain_tris), w.n_links, len(w.link_tris[0]), sensor, form))


def peaks():
    try:
        with open(PEAKS) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash():
    """Hash of the kernel sources with line comments and blank lines removed, so that a change of
    comments alone keeps a traffic capture valid."""
    h = hashlib.sha256()
    for f in ("render.cu", "render.h", "bvh.h", "bvh4.h", "bvh8.h"):
        with open(os.path.join(ROOT, "paper_2602_03002_gb300", "csrc", f), encoding="utf-8") as fh:
            for line in fh:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def counters_for_launch(rays, variant, tuning, bvh):
    """The committed ncu counters of one render_kernel launch of exactly this workload: same kernel
    source hash, variant, terrain BVH layout, launch shape and rays per launch (no scaling).  None
    when no capture matches (the kernel or the workload changed since the counters were taken)."""
    try:
        with open(COUNTERS) as f:
            entries = json.load(f)["captures"]
    except Exception:
        return None
    sha = kernel_hash()
    for t in entries:
        if (t.get("kernel_sha") == sha and t.get("variant") == variant and t.get("tuning") == tuning
                and t.get("bvh", 2) == bvh and int(t.get("rays", -1)) == int(rays)):
            return t
    return None


def l2_read_gbs(dev):
    """L2 read bandwidth: one reduction kernel that reads a 32 MiB buffer 64 times (row sums of a
    stride-0 view, rows spread over the SMs, so the re-reads come from L2, not L1), bytes read over
    the best of 10 launches (torch's reduction kernel, CUDA events; 2 GiB per launch, so launch
    overhead does not count).  The L2 counterpart of the HBM copy peak; a lower bound on what L2 can
    deliver, since a reduction kernel is measured, not the hardware's limit."""
    import torch
    n, rows = 8 << 20, 64                               # float32 elements in 32 MiB, passes over them
    a = torch.rand(n, device=f"cuda:{dev}")
    v = a.as_strided((rows, n), (0, 1))
    for _ in range(3):
        v.sum(dim=1)
    best = float("inf")
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        v.sum(dim=1)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return rows * 4 * n / best / 1e9


def roofline(ctr, k_s, alg_bytes, rays, sms, clock_mhz, l2_peak, cnt):
    """Roofline of the render kernel against the resource that binds.  From the committed counters of
    this launch: DRAM bytes against the measured HBM copy peak, L2 bytes against the L2 read bandwidth
    measured in this run, and warp instructions against the issue capacity (SMs x 4 schedulers x the
    SM clock sampled during the timed region), each divided by the launch's CUDA-event time.  `bound`
    names the highest of the three fractions and the top-level figures are that resource's.  The
    traversal's fetch bytes per ray (nodes, triangles, link boxes; counting kernel) are kept as
    fetch_bytes_per_ray: most of them are served by L1/L2, so they are not an HBM figure."""
    hbm_peak, hbm_src = peaks()
    out = {"kernel": "render_kernel", "kernel_ms": 1e3 * k_s,
           "fetch_bytes_per_ray": alg_bytes / rays,
           "fetch_note": "node (64 B), triangle (48 B) and link-box (32 B) fetches of the traversal per ray plus "
                         "its output and ring bytes, from the counting kernel; most are L1/L2 hits",
           "per_ray": {k: cnt[k] / rays for k in ("terrain_nodes", "terrain_tris", "link_boxes",
                                                  "link_nodes", "link_tris")}}
    if ctr is None:
        out.update({"bound": None, "achieved": None, "peak": hbm_peak, "unit": "GB/s", "frac": None,
                    "traffic": None, "counters": "no committed ncu capture of this kernel source, workload and "
                                                 "launch shape"})
        return out
    issue_peak = sms * SMSP_PER_SM * clock_mhz * 1e6
    res = {
        "hbm": {"achieved": ctr["dram_bytes"] / k_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "peak_source": hbm_src + " hbm_gbs (copy)"},
        "l2": {"achieved": ctr["lts_bytes"] / k_s / 1e9, "peak": l2_peak, "unit": "GB/s",
               "peak_source": "measured in this run: L2 read bandwidth of a reduction that reads a 32 MiB "
                              "buffer 64 times in one launch"},
        "issue": {"achieved": ctr["inst_executed"] / k_s / 1e9, "peak": issue_peak / 1e9,
                  "unit": "G warp-instructions/s",
                  "peak_source": "%d SMs x %d schedulers x %.0f MHz (SM clock sampled during the timed region)"
                                 % (sms, SMSP_PER_SM, clock_mhz)},
    }
    for v in res.values():
        v["frac"] = v["achieved"] / v["peak"] if v["peak"] else None
    bound = max(res, key=lambda k: res[k]["frac"] or 0.0)
    out.update({"bound": bound, "achieved": res[bound]["achieved"], "peak": res[bound]["peak"],
                "unit": res[bound]["unit"], "frac": res[bound]["frac"], "traffic": ctr["dram_bytes"],
                "hbm": res["hbm"], "l2": res["l2"], "issue": res["issue"],
                "counters": {"source": "ncu (--clock-control none) on one launch of this workload and launch "
                                       "shape; committed in profiles/render_kernel_counters.json",
                             "dram_bytes": ctr["dram_bytes"], "lts_bytes": ctr["lts_bytes"],
                             "inst_executed": ctr["inst_executed"],
                             "warps_active_pct": ctr.get("warps_active_pct"),
                             "issue_active_pct": ctr.get("issue_active_pct")}})
    return out


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def sample_rays(w, n, rng):
    """n output pixels (env, camera, x, y) drawn uniformly."""
    c = rng.integers(0, len(w.cameras), n)
    wd = np.array([cam.out_width for cam in w.cameras])[c]
    ht = np.array([cam.out_height for cam in w.cameras])[c]
    x = (rng.random(n) * wd).astype(np.int64)
    y = (rng.random(n) * ht).astype(np.int64)
    return np.stack([rng.integers(0, w.n_envs, n), c, x, y], 1).astype(np.int64)


def cpu_baseline(w, seconds, gpu_step0=None, sc=None, single_core=True):
    """The FP64 oracle, as it stands, on a bounded sample of rays of step 0 of the same workload.  When
    the GPU's step-0 frame is given, the sample also yields the GPU's error against the oracle.  `sc`
    reuses an oracle scene across calls; single_core adds a one-thread slice of the sample."""
    import oracle
    cores = os.cpu_count() or 1
    own = sc is None
    if own:
        sc = oracle.OracleScene.from_workload(w)
    rng = np.random.default_rng(1234)
    extra = dict(per_env_intrinsics=w.per_env_intrinsics, mount_dr=w.mount_delta, rsm_mode=w.rsm_modes,
                 rsm_cols=w.rsm_cols, flags=False, threads=cores)
    t = time.perf_counter()
    sc.render(w.cameras, w.poses, 0, sample_rays(w, cores, rng), w.sensor, **extra)
    probe = time.perf_counter() - t
    n = max(cores, int(cores * seconds / max(probe, 1e-3)))
    rays = sample_rays(w, n, rng)
    t = time.perf_counter()
    ref = sc.render(w.cameras, w.poses, 0, rays, w.sensor, **extra)
    dt = time.perf_counter() - t
    per_px = np.array([max(1, c.downsample) ** 2 for c in w.cameras])
    n_rays = int(per_px[rays[:, 1]].sum())           # a downsampled pixel costs f^2 ray casts
    rate = n_rays / dt
    out = {"value": rate / 1e9, "unit": "Grays/s", "cores": cores, "kind": "oracle",
           "sample": "%d output pixels (%d ray casts) drawn uniformly over (env, camera, pixel) of step 0, FP64 "
                     "brute force over all triangles, %.1f s" % (n, n_rays, dt),
           "full_step_s_extrapolated": w.rays_per_step / rate}
    if single_core:
        # one core, on a small slice of the same sample (about a tenth of the all-core time)
        one = rays[:max(1, int(n * 0.1 / cores))]
        t = time.perf_counter()
        sc.render(w.cameras, w.poses, 0, one, w.sensor, **dict(extra, threads=1))
        dt1 = time.perf_counter() - t
        out["single_core_value"] = int(per_px[one[:, 1]].sum()) / dt1 / 1e9
        out["single_core_sample"] = "%d output pixels of the same sample on one thread, %.1f s" % (len(one), dt1)
    if own:
        sc.close()
    if gpu_step0 is not None:
        offs = w.cam_offsets()
        cw = np.array([c.out_width for c in w.cameras])
        got = gpu_step0[rays[:, 0], offs[rays[:, 1]] + rays[:, 3] * cw[rays[:, 1]] + rays[:, 2]]
        if w.sensor.out_dtype == 2:
            got = got * (w.cameras[0].d_max / 65535.0)
        err = np.abs(got.astype(np.float64) - ref["depth"])
        allow = 1e-4 + (np.spacing(np.abs(ref["depth"]).astype(np.float16)).astype(np.float64) / 2
                        if w.sensor.out_dtype == 1 else 0.0)
        out["error_vs_oracle"] = {"rays": int(n), "max_abs_m": float(err.max()),
                                  "p99_abs_m": float(np.quantile(err, 0.99)), "mean_abs_m": float(err.mean()),
                                  "mismatch_frac": float(np.mean(err > allow)),
                                  "allowance_m": "1e-4" + (" + half an FP16 ulp" if w.sensor.out_dtype == 1 else "")}
    return n_rays, dt, cores, out


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    w = workload(args, 0)
    n_tot = dt_tot = 0
    cores = os.cpu_count() or 1
    import oracle
    sc = oracle.OracleScene.from_workload(w)
    cb = {}
    for k in range(args.warmup + args.steps):
        last = k == args.warmup + args.steps - 1
        n, dt, cores, cb = cpu_baseline(w, max(1.0, args.cpu_seconds / max(1, args.steps)), sc=sc, single_core=last)
        if k >= args.warmup:
            n_tot += n
            dt_tot += dt
    sc.close()
    rate = n_tot / dt_tot
    sample = "%d ray casts per step for output pixels drawn uniformly over (env, camera, pixel), brute force over all %d triangles" % (
        n_tot // max(1, args.steps), len(w.terrain_tris) + sum(len(t) for t in w.link_tris))
    line = {"impl": "reference", "metric": METRIC, "value": rate / 1e9, "unit": "Grays/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt_tot / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(w, args.variant, bvh_number(args))},
            "frames_per_s": rate / (w.raw_pixels_per_env / len(w.cameras)),
            "e2e": {"value": rate / 1e9, "unit": "Grays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": rate / 1e9, "unit": "Grays/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "single_core_value": cb.get("single_core_value"),
                             "full_step_s_extrapolated": w.rays_per_step / rate}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = local if torch.cuda.is_available() else 0
    torch.cuda.set_device(dev)
    from paper_2602_03002_gb300 import build as B, rpl
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    w = workload(args, rank)
    env_offset = rank * args.envs
    kind = bvh_kind(args, rpl)
    free0 = torch.cuda.mem_get_info(dev)[0]
    t0 = time.perf_counter()
    scene = rpl.Scene(w.terrain_verts, w.terrain_tris, device=dev, bvh_kind=kind)
    for l, (v_, t_) in enumerate(zip(w.link_verts, w.link_tris)):
        scene.add_link(l, v_, t_)
    build_s = time.perf_counter() - t0
    free1 = torch.cuda.mem_get_info(dev)[0]
    view = rpl.View.from_workload(scene, w)
    free2 = torch.cuda.mem_get_info(dev)[0]
    vram = {"scene_gb": (free0 - free1) / 1e9, "view_gb": (free1 - free2) / 1e9,
            "note": "device memory taken by the library's scene (BVHs) and view (transforms, ring, raw and "
                    "staging buffers), from cudaMemGetInfo around their creation"}
    info = scene.info()
    stream = torch.cuda.Stream(dev)
    poses = torch.from_numpy(w.poses).to(f"cuda:{dev}")
    out = view.out_tensor(torch.device("cuda", dev))
    # poses and out come from the default stream's memory pool; the side stream waits for that stream
    stream.wait_stream(torch.cuda.current_stream(dev))
    rays = w.rays_per_step
    graph = args.variant == "batching"

    # launch shape first: the counted traversal below then takes the order and tiles that are timed.
    # The variants keep the library's default shape (the fastest of the autotuner's sweep on the scale
    # workload) unless --autotune is given, so that their launch matches the committed ncu counters;
    # the batching configuration runs the autotuner, which is part of it.
    tuning, tune_ms = rpl.rpl_view_tuning_get(view.h), None
    tuning_source = "library default"
    if args.tuning:
        rpl.rpl_view_tuning_set(view.h, *(int(v) for v in args.tuning.split(",")))
        tuning = rpl.rpl_view_tuning_get(view.h)
        tuning_source = "--tuning"
    elif not args.no_autotune and (args.variant == "batching" or args.autotune):
        with torch.cuda.stream(stream):
            tuning, tune_ms = rpl.rpl_view_autotune(view.h, poses[0], 0, env_offset, out, stream, 3)
        tuning_source = "autotuner (192 shapes, 3 renders each)"
    # traversal counters (untimed, step 0, the chosen launch shape): algorithmic fetch bytes per ray
    with torch.cuda.stream(stream):
        cnt = view.render_counters(poses[0], 0, env_offset, out, stream)
    stream.synchronize()
    gpu_step0 = out.float().cpu().numpy() if out.dtype != torch.uint16 else out.cpu().numpy().astype(np.float32)
    node_bytes = {rpl.RPL_BVH2: 64, rpl.RPL_BVH8Q8: 80, rpl.RPL_BVH4: 128}[kind]
    b_nodes = cnt["terrain_nodes"] * node_bytes + cnt["link_nodes"] * 64
    b_tris = (cnt["terrain_tris"] + cnt["link_tris"]) * TRI_BYTES
    b_boxes = cnt["link_boxes"] * BOX_BYTES
    # compulsory traffic of the render kernel: per output ray the store, ring write and (k > 0) ring
    # read; per ray of a downsampled camera the raw-depth store (the downsample kernel does the rest)
    out_b = out.element_size()
    raw_rays = w.n_envs * sum(c.width * c.height for c in w.cameras if c.downsample > 1)
    b_io = (rays - raw_rays) * (out_b + (8 if w.sensor.max_latency > 0 else 0)) + raw_rays * 4
    alg_bytes = b_nodes + b_tris + b_boxes + b_io

    view.reset(None, 0)
    S = poses.shape[0]
    pose_buf = poses[0].clone()
    step = 0

    def one_step(s):
        if graph:
            pose_buf.copy_(poses[s % S])
            rpl.rpl_render_graph(view.h, pose_buf, env_offset, out, stream)
        else:
            rpl.rpl_render(view.h, poses[s % S], s, env_offset, out, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step(step)
            step += 1
    stream.synchronize()
    rpl.rpl_view_timing(view.h, True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        start.record(stream)
        for _ in range(args.steps):
            one_step(step)
            step += 1
        end.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = start.elapsed_time(end)
    kms = rpl.rpl_view_kernel_ms(view.h, min(args.steps, 256))
    rpl.rpl_view_timing(view.h, False)
    view.sync()
    if world > 1:
        t = torch.tensor([ms], device=f"cuda:{dev}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    value = world * rays / (ms_step / 1e3) / 1e9
    frames = world * w.n_envs * len(w.cameras) / (ms_step / 1e3)

    # end to end through the C ABI with host buffers (pinned): H2D poses, render, D2H depth
    e2e = None
    if not args.no_e2e:
        hp = [torch.from_numpy(w.poses[s]).pin_memory() for s in range(S)]
        ho = torch.empty(tuple(out.shape), dtype=out.dtype).pin_memory()
        # host copies of the depth run on the view's copy stream, overlapped with the next render;
        # the timed region ends after rpl_sync, i.e. after every step's copy has landed
        rpl.rpl_view_host_async(view.h, True)
        for _ in range(2):
            rpl.rpl_render(view.h, hp[step % S], step, env_offset, ho, stream)
            step += 1
        view.sync()
        if world > 1:
            torch.distributed.barrier()
        t = time.perf_counter()
        n_e2e = max(3, args.steps // 2)
        for _ in range(n_e2e):
            rpl.rpl_render(view.h, hp[step % S], step, env_offset, ho, stream)
            step += 1
        view.sync()
        e2e_s = (time.perf_counter() - t) / n_e2e
        rpl.rpl_view_host_async(view.h, False)
        if world > 1:
            tt = torch.tensor([e2e_s], device=f"cuda:{dev}")
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            e2e_s = float(tt.item())
        e2e = {"value": world * rays / e2e_s / 1e9, "unit": "Grays/s",
               "h2d_bytes_per_step": int(hp[0].numel() * 4), "d2h_bytes_per_step": int(ho.numel() * ho.element_size()),
               "ms_per_step": 1e3 * e2e_s, "steps": n_e2e,
               "host_copies": "pinned; depth copied on the view's copy stream while the next step renders "
                              "(rpl_view_host_async); timed on the host clock until rpl_sync"}

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    k_avg_s = statistics.mean(kms) / 1e3 if kms else ms_step / 1e3
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clock_mhz = ck.get("sm_mhz") or ck.get("sm_max_mhz") or 2070.0
    ctr = counters_for_launch(rays, args.variant, tuning, bvh_number(args))
    roof = roofline(ctr, k_avg_s, alg_bytes, rays, sms, clock_mhz, l2_read_gbs(dev), cnt)
    roof["kernel_ms_source"] = ("CUDA events around each render launch" if kms else
                                "whole graph replay (events cannot be recorded inside the graph)")
    line = {
        "metric": METRIC, "value": value, "unit": "Grays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "f32", 1: "f32 (f16 output)", 2: "f32 (unorm16 output)"}[w.sensor.out_dtype],
        "data": "synthetic", "variant": args.variant,
        "config": {"workload": workload_name(w, args.variant, bvh_number(args)), "envs_per_gpu": w.n_envs,
                   "cameras": len(w.cameras), "bvh": BVH_NAMES[bvh_number(args)],
                   "rays_per_step_per_gpu": rays, "pose_sets": S, "tuning": tuning,
                   "tuning_source": tuning_source, "autotune_best_ms": tune_ms,
                   "l2": "inputs larger than L2: terrain BVH %.2f GB resident, new poses each step"
                         % (info["terrain_bytes"] / 1e9)},
        "frames_per_s": frames,
        "env_steps_per_s": world * w.n_envs / (ms_step / 1e3),
        # per step: prep, tile prep and render kernels, the env-order sort when the shape asks for it,
        # the downsample kernel for downsampled cameras, the step advance of a graph replay
        "gpu_launches": (3 + (1 if tuning.get("env_order") else 0) + (1 if graph else 0)
                         + (1 if raw_rays else 0)) * args.steps,
        "roofline": roof,
        "clocks": ck,
        "vram": vram,
        "e2e": e2e,
        "scene": {"terrain_tris": info["terrain_tris"], "terrain_nodes": info["terrain_nodes"],
                  "terrain_depth": info["terrain_depth"], "terrain_bytes": info["terrain_bytes"],
                  "bvh_build_s": build_s},
    }
    if not args.no_serve and args.variant == "plain":
        # the serving half of the metric on the same GPU and resident scene (config 5, shortened)
        from paper_2602_03002_gb300 import workloads as W
        view.close()
        line["serve"] = serve_summary(serve_measure(rpl, W, scene, args.tiles, args.serve_requests, 8))
    if world == 1 and not args.no_cpu_baseline:
        _, _, _, cb = cpu_baseline(w, args.cpu_seconds, gpu_step0)
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def serve_measure(rpl, W, scene, tiles, n_req, rounds, load=0.8, seed=5):
    """Config 5 on a resident scene: Poisson streams of render requests from 4 trainer threads (4 views
    each: env counts log-uniform in 64..8192, 1-4 cameras front/back 64x48, left/right 48x36).  The
    same seeded arrival schedule (at `load` times the one-request capacity) is served by the
    continuous-batching server (up to 32 requests per launch, 2 streams) and by plain per-request
    launches (batches of one on one stream); latency is submit to completion on the host clock.  Also
    a closed loop with every request outstanding (`rounds` rounds): the throughput each form sustains."""
    import threading
    import torch
    rng = np.random.default_rng(seed)
    n_tr, per_tr = 4, 4
    sizes = [(64, 48), (64, 48), (48, 36), (48, 36)]
    shapes = []
    for k in range(n_tr * per_tr):
        E = int(round(float(np.exp(rng.uniform(np.log(64), np.log(8192))))))
        C = int(rng.integers(1, 5))
        poses, cams = W.scale_envs(E, 4, tiles, sizes[:C], seed=100 + k)
        shapes.append((E, cams, torch.from_numpy(poses).cuda()))
    sensor = W.scale_sensor()

    def make_views():
        vs = []
        for k, (E, cams, poses) in enumerate(shapes):
            v = rpl.View(scene, E, 30)
            v.set_cameras(cams)
            v.set_sensor(sensor)
            vs.append((v, v.out_tensor(), poses, E * sum(c.width * c.height for c in cams)))
        return vs

    # calibration: mean time of one request rendered alone (back to back, no server)
    vs = make_views()
    times = []
    for k, (v, out, poses, rays) in enumerate(vs):
        for s in range(3):
            v.render(poses[s % 4], s, 0, out)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for s in range(3, 6):
            v.render(poses[s % 4], s, 0, out)
        torch.cuda.synchronize()
        times.append((time.perf_counter() - t) / 3)
    for v, _, _, _ in vs:
        v.close()
    service = float(np.mean(times))

    def run_mode(max_batch, n_streams):
        vs = make_views()
        server = rpl.Server(scene, max_batch=max_batch, n_streams=n_streams)
        lat, rays_done = [], [0]
        lock = threading.Lock()
        steps = [0] * len(vs)
        t0 = time.perf_counter() + 0.05

        def trainer(tr):
            import queue as q
            pending = q.Queue()

            def waiter():
                while True:
                    item = pending.get()
                    if item is None:
                        return
                    tk, rays = item
                    dt = server.wait(tk)
                    with lock:
                        lat.append(dt)
                        rays_done[0] += rays
            w_th = threading.Thread(target=waiter)
            w_th.start()
            for i, ta in enumerate(sched[tr]):
                k = tr * per_tr + i % per_tr
                v, out, poses, rays = vs[k]
                now = time.perf_counter()
                if t0 + ta > now:
                    time.sleep(t0 + ta - now)
                s = steps[k]
                steps[k] += 1
                pending.put((server.submit(v, poses[s % 4], s, out), rays))
            pending.put(None)
            w_th.join()

        th = [threading.Thread(target=trainer, args=(tr,)) for tr in range(n_tr)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        wall = time.perf_counter() - t0
        st = server.stats()
        server.close()
        for v, _, _, _ in vs:
            v.close()
        lat_ms = np.asarray(lat) * 1e3
        return {"p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                "mean_ms": float(lat_ms.mean()), "requests": len(lat), "grays_per_s": rays_done[0] / wall / 1e9,
                "wall_s": wall, "batches": st["batches"], "mean_batch": st["fused_requests"] / max(1, st["batches"]),
                "max_batch_seen": st["max_batch_seen"], "max_inflight_batches": st["max_inflight_batches_seen"]}

    def run_saturated(max_batch, n_streams):
        """Closed loop: every trainer keeps its four views' requests in flight (submit all four, wait
        for all four, repeat), so 16 requests are outstanding and the GPU never waits for arrivals."""
        vs = make_views()
        server = rpl.Server(scene, max_batch=max_batch, n_streams=n_streams)
        rays_done = [0]
        lock = threading.Lock()

        def trainer(tr):
            mine = [vs[tr * per_tr + j] for j in range(per_tr)]
            for rnd in range(rounds):
                tks = [server.submit(v, poses[rnd % 4], rnd, out) for v, out, poses, _ in mine]
                for tk in tks:
                    server.wait(tk)
                with lock:
                    rays_done[0] += sum(r for _, _, _, r in mine)

        th = [threading.Thread(target=trainer, args=(tr,)) for tr in range(n_tr)]
        t = time.perf_counter()
        for x in th:
            x.start()
        for x in th:
            x.join()
        wall = time.perf_counter() - t
        st = server.stats()
        server.close()
        for v, _, _, _ in vs:
            v.close()
        return {"grays_per_s": rays_done[0] / wall / 1e9, "wall_s": wall, "requests": st["completed"],
                "mean_batch": st["fused_requests"] / max(1, st["batches"])}

    # the offered load: `load` times the request rate the plain per-request form sustains in a closed
    # loop (with its host work per request), so that both forms see a load the baseline can carry
    sat_plain = run_saturated(1, 1)
    sat_batched = run_saturated(32, 2)
    rate = load * sat_plain["requests"] / sat_plain["wall_s"]   # requests per second, all trainers
    sched = []
    for tr in range(n_tr):
        gaps = rng.exponential(n_tr / rate, size=n_req // n_tr)
        sched.append(np.cumsum(gaps))
    batched = run_mode(32, 2)
    plain = run_mode(1, 1)
    return {"batched": batched, "per_request": plain,
            "saturated": {"note": "closed loop, 16 requests outstanding: throughput each form sustains",
                          "batched": sat_batched, "per_request": sat_plain},
            "workload": "4 trainers x 4 views (env counts log-uniform 64..8192, 1-4 cameras 64x48/48x36), "
                        "Poisson arrivals at %.0f%% of the request rate the per-request form sustains, scale "
                        "terrain resident, sensor on, FP32 depth" % (100 * load),
            "views": [{"envs": E, "cams": len(c)} for E, c, _ in shapes],
            "arrival_rate_per_s": rate, "service_ms_alone": 1e3 * service, "requests_per_form": n_req}


def serve_summary(m):
    """The headline serving figures: both forms' p50/p99 and throughput on the same arrival schedule."""
    b, p = m["batched"], m["per_request"]
    return {"p50_ms": b["p50_ms"], "p99_ms": b["p99_ms"], "grays_per_s": b["grays_per_s"],
            "mean_batch": b["mean_batch"], "max_batch_seen": b["max_batch_seen"],
            "per_request": {"p50_ms": p["p50_ms"], "p99_ms": p["p99_ms"], "grays_per_s": p["grays_per_s"]},
            "saturated_grays_per_s": {"batched": m["saturated"]["batched"]["grays_per_s"],
                                      "per_request": m["saturated"]["per_request"]["grays_per_s"]},
            "requests_per_form": m["requests_per_form"], "arrival_rate_per_s": m["arrival_rate_per_s"],
            "service_ms_alone": m["service_ms_alone"], "workload": m["workload"],
            "latency": "submit to completion on the host clock; batched = continuous-batching server "
                       "(up to 32 requests per launch, 2 streams), per_request = one plain FP32 launch per "
                       "request on one stream, same arrival schedule"}


def run_serving(args):
    """The serving configuration on its own (more requests than the default line's serve object)."""
    import torch
    from paper_2602_03002_gb300 import build as B, rpl, workloads as W
    rank, world, local = dist_info()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    B.build()
    base = W.config_scale(n_steps=1, n_envs=16, tiles=args.tiles)
    scene = rpl.Scene(base.terrain_verts, base.terrain_tris, device=local)
    for l, (v_, t_) in enumerate(zip(base.link_verts, base.link_tris)):
        scene.add_link(l, v_, t_)
    n_req = max(400, args.steps * 8)
    m = serve_measure(rpl, W, scene, args.tiles, n_req, 20)
    batched = m["batched"]
    line = {"metric": METRIC, "value": batched["grays_per_s"], "unit": "Grays/s", "n_gpus": 1,
            "steps": n_req, "warmup": 3, "ms_per_step": batched["mean_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "variant": "serving",
            "config": {"workload": "serving: " + m["workload"] + " (%d-tri terrain)" % len(base.terrain_tris),
                       "views": m["views"], "arrival_rate_per_s": m["arrival_rate_per_s"],
                       "service_ms_alone": m["service_ms_alone"]},
            "serve": serve_summary(m), "serve_detail": m,
            "p50_ms": batched["p50_ms"], "p99_ms": batched["p99_ms"]}
    print(json.dumps(line), flush=True)


def run_table1(args):
    """The setting of the paper's Table 1 (1024 envs, 240x135 depth, 1 / 2 / 4 cameras) with the
    perception workload's cameras, randomisation and sensor: time per render and device memory for
    each camera count.  The paper's own figures are training-iteration times on an L40S, not render
    times, so they are context only."""
    import torch
    from paper_2602_03002_gb300 import build as B, rpl, workloads as W
    rank, world, local = dist_info()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    B.build()
    envs = 1024
    w = W.config_perception(n_steps=args.pose_sets, n_envs=envs, tiles=args.tiles, n_cams=4)
    free0 = torch.cuda.mem_get_info(local)[0]
    scene = rpl.Scene(w.terrain_verts, w.terrain_tris, device=local, bvh_kind=bvh_kind(args, rpl))
    for l, (v_, t_) in enumerate(zip(w.link_verts, w.link_tris)):
        scene.add_link(l, v_, t_)
    scene_gb = (free0 - torch.cuda.mem_get_info(local)[0]) / 1e9
    poses = torch.from_numpy(w.poses).cuda()
    S = poses.shape[0]
    rows = []
    for n_cams in (1, 2, 4):
        free1 = torch.cuda.mem_get_info(local)[0]
        view = rpl.View(scene, envs, w.n_links)
        view.set_cameras(w.cameras[:n_cams], w.per_env_intrinsics[:, :n_cams])
        view.randomize_cameras(w.mount_delta[:, :n_cams])
        view.set_side_mask(w.rsm_cols, w.rsm_modes)
        view.set_sensor(w.sensor)
        out = view.out_tensor()
        view_gb = (free1 - torch.cuda.mem_get_info(local)[0]) / 1e9
        tuning, _ = rpl.rpl_view_autotune(view.h, poses[0], 0, 0, out, None, 2)
        view.reset(None, 0)
        for s in range(args.warmup):
            rpl.rpl_render(view.h, poses[s % S], s, 0, out, None)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for s in range(args.warmup, args.warmup + args.steps):
            rpl.rpl_render(view.h, poses[s % S], s, 0, out, None)
        b.record()
        torch.cuda.synchronize()
        view.sync()
        ms = a.elapsed_time(b) / args.steps
        rays = envs * n_cams * 240 * 135
        rows.append({"n_cam": n_cams, "ms_per_render": ms, "grays_per_s": rays / ms / 1e6,
                     "depth_frames_per_s": envs * n_cams / (ms / 1e3), "view_vram_gb": view_gb, "tuning": tuning})
        view.close()
    two = rows[1]
    line = {"metric": METRIC, "value": two["grays_per_s"], "unit": "Grays/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": two["ms_per_render"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "variant": "table1",
            "config": {"workload": "the paper's Table 1 setting: 1024 envs, 240x135 ray cast (averaged to 48x27), "
                                   "1 / 2 / 4 cameras, scale terrain (%d tris), perception randomisation and sensor; "
                                   "value = the 2-camera row" % len(w.terrain_tris)},
            "table1": rows, "scene_vram_gb": scene_gb,
            "paper_context": "Table 1 (one L40S, 1024 envs, 240x135): 1.3 / 1.5 / 1.9 s per training iteration "
                             "and 13.3 / 14.6 / 17.3 GB for 1 / 2 / 4 cameras; iteration times include physics "
                             "and learning, so they are not render times"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.variant == "serving":
        run_serving(args)
    elif args.variant == "table1":
        run_table1(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
