#!/usr/bin/env python3
"""Throughput benchmark of the GB300 Gaussian-primitive path tracer.

Workload (the paper-scale configuration, the analogue of the paper's largest timed scene): a
procedural room of 5,500,000 Gaussian primitives (70 % surface splats on planes, spheres and
boxes, 30 % isotropic aggregates in 300 clusters; 50 / 40 / 10 % diffuse / GGX / emissive
shapes, a tenth of the shapes near-specular GGX with roughness 0.02) lit by a 0.3 x 0.3 area
light and a background (lighting A), rendered at 1920 x 1080 with max depth 12.  One step =
BVH build over the primitives + one sample per pixel of the wavefront path tracer (camera,
free-flight extend, shading with light sampling + MIS, shadow transmittance, accumulation);
256 steps are the full 256-spp frame.  Inputs are synthetic (seeded generator).

Metric: Mrays/s = (free-flight queries + shadow queries) / time, plus the equal-time MSE of
the learned-guide renderer against plain phase sampling: on the same scene and BVH at a
reduced image size, a converged plain reference is rendered first; then the plain renderer
runs for a budget of spp and the guided renderer (trained online during its first spp, the
training time counted) runs for the same wall time; both MSEs are taken against the reference
with the reference's own variance subtracted.  The many-small-emitter lighting (B) of the same
scene is timed as a study in the same line.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ugp|reference]
For N > 1 run under torch.distributed.run: every rank renders its own replica of the
workload (the path does not shard across GPUs in this build), timings are max-reduced
and rays sum-reduced.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mrays/s + equal-time MSE vs converged ref, MLP-guided vs plain, 1 GB300"
UNIT = "Mrays/s"


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=16)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ugp", "reference"], default="ugp")
    p.add_argument("--n-prims", type=int, default=5_500_000)
    p.add_argument("--width", type=int, default=1920)
    p.add_argument("--height", type=int, default=1080)
    p.add_argument("--depth", type=int, default=12)
    p.add_argument("--lighting", choices=["A", "B"], default="A",
                   help="A: quad area light + background; B: 12,000 small emissive primitives")
    p.add_argument("--near-specular", type=float, default=0.1,
                   help="fraction of surface shapes made near-specular GGX (roughness 0.02)")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end loop")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-pixels", type=int, default=4096, help="pixels of the CPU-baseline sample")
    p.add_argument("--kernel-case", choices=["ff_camera512", "render_960x540", "guide_rows256k"], default=None,
                   help="run one small kernel case for profilers and exit (no bench line)")
    p.add_argument("--no-mse", action="store_true", help="skip the equal-time MSE study")
    p.add_argument("--mse-width", type=int, default=480, help="image width of the MSE study")
    p.add_argument("--mse-height", type=int, default=270, help="image height of the MSE study")
    p.add_argument("--mse-ref-spp", type=int, default=2048, help="spp of the plain reference")
    p.add_argument("--mse-budget-spp", type=int, default=256, help="plain spp that set the time budget")
    p.add_argument("--mse-train-spp", type=int, default=32, help="guided spp that also train the guide")
    p.add_argument("--mse-minibatch", type=int, default=1 << 14)
    p.add_argument("--mse-min-steps", type=int, default=128, help="Adam steps per training spp, at least")
    p.add_argument("--guide-alpha", type=float, default=0.5)
    p.add_argument("--no-serving", action="store_true", help="skip the batched-serving study")
    p.add_argument("--no-rf", action="store_true", help="skip the radiance-field render study")
    p.add_argument("--no-exp", action="store_true", help="skip the exponential-variant query study")
    p.add_argument("--no-emitters", action="store_true", help="skip the emitter light-sampling study")
    p.add_argument("--no-kdtree", action="store_true", help="skip the paper's kd-tree sampler study")
    p.add_argument("--no-codebook", action="store_true", help="skip the codebook-record study")
    p.add_argument("--kd-prims", type=int, default=1_000_000, help="primitives of the kd-tree study's scene")
    p.add_argument("--serve-requests", type=int, default=64)
    p.add_argument("--serve-spp-max", type=int, default=64,
                   help="spp of the serving requests are log-uniform in [1, this] (64 = the full workload)")
    p.add_argument("--guide-lr", type=float, default=1e-3)
    p.add_argument("--guide-min-roughness", type=float, default=0.0,
                   help="vertices with a glossier base scatter by phase sampling alone in the MSE study")
    p.add_argument("--guide-target", type=int, choices=[0, 1], default=0,
                   help="guide training target: 0 incident radiance, 1 its product with the phase function")
    return p.parse_args(argv)


# ------------------------------------------------------------------------------- helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured"
    except Exception:
        return 6800.0, "of fallback"


def measured_bf16_peak():
    """Burst dense BF16 tensor throughput (TFLOP/s) for kernels timed alone."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "of measured"
    except Exception:
        return 1900.0, "of fallback"


# Algorithmic FLOP per row of the guide network (4 x 64x64 layers and a 64 -> 40 head):
# forward 2 (4*64*64 + 40*64); training adds dW of every layer (same count) and dX of layers 1..4.
GUIDE_FWD_FLOP = 2 * (4 * 64 * 64 + 40 * 64)
GUIDE_GRAD_FLOP = 2 * GUIDE_FWD_FLOP + 2 * (3 * 64 * 64 + 40 * 64)


# DRAM bytes (read + write) per k_extend launch of a workload, averaged over the launches of one
# step, from one ncu capture of the current kernel (its summary is kept under profiles/); None for any
# other workload, and to be reset whenever k_extend changes.
EXTEND_TRAFFIC_BYTES = {(5_500_000, 1920, 1080, 12, "A", 0.1): 1371.15e6}

# Algorithmic bytes of a free-flight query are counted against a fixed reference traversal, so
# that a tree that makes a query visit more nodes cannot raise the figure: the nodes and records
# a query loads on the binary LBVH of the same build (64 B each) with the same scan (its bins and
# pruning), measured once per workload with that traversal's counters. Workloads without a
# reference use the live counts.
REFERENCE_COUNTS = {(5_500_000, 1920, 1080, 12, "A", 0.1): (264.18, 135.91)}


def workload_key(args):
    return (args.n_prims, args.width, args.height, args.depth, args.lighting, args.near_specular)


def extend_traffic(args):
    return EXTEND_TRAFFIC_BYTES.get(workload_key(args))


def bench_scene(args, lighting=None):
    from paper_2406_09733_gb300 import scenes
    return scenes.room_scene(args.n_prims, width=args.width, height=args.height,
                             near_specular_frac=args.near_specular, lighting=lighting or args.lighting)


def guide_kernel_timing(dev, rows=1 << 20, reps=10):
    """CUDA-event time of the guide's forward and gradient calls on `rows` random vertices."""
    import torch
    from paper_2406_09733_gb300 import scenes, ugp
    t = lambda a: torch.from_numpy(a).to(dev)
    g = ugp.Guide(scenes.guide_init_params(seed=0, bias_scale=0.2), device=dev)
    b = scenes.guide_batch(rows, seed=1)
    x, wo, wi, w = t(b.x), t(b.wo), t(b.wi), t(b.weight)
    out = {}
    peak, note = measured_bf16_peak()
    for name, fn, flop in (("forward", lambda: g.forward(x, wo, head=False), GUIDE_FWD_FLOP),
                           ("grad", lambda: g.grad(x, wo, wi, w), GUIDE_GRAD_FLOP)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        ugp.profile_begin(4096)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        prof = ugp.profile_end()
        ms = e0.elapsed_time(e1) / reps
        tf = rows * flop / (ms / 1e3) / 1e12
        out[name] = {"rows": rows, "ms_per_call": ms, "algorithmic_flop_per_row": flop, "achieved_tflops": tf,
                     "peak_tflops": peak, "frac": tf / peak, "peak_note": note,
                     "launches_per_call": prof["guide"][1] / reps}
    g.check()
    return out


def serving_study(args, dev):
    """Batched serving: the same requests served one by one (ugp_render, sequentially) and as one
    batch (ugp_render_batch: one CUDA graph launch, autotuned tile and pool, shortest first)."""
    import numpy as np
    import torch
    from paper_2406_09733_gb300 import scenes, ugp
    ns, specs = scenes.serving_batch(args.serve_requests, 8, seed=0, spp_range=(1, args.serve_spp_max))
    sd = []
    for i, n in enumerate(ns):
        sc = scenes.serving_scene(n, seed=i)
        sd.append((sc, ugp.scene_to_device(sc, device=dev)))

    def make_reqs():
        out = []
        for q in specs:
            sc, (bvh, mats, _, lights) = sd[q.scene]
            c = sc.camera
            cam = ugp.camera_struct(c.eye, c.look, c.up, c.vfov_deg, q.width, q.height)
            out.append(ugp.Request(bvh, mats, cam, lights, q.spp, q.max_depth, seed=q.seed, device=dev))
        return out

    paths = int(sum(q.width * q.height * q.spp for q in specs))
    # one by one, in the given order (latency = time until the request's image is done)
    reqs = make_reqs()
    rends = {}
    for q in specs:   # workspaces allocated before timing
        rends.setdefault((q.width, q.height), ugp.Renderer(q.width, q.height, device=dev))
    rc = torch.zeros(3, dtype=torch.int64, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    lat_seq = []
    for q, spec in zip(reqs, specs):
        sc, (bvh, mats, _, lights) = sd[spec.scene]
        rends[(spec.width, spec.height)].render(bvh, mats, q.c.camera, lights, spp=spec.spp, max_depth=spec.max_depth,
                                                seed=spec.seed, accum=q.accum, accum_sq=q.accum_sq, ray_counts=rc)
        torch.cuda.synchronize(dev)
        lat_seq.append(1e3 * (time.perf_counter() - t0))
    t_seq = time.perf_counter() - t0
    rays_seq = int(rc[0] + rc[1])
    ref = [q.accum for q in reqs]

    br = ugp.BatchRenderer(len(specs), pool_log2=20, tile=16, use_graph=True, shortest_first=True, device=dev)
    t0 = time.perf_counter()
    (tile, lg), table = br.autotune(make_reqs()[:16], probe_spp=1, pool_log2_range=(20, 24))
    t_tune = time.perf_counter() - t0
    br.render(make_reqs())   # builds the graph of the chosen pool once
    reqs = make_reqs()
    rc = torch.zeros(3, dtype=torch.int64, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    lat = br.render(reqs, ray_counts=rc)
    torch.cuda.synchronize(dev)
    t_b = time.perf_counter() - t0
    rays_b = int(rc[0] + rc[1])
    rel = max(float(((a - b).abs().max() / (b.abs().max() + 1e-6)).item()) for a, b in zip([q.accum for q in reqs], ref))
    return {
        "workload": (f"{len(specs)} requests over 8 room scenes of {min(ns)}-{max(ns)} primitives, "
                     f"images 256^2/512^2/1024^2, spp log-uniform 1..{args.serve_spp_max}, depth 4..8, all at t=0"),
        "paths": paths, "rays": rays_b,
        "batch": {"makespan_ms": 1e3 * t_b, "Mrays_per_s": rays_b / t_b / 1e6,
                  "latency_p50_ms": float(np.percentile(lat, 50)), "latency_p99_ms": float(np.percentile(lat, 99)),
                  "config": {"tile": tile, "pool": 1 << lg, "graph": True, "order": "shortest first"}},
        "one_by_one": {"makespan_ms": 1e3 * t_seq, "Mrays_per_s": rays_seq / t_seq / 1e6,
                       "latency_p50_ms": float(np.percentile(lat_seq, 50)),
                       "latency_p99_ms": float(np.percentile(lat_seq, 99))},
        "same_rays": rays_b == rays_seq, "max_rel_diff_images": rel,
        "autotune": {"seconds": t_tune, "probe": "first 16 requests at 1 spp",
                     "pool_range": "2^20..2^24", "ms": {f"tile{k[0]}_pool2^{k[1]}": v for k, v in table.items()}},
    }


def equal_time_mse(args, d, mats, scene, dev):
    """Equal-time MSE of guided vs plain rendering against a converged plain reference."""
    import numpy as np
    import torch
    from paper_2406_09733_gb300 import scenes, ugp
    MW, MH = args.mse_width, args.mse_height
    cam = scene.camera
    camera = ugp.camera_struct(cam.eye, cam.look, cam.up, cam.vfov_deg, MW, MH)
    li = scene.lights
    lights = ugp.lights_struct(li.has_quad, li.quad_corner, li.quad_e1, li.quad_e2, li.quad_Le, li.bg)
    bvh = ugp.build_bvh(d["mean"], d["quat"], d["scale"], d["magnitude"])
    info = bvh.info()
    r = ugp.Renderer(MW, MH, device=dev)
    z = lambda: torch.zeros((MH, MW, 3), dtype=torch.float32, device=dev)
    depth = args.depth

    # converged plain reference (different seed), in chunks of 64 spp
    ref, ref2 = z(), z()
    for s0 in range(0, args.mse_ref_spp, 64):
        r.render(bvh, mats, camera, lights, spp=min(64, args.mse_ref_spp - s0), max_depth=depth, seed=777,
                 spp_begin=s0, accum=ref, accum_sq=ref2)
    torch.cuda.synchronize(dev)
    ref_mean = (ref / args.mse_ref_spp).double()
    ref_var = ((ref2 / args.mse_ref_spp).double() - ref_mean ** 2).clamp(min=0) / args.mse_ref_spp
    ref_var_mean = float(ref_var.mean())

    def mse(acc, spp):
        return float(((acc.double() / spp - ref_mean) ** 2).mean()) - ref_var_mean

    checkpoints = sorted({8, 16, 32, args.mse_budget_spp})
    # plain: one spp per call, timed on the host around synchronised calls
    acc, acc2 = z(), z()
    torch.cuda.synchronize(dev)
    t_plain, curve_p = 0.0, []
    for k in range(args.mse_budget_spp):
        t0 = time.perf_counter()
        r.render(bvh, mats, camera, lights, spp=1, max_depth=depth, seed=1, spp_begin=k, accum=acc, accum_sq=acc2)
        torch.cuda.synchronize(dev)
        t_plain += time.perf_counter() - t0
        if k + 1 in checkpoints:
            curve_p.append([1e3 * t_plain, mse(acc, k + 1)])
    mse_plain = mse(acc, args.mse_budget_spp)

    # guided: trained during its first mse_train_spp samples, then frozen, until the same time
    g = ugp.Guide(scenes.guide_init_params(seed=0, bias_scale=0.0), info["bounds_lo"], info["bounds_hi"],
                  lr=args.guide_lr, device=dev, train_target=args.guide_target)
    gacc, gacc2 = z(), z()
    t_g, k, curve_g, n_train, losses = 0.0, 0, [], 0, []
    while t_g < t_plain and k < 64 * args.mse_budget_spp:
        train = k < args.mse_train_spp
        t0 = time.perf_counter()
        r.render(bvh, mats, camera, lights, spp=1, max_depth=depth, seed=2, spp_begin=k, accum=gacc,
                 accum_sq=gacc2, guide=g, guide_alpha=args.guide_alpha, guide_log=train,
                 guide_min_roughness=args.guide_min_roughness)
        if train:
            ns, loss = g.train_from(r, max_samples=1 << 20, minibatch=args.mse_minibatch,
                                    min_steps=args.mse_min_steps)
            n_train += ns
            losses.append(loss)
        torch.cuda.synchronize(dev)
        t_g += time.perf_counter() - t0
        k += 1
        if k in checkpoints or t_g >= t_plain:
            curve_g.append([1e3 * t_g, mse(gacc, k)])
    g.check()
    mse_guided = mse(gacc, k)
    return {"plain": mse_plain, "guided": mse_guided, "ratio_guided_over_plain": mse_guided / mse_plain,
            "budget_ms": 1e3 * t_plain, "plain_spp": args.mse_budget_spp, "guided_spp": k, "guided_ms": 1e3 * t_g,
            "train_spp": min(args.mse_train_spp, k), "train_samples": n_train, "adam_steps": g.step,
            "loss_first_last": [losses[0], losses[-1]] if losses else None,
            "reference_spp": args.mse_ref_spp, "reference_var_subtracted": ref_var_mean,
            "image": f"{MW}x{MH} (the bench scene and camera at a reduced image size)",
            "lighting": "B: emissive primitives only, found by phase sampling" if not li.has_quad
                        else "A: area light (light-sampled) and background",
            "max_depth": depth, "guide_alpha": args.guide_alpha, "guide_min_roughness": args.guide_min_roughness,
            "train_target": ("incident radiance" if args.guide_target == 0 else "phase function x incident radiance"),
            "curve_ms_mse": {"plain": curve_p, "guided": curve_g},
            "note": "MSE over linear RGB, no clamping; times include the guide's training"}


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def aggregate(elapsed_ms: float, units: float, dist):
    """Whole-job totals over ranks: (max elapsed ms, sum of units)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return elapsed_ms, units
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def workload_config(args, l2_note):
    light = ("lighting A (0.3x0.3 area light + background 0.2)" if args.lighting == "A"
             else "lighting B (12,000 small emissive primitives, no area light)")
    return {
        "workload": (f"procedural room, {args.n_prims} Gaussian primitives (70% surface splats, 30% "
                     f"aggregate clusters; {args.near_specular:g} of the surface shapes near-specular GGX "
                     f"0.02), {light}, {args.width}x{args.height}, 1 spp per step, max depth {args.depth}"),
        "n_prims": args.n_prims, "width": args.width, "height": args.height, "spp_per_step": 1,
        "max_depth": args.depth, "lighting": args.lighting, "near_specular_frac": args.near_specular,
        "step": "BVH build + 1 spp wavefront render", "l2": l2_note,
        "parallelism": f"replicas x{args.gpus}",
    }


def host_cpu() -> str:
    """The host processor: architecture, and the model name (x86) or implementer/part (Arm) of
    /proc/cpuinfo when it has them."""
    import platform
    desc = platform.machine()
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return desc
    for key in ("model name", "CPU implementer", "CPU part"):
        for line in info:
            if line.startswith(key):
                desc += f", {key}: {line.split(':', 1)[1].strip()}"
                break
    return desc


def cpu_baseline_run(scene, args, pixels, spp=1, seed=0, accel=False, threads=None):
    """The FP64 oracle on a bounded sample of the workload: `pixels` consecutive pixels centred
    in the middle image row, one sample each. With `accel` the oracle finds each ray's intervals
    with its own BVH (the same intervals and results as brute force); the BVH's build time,
    taken by a call that renders no pixel, is not counted."""
    import oracle
    mid = (args.height // 2) * args.width + max(0, (args.width - pixels) // 2)
    if threads:
        oracle.set_num_threads(threads)
    # calls that render no pixel: the first builds the BVH (kept by the oracle for the same
    # arrays), the second times the per-call set-up (the primitives' records) that the timed call
    # also pays
    build = setup = 0.0
    for k in range(2 if accel else 1):
        t0 = time.perf_counter()
        oracle.render(scene, spp=spp, max_depth=args.depth, seed=seed, pixels=(mid, mid), accel=accel)
        if k == 0 and accel:
            build = time.perf_counter() - t0
        else:
            setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, _, (ne, ns) = oracle.render(scene, spp=spp, max_depth=args.depth, seed=seed,
                                   pixels=(mid, mid + pixels), accel=accel)
    dt = max(time.perf_counter() - t0 - setup, 1e-9)
    cores = oracle.num_threads()
    if threads:
        oracle.set_num_threads(os.cpu_count() or 1)
    return (ne + ns) / dt / 1e6, cores, ne + ns, dt, build


def cpu_baseline_configs(args):
    """The oracle's timings on the three plain configurations of the workload set: the
    1,000-primitive scene in full (128^2, 4 spp, depth 4, brute force), a 128 x 128 centre crop
    of the 1M-primitive room at 1024^2 (4 spp, depth 8) and a 64 x 64 centre crop of the bench
    scene (1 spp, the bench's depth), both with the oracle's BVH; rates in Mrays/s on all host
    cores, BVH builds excluded and reported."""
    import oracle
    from paper_2406_09733_gb300 import scenes
    out = {}
    s1 = scenes.tiny_scene()
    t0 = time.perf_counter()
    _, _, (ne, ns) = oracle.render(s1, spp=4, max_depth=4, seed=0)
    dt = time.perf_counter() - t0
    out["tiny_1000_full_128x128_4spp"] = {"Mrays_per_s": (ne + ns) / dt / 1e6, "queries": ne + ns, "s": dt}
    for name, sc, depth, crop, spp in (
            ("room_1M_crop_128x128_4spp", scenes.room_scene(1_000_000, width=1024, height=1024), 8, 128, 4),
            ("bench_scene_crop_64x64_1spp", bench_scene(args), args.depth, 64, 1)):
        W, H = sc.camera.width, sc.camera.height
        rect = ((W - crop) // 2, (H - crop) // 2, crop, crop)
        ts = []
        for _ in range(2):   # BVH build, then the per-call set-up alone (an empty range)
            t0 = time.perf_counter()
            oracle.render(sc, spp=1, max_depth=depth, seed=0, pixels=(0, 0), accel=True)
            ts.append(time.perf_counter() - t0)
        build = ts[0] - ts[1]
        t0 = time.perf_counter()
        _, _, (ne, ns) = oracle.render(sc, spp=spp, max_depth=depth, seed=0, rect=rect, accel=True)
        dt = max(time.perf_counter() - t0 - ts[1], 1e-9)
        out[name] = {"Mrays_per_s": (ne + ns) / dt / 1e6, "queries": ne + ns, "s": dt, "bvh_build_s": build}
    out["cores"] = oracle.num_threads()
    return out


# ------------------------------------------------------------------------------- arms
def run_reference(args):
    """Reference arm: the FP64 CPU oracle (the correctness reference) on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2406_09733_gb300 import scenes
    scene = bench_scene(args)
    px = max(16, args.cpu_pixels // 128)
    for w in range(args.warmup):
        cpu_baseline_run(scene, args, px, seed=1000 + w)
    rays = 0
    total = 0.0
    cores = None
    for k in range(args.steps):
        v, cores, r, dt, _ = cpu_baseline_run(scene, args, px, seed=k)
        rays += r
        total += dt
    value = rays / total / 1e6
    sample = f"{px} pixels x 1 spp centred in the middle row per step, brute force over all primitives"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded generator)",
        "config": workload_config(args, "n/a (CPU)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ugp(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2406_09733_gb300 import scenes, ugp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    scene = bench_scene(args)
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k)))
            for k in ("mean", "quat", "scale", "magnitude", "sggx", "mtype", "albedo", "roughness", "emission")}
    d = {k: v.to(dev) for k, v in host.items()}
    mats = ugp.Materials(d["sggx"], d["mtype"], d["albedo"], d["roughness"], d["emission"])
    cam = scene.camera
    camera = ugp.camera_struct(cam.eye, cam.look, cam.up, cam.vfov_deg, cam.width, cam.height)
    li = scene.lights
    lights = ugp.lights_struct(li.has_quad, li.quad_corner, li.quad_e1, li.quad_e2, li.quad_Le, li.bg)
    renderer = ugp.Renderer(args.width, args.height, device=dev)
    acc = torch.zeros((args.height, args.width, 3), dtype=torch.float32, device=dev)
    acc2 = torch.zeros_like(acc)
    counts = torch.zeros(3, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB of L2
    stream = torch.cuda.current_stream(dev)
    bvh_ws = torch.empty(ugp.build_bvh_workspace_size(args.n_prims), dtype=torch.uint8, device=dev)

    def step(k, ray_counts):
        bvh = ugp.build_bvh(d["mean"], d["quat"], d["scale"], d["magnitude"], workspace=bvh_ws)
        renderer.render(bvh, mats, camera, lights, spp=1, max_depth=args.depth, seed=rank, spp_begin=k,
                        accum=acc, accum_sq=acc2, ray_counts=ray_counts)
        return bvh

    for w in range(args.warmup):
        step(1000 + w, None)
    torch.cuda.synchronize(dev)

    # -------- timed region: K steps, L2 flushed between steps (outside the step events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    keep = None
    launches0 = ugp.launch_count()
    ugp.profile_begin(64 * (args.depth + 4) * max(args.steps, 1) + 64)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            keep = step(k, counts)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    prof = ugp.profile_end()
    launches = ugp.launch_count() - launches0
    del keep
    step_ms = [a.elapsed_time(b) for a, b in ev]
    elapsed = float(sum(step_ms))
    c = counts.cpu().numpy()
    rays_local = float(c[0] + c[1])
    max_ms, rays_total = aggregate(elapsed, rays_local, dist if world > 1 else None)
    value = rays_total / (max_ms / 1e3) / 1e6

    # -------- algorithmic bytes of the dominant kernel (extend) from one counted step
    stats = torch.zeros(12, dtype=torch.int64, device=dev)
    ugp.set_trace_counters(stats)
    cnt2 = torch.zeros(3, dtype=torch.int64, device=dev)
    step(5000, cnt2)
    torch.cuda.synchronize(dev)
    ugp.set_trace_counters(None)
    st = stats.cpu().numpy()
    # per extend query: 64 B per node and 64 B per primitive record loaded (hot geometry), plus the
    # path state it reads (queue index, origin, direction, exclusion: 32 B) and writes (16 B)
    nodes_per_query = st[0] / max(st[2], 1)
    prims_per_query = st[1] / max(st[2], 1)
    ref_counts = REFERENCE_COUNTS.get(workload_key(args))
    ref_nodes, ref_prims = ref_counts if ref_counts else (nodes_per_query, prims_per_query)
    alg_bytes_per_launch = ((ref_nodes + ref_prims) * 64 + 48) * st[2] / (args.depth + 1)
    ext_launches = prof["extend"][1]
    avg_ext_ms = prof["extend"][0] / max(ext_launches, 1)
    queries_per_step = c[0] / args.steps
    achieved_gbs = alg_bytes_per_launch / (avg_ext_ms / 1e3) / 1e9 if avg_ext_ms > 0 else None
    peak, peak_note = measured_peaks()

    # -------- end to end through host buffers (pinned): H2D scene + build + render + D2H image
    e2e = None
    if not args.no_e2e and rank == 0:
        pinned = {k: v.pin_memory() for k, v in host.items()}
        out_acc = torch.empty(acc.shape, dtype=torch.float32).pin_memory()
        out_acc2 = torch.empty(acc.shape, dtype=torch.float32).pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in pinned.values())
        d2h = 2 * out_acc.numel() * 4
        cnt3 = torch.zeros(3, dtype=torch.int64, device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 4))
        for k in range(n_e2e):
            for key, v in pinned.items():
                d[key].copy_(v, non_blocking=True)
            step(7000 + k, cnt3)
            out_acc.copy_(acc, non_blocking=True)
            out_acc2.copy_(acc2, non_blocking=True)
            torch.cuda.synchronize(dev)
        t_e2e = time.perf_counter() - t0
        r3 = cnt3.cpu().numpy()
        e2e = {"value": float(r3[0] + r3[1]) / t_e2e / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": n_e2e}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, r, dt, build = cpu_baseline_run(scene, args, args.cpu_pixels, accel=True)
        v1, _, r1, dt1, _ = cpu_baseline_run(scene, args, max(16, args.cpu_pixels // 32), accel=True, threads=1)
        vb, _, rb, dtb, _ = cpu_baseline_run(scene, args, 32)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": (f"{args.cpu_pixels} pixels x 1 spp centred in the middle row, {r} queries in {dt:.1f} s, "
                          f"FP64, intervals found with the oracle's own BVH (built in {build:.1f} s, not counted)"),
               "single_thread": {"value": v1, "queries": r1, "s": dt1},
               "brute_force": {"value": vb, "queries": rb, "s": dtb,
                               "sample": "32 pixels centred in the middle row, every primitive tested per query"},
               "configs": cpu_baseline_configs(args), "cpu": host_cpu()}

    # lighting B (12,000 small emissive primitives, no area light): built once for the studies
    lit_b = {}

    def lighting_b():
        if not lit_b:
            sb = bench_scene(args, lighting="B")
            tb = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
            db = {"mean": tb(sb.mean), "quat": tb(sb.quat), "scale": tb(sb.scale), "magnitude": tb(sb.magnitude)}
            mb = ugp.Materials(tb(sb.sggx), tb(sb.mtype), tb(sb.albedo), tb(sb.roughness), tb(sb.emission))
            lit_b.update(scene=sb, d=db, mats=mb)
        return lit_b["scene"], lit_b["d"], lit_b["mats"]

    guide_perf = None
    mse = None
    serving = None
    if rank == 0 and world == 1 and not args.no_mse:
        guide_perf = guide_kernel_timing(dev)
        mse = equal_time_mse(args, d, mats, scene, dev)
        try:
            sb, db, mb = lighting_b()
            mse["lighting_B"] = equal_time_mse(args, db, mb, sb, dev)
        except Exception as e:  # reported in the line; the measured step above stands
            mse["lighting_B"] = {"error": repr(e)}
    if rank == 0 and world == 1 and not args.no_serving:
        serving = serving_study(args, dev)
    rf = None
    if rank == 0 and world == 1 and not args.no_rf:
        rf = radiance_field_study(args, d, scene, dev)
    expo = None
    if rank == 0 and world == 1 and not args.no_exp:
        expo = exponential_study(args, d, scene, dev)
    kdst = None
    if rank == 0 and world == 1 and not args.no_kdtree:
        try:
            kdst = kdtree_study(args, dev)
        except Exception as e:  # reported in the line; the measured step above stands
            kdst = {"error": repr(e)}
    cbst = None
    if rank == 0 and world == 1 and not args.no_codebook:
        try:
            cbst = codebook_study(args, d, mats, scene, dev)
        except Exception as e:
            cbst = {"error": repr(e)}
    emit = None
    if rank == 0 and world == 1 and not args.no_emitters:
        try:
            emit = emitter_study(args, d, mats, scene, dev, lighting_b)
        except Exception as e:  # reported in the line; the measured step above stands
            emit = {"error": repr(e)}

    if rank == 0:
        clk = clocks.summary()
        line = {
            "impl": "ugp", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generator)",
            "config": workload_config(args, "flushed between steps (256 MB write)"),
            "rays_per_step": rays_local / args.steps, "extend_queries_per_step": queries_per_step,
            "queries_with_error_status": int(c[2]),
            "stage_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
            "roofline": {"bound": "hbm", "kernel": "k_extend (free-flight sampling)",
                         "achieved": achieved_gbs, "peak": peak, "unit": "GB/s",
                         "frac": (achieved_gbs / peak) if achieved_gbs else None, "peak_note": peak_note,
                         "traffic": extend_traffic(args),
                         "algorithmic_bytes_per_launch": alg_bytes_per_launch,
                         "algorithmic_bytes_basis": (f"per query {ref_nodes:.2f} nodes + {ref_prims:.2f} records "
                                                     f"x 64 B + 48 B of path state, "
                                                     + ("the binary LBVH reference traversal" if ref_counts
                                                        else "this build's traversal counters")),
                         "dram_frac": (extend_traffic(args) / (avg_ext_ms / 1e3) / 1e9 / peak)
                                      if extend_traffic(args) and avg_ext_ms > 0 else None,
                         "nodes_per_query": nodes_per_query, "prims_per_query": prims_per_query,
                         "avg_launch_ms": avg_ext_ms},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "wall_s_timed_region": wall, "equal_time_mse": mse, "guide_kernels": guide_perf, "serving": serving,
            "exponential_variant": expo, "emitter_light_sampling": emit,
            "kdtree_paper_sampler": kdst, "codebook_records": cbst,
            "radiance_field": rf,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def pinhole_rays(cam, W, H):
    """Unit directions of W x H pixel-centre pinhole rays of a scene camera (row-major)."""
    import numpy as np
    f = np.array(cam.look, float) - cam.eye
    f /= np.linalg.norm(f)
    r = np.cross(f, cam.up); r /= np.linalg.norm(r)
    up = np.cross(r, f)
    th = np.tan(np.radians(cam.vfov_deg) / 2)
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    d = f + ((W / H) * (2 * px / W - 1) * th)[..., None] * r + ((1 - 2 * py / H) * th)[..., None] * up
    return (d / np.linalg.norm(d, axis=-1, keepdims=True)).reshape(-1, 3).astype(np.float32)


def radiance_field_study(args, d, scene, dev, reps=10):
    """Radiance-field forward render (Sec. 7, Eq. rf) of the bench scene's camera view, every
    primitive emitting its albedo, background 0.2: one camera ray per pixel, CUDA-event time per
    frame after 3 warm-up frames."""
    import numpy as np
    import torch
    from paper_2406_09733_gb300 import ugp
    W, H = args.width, args.height
    dirs = torch.from_numpy(pinhole_rays(scene.camera, W, H)).to(dev)
    n = dirs.shape[0]
    O = torch.tensor(np.array(scene.camera.eye, np.float32), device=dev).expand(n, 3).contiguous()
    T0, T1 = torch.zeros(n, device=dev), torch.full((n,), 1e30, device=dev)
    em = torch.from_numpy(np.ascontiguousarray(scene.albedo, dtype=np.float32)).to(dev)
    bvh = ugp.build_bvh(d["mean"], d["quat"], d["scale"], d["magnitude"])
    ws = torch.empty(int(ugp.lib().ugp_render_radiance_field_workspace_size(n)), dtype=torch.uint8, device=dev)
    for _ in range(3):
        rgb, st = ugp.render_radiance_field(bvh, O, dirs, T0, T1, em, (0.2, 0.2, 0.2), workspace=ws)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        rgb, st = ugp.render_radiance_field(bvh, O, dirs, T0, T1, em, (0.2, 0.2, 0.2), workspace=ws)
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    return {"image": f"{W}x{H}", "rays": n, "ms_per_frame": ms, "Mrays_per_s": n / (ms / 1e3) / 1e6,
            "queries_with_error_status": int((st != 0).sum().item()), "mean_rgb": rgb.mean(0).tolist(),
            "emission": "per-primitive albedo, background 0.2"}


def exponential_study(args, d, scene, dev, reps=10):
    """The exponential-transmittance variant's two queries (appendix on analog decomposition
    tracking) on the bench scene's camera view: one camera ray per pixel, unbounded; CUDA-event
    time per launch after 3 warm-up launches of each."""
    import numpy as np
    import torch
    from paper_2406_09733_gb300 import scenes, ugp
    W, H = args.width, args.height
    dirs = torch.from_numpy(pinhole_rays(scene.camera, W, H)).to(dev)
    n = dirs.shape[0]
    O = torch.tensor(np.array(scene.camera.eye, np.float32), device=dev).expand(n, 3).contiguous()
    T0, T1 = torch.zeros(n, device=dev), torch.full((n,), 1e30, device=dev)
    U = torch.from_numpy(scenes.uniforms24(5, n)).to(dev)
    bvh = ugp.build_bvh(d["mean"], d["quat"], d["scale"], d["magnitude"])
    out = {"image": f"{W}x{H}", "rays": n}
    for name, fn in (("free_flight", lambda: ugp.sample_free_flight_exponential(bvh, O, dirs, T0, T1, U)),
                     ("transmittance", lambda: ugp.trace_transmittance_exponential(bvh, O, dirs, T0, T1))):
        for _ in range(3):
            res = fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            res = fn()
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": ms, "Mrays_per_s": n / (ms / 1e3) / 1e6,
                     "queries_with_error_status": int((res[-1] != 0).sum().item())}
        if name == "free_flight":
            out[name]["collided"] = float((res[0] >= 0).float().mean().item())
        else:
            out[name]["mean_T"] = float(res[0].mean().item())
    return out


def emitter_study(args, d, mats, scene, dev, lighting_b, spp=4):
    """Light sampling of emissive primitives, no area light, no background, on two scenes of the
    bench's size: the bench scene's own emitters (a tenth of the surface shapes), and the
    generator's lighting B (the paper's night: 12,000 small emissive aggregate primitives added).
    The same frames (bench image and depth) with and without the emitter table: CUDA-event time
    per spp after one warm-up spp, queries, and the mean per-pixel sample variance; efficiency =
    (variance x time) without over with."""
    import numpy as np
    import torch
    from paper_2406_09733_gb300 import scenes, ugp
    W, H = args.width, args.height
    lights = ugp.lights_struct(False, (0, 0, 0), (0, 0, 0), (0, 0, 0), (0, 0, 0), (0.0, 0.0, 0.0))
    ev = lambda: torch.cuda.Event(enable_timing=True)
    t0, t1 = ev(), ev()
    r = ugp.Renderer(W, H, device=dev)

    def one(sc, arrays, m):
        cam = sc.camera
        camera = ugp.camera_struct(cam.eye, cam.look, cam.up, cam.vfov_deg, W, H)
        bvh = ugp.build_bvh(arrays["mean"], arrays["quat"], arrays["scale"], arrays["magnitude"])
        torch.cuda.synchronize(dev)
        t0.record()
        table = ugp.build_emitter_table(bvh, m)
        t1.record()
        torch.cuda.synchronize(dev)
        out = {"table_build_ms": t0.elapsed_time(t1), "n_emitters": int(table[:8].cpu().view(torch.int64)[0])}
        res = {}
        for name, tab in (("phase_only", None), ("light_sampling", table)):
            r.render(bvh, m, camera, lights, spp=1, max_depth=args.depth, seed=3, emitters=tab)
            torch.cuda.synchronize(dev)
            cnt = torch.zeros(3, dtype=torch.int64, device=dev)
            acc = torch.zeros((H, W, 3), dtype=torch.float32, device=dev)
            acc2 = torch.zeros_like(acc)
            t0.record()
            r.render(bvh, m, camera, lights, spp=spp, max_depth=args.depth, seed=5, accum=acc, accum_sq=acc2,
                     ray_counts=cnt, emitters=tab)
            t1.record()
            torch.cuda.synchronize(dev)
            ms = t0.elapsed_time(t1)
            mean = acc.double() / spp
            var = ((acc2.double() / spp - mean ** 2).clamp(min=0) * spp / (spp - 1)).mean().item()
            c = cnt.cpu().tolist()
            res[name] = (var, ms)
            out[name] = {"ms_per_spp": ms / spp, "Mrays_per_s": (c[0] + c[1]) / (ms / 1e3) / 1e6,
                         "extend_queries": c[0], "shadow_queries": c[1], "queries_with_error_status": c[2],
                         "mean_rgb": mean.mean((0, 1)).tolist(), "mean_pixel_variance": var}
        vp, tp = res["phase_only"]
        vl, tl = res["light_sampling"]
        out["efficiency_gain"] = (vp * tp) / (vl * tl) if vl > 0 and tl > 0 else None
        return out

    out = {"image": f"{W}x{H}", "spp": spp, "depth": args.depth,
           "lights": "emissive primitives only (no area light, no background)"}
    out["bench_scene_emitters"] = one(scene, d, mats)
    sb, db, mb = lighting_b()
    out["lighting_B"] = one(sb, db, mb)
    return out


def kdtree_study(args, dev):
    """The paper's own sampler (kd-tree, per-leaf accumulation, binned disambiguation) beside the
    exact BVH sampler on the same rays: 1024^2 pinhole camera rays of a room scene of
    --kd-prims primitives (t in [0, inf)), one uniform pair per ray; CUDA-event time per launch
    after 2 warm-up launches, build times, tree statistics and how often the rule disambiguated."""
    import numpy as np
    import torch
    from paper_2406_09733_gb300 import scenes, ugp
    s = scenes.room_scene(args.kd_prims, width=1024, height=1024, near_specular_frac=args.near_specular)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    e0, e1 = ev(), ev()
    mean, quat, scale, mag = t(s.mean), t(s.quat), t(s.scale), t(s.magnitude)
    torch.cuda.synchronize(dev)
    e0.record()
    bvh = ugp.build_bvh(mean, quat, scale, mag)
    e1.record()
    torch.cuda.synchronize(dev)
    bvh_ms = e0.elapsed_time(e1)
    t0w = time.perf_counter()
    kd = ugp.KdTree(bvh)
    kd_ms = 1e3 * (time.perf_counter() - t0w)
    dirs = t(pinhole_rays(s.camera, 1024, 1024))
    n = dirs.shape[0]
    O = torch.tensor(np.array(s.camera.eye, np.float32), device=dev).expand(n, 3).contiguous()
    T0, T1 = torch.zeros(n, device=dev), torch.full((n,), 1e30, device=dev)
    U, U2 = t(scenes.uniforms24(21, n)), t(scenes.uniforms24(22, n))
    out = {"scene": f"room, {args.kd_prims} primitives", "rays": n, "bvh_build_ms": bvh_ms,
           "kdtree_build_ms_wall": kd_ms, "kdtree": kd.info()}
    ws = torch.empty(int(ugp.lib().ugp_sample_free_flight_workspace_size(n)), dtype=torch.uint8, device=dev)
    for name, fn in (("bvh_exact", lambda: ugp.sample_free_flight(bvh, O, dirs, T0, T1, U, U2, workspace=ws)),
                     ("kdtree_paper_rule", lambda: kd.sample_free_flight(O, dirs, T0, T1, U, U2))):
        for _ in range(2):
            res = fn()
        torch.cuda.synchronize(dev)
        e0.record()
        res = fn()
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        prim, st = res[0], res[-1]
        out[name] = {"ms": ms, "Mrays_per_s": n / (ms / 1e3) / 1e6, "escaped": float((prim < 0).float().mean()),
                     "queries_with_error_status": int((st != 0).sum().item())}
    out["same_escape"] = float(((out["bvh_exact"]["escaped"] > 0) == (out["kdtree_paper_rule"]["escaped"] > 0)))
    return out


def codebook_study(args, d, mats, scene, dev):
    """Codebook-quantised records of the bench scene: encode time (6 Lloyd iterations of the
    four 4096-entry codebooks), bytes per primitive against the uncompressed SoA arrays, decode
    time, and a 1-spp frame of the decoded scene beside the same frame of the original (image
    means and the relative difference of the means)."""
    import numpy as np
    import torch
    from paper_2406_09733_gb300 import ugp
    ev = lambda: torch.cuda.Event(enable_timing=True)
    e0, e1 = ev(), ev()
    torch.cuda.synchronize(dev)
    e0.record()
    book, rec = ugp.codebook_encode(d["mean"], d["quat"], d["scale"], d["magnitude"], mats, iters=6)
    e1.record()
    torch.cuda.synchronize(dev)
    enc_ms = e0.elapsed_time(e1)
    e0.record()
    dec = ugp.codebook_decode(rec, book, disney=False)
    e1.record()
    torch.cuda.synchronize(dev)
    dec_ms = e0.elapsed_time(e1)
    raw = sum(v.numel() * v.element_size() for v in d.values())
    W, H = args.width, args.height
    cam = scene.camera
    camera = ugp.camera_struct(cam.eye, cam.look, cam.up, cam.vfov_deg, W, H)
    li = scene.lights
    lights = ugp.lights_struct(li.has_quad, li.quad_corner, li.quad_e1, li.quad_e2, li.quad_Le, li.bg)
    r = ugp.Renderer(W, H, device=dev)
    means = {}
    for name, arr, m in (("original", d, mats),
                         ("decoded", dec, ugp.Materials(dec["sggx"], dec["mtype"], dec["albedo"], dec["roughness"],
                                                        dec["emission"]))):
        bvh = ugp.build_bvh(arr["mean"], arr["quat"], arr["scale"], arr["magnitude"])
        acc, _ = r.render(bvh, m, camera, lights, spp=4, max_depth=args.depth, seed=9)
        torch.cuda.synchronize(dev)
        means[name] = (acc.double() / 4).mean((0, 1)).tolist()
    rel = float(np.abs(np.array(means["decoded"]) - np.array(means["original"])).max() / max(means["original"]))
    return {"primitives": scene.n, "record_bytes": int(rec.shape[1]), "uncompressed_bytes_per_primitive": raw / scene.n,
            "ratio": raw / (rec.numel() + book.numel() * 4), "codebook_bytes": book.numel() * 4,
            "encode_ms": enc_ms, "decode_ms": dec_ms, "image_mean_rgb": means,
            "max_rel_diff_of_image_means_4spp": rel}


def run_kernel_case(args):
    """One launch of each scene query on 512 x 512 pinhole camera rays of the room scene (t in
    [0, 4]): a small, fixed case for ncu captures of the free-flight and transmittance kernels."""
    import numpy as np
    import torch
    from paper_2406_09733_gb300 import scenes, ugp
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    s = scenes.room_scene(args.n_prims, near_specular_frac=args.near_specular)
    bvh = ugp.build_bvh(t(s.mean), t(s.quat), t(s.scale), t(s.magnitude))
    cam = s.camera
    d = pinhole_rays(cam, 512, 512)
    n = d.shape[0]
    O, D = t(np.tile(np.array(cam.eye, np.float32), (n, 1))), t(d)
    T0, T1 = torch.zeros(n, device=dev), torch.full((n,), 4.0, device=dev)
    prim, tu, tsp, st = ugp.sample_free_flight(bvh, O, D, T0, T1, t(scenes.uniforms24(1, n)),
                                               t(scenes.uniforms24(2, n)))
    T, st2 = ugp.trace_transmittance(bvh, O, D, T0, T1)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": args.kernel_case, "rays": n, "scattered": int((prim >= 0).sum()),
                      "status_max": int(max(st.max(), st2.max()))}))
    return 0


def run_render_case(args):
    """One frame of the bench scene (the workload's primitives and lighting) at 960 x 540, 1 spp,
    max depth 4: a small case for ncu captures of the renderer's kernels (k_extend, k_dense,
    k_dense_big, k_shade, k_shadow), a few GB on the device."""
    import torch
    from paper_2406_09733_gb300 import ugp
    dev = torch.device("cuda")
    args.width, args.height = 960, 540
    scene = bench_scene(args)
    bvh, mats, camera, lights = ugp.scene_to_device(scene, device=dev)
    r = ugp.Renderer(args.width, args.height, device=dev)
    cnt = torch.zeros(3, dtype=torch.int64, device=dev)
    r.render(bvh, mats, camera, lights, spp=1, max_depth=4, seed=3, ray_counts=cnt)
    torch.cuda.synchronize()
    c = cnt.cpu().tolist()
    print(json.dumps({"kernel_case": args.kernel_case, "extend_queries": c[0], "shadow_queries": c[1],
                      "queries_with_error_status": c[2]}))
    return 0


def run_guide_case(args):
    """One forward and one gradient call of the guide on 2^18 random vertices (ncu case)."""
    import torch
    from paper_2406_09733_gb300 import scenes, ugp
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(a).to(dev)
    g = ugp.Guide(scenes.guide_init_params(seed=0, bias_scale=0.2), device=dev)
    b = scenes.guide_batch(1 << 18, seed=1)
    _, mix = g.forward(t(b.x), t(b.wo), head=False)
    grad, loss = g.grad(t(b.x), t(b.wo), t(b.wi), t(b.weight))
    torch.cuda.synchronize()
    g.check()
    print(json.dumps({"kernel_case": args.kernel_case, "rows": b.n, "loss": float(loss.item()),
                      "grad_norm": float(grad.norm().item())}))
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.kernel_case == "guide_rows256k":
        return run_guide_case(args)
    if args.kernel_case == "render_960x540":
        return run_render_case(args)
    if args.kernel_case:
        return run_kernel_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ugp(args)


if __name__ == "__main__":
    sys.exit(main())
