"""Benchmark of the mapping hot path at 1200x680 with a 1M-Gaussian map.

Workload (synthetic stand-in for a Replica-sized RGB-D sequence): a room-shaped
1M-Gaussian map, a ground-truth room scene whose renders are the frames, and a
seeded smooth 1200x680 (f = 600) camera trajectory.  One step is one frame:

  1. render the map at the frame's pose (project, bin + sort, blend);
  2. Fourier seeding of the frame (DFT, high-pass, triangle threshold, missing
     region, equidistant samples, back-projection; learned prior when trained),
     appending up to 50k Gaussians;
  3. ITERS_PER_FRAME mapping iterations (project, bin + sort, blend, loss with
     SSIM and the scale regulariser, adjoint, Adam).

The metric is mapping iterations per second (ITERS_PER_FRAME per step).  Inputs
(the map, all frames' colour and depth) are resident in HBM before timing; the
working set is far larger than the 129 MB L2.  ``e2e`` repeats the measurement
with each frame copied from pinned host memory and the loss read back every step.

``--impl reference`` times the FP64 CPU oracle of the same iteration instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

W, H, F = 1200, 680, 600.0
N_MAP = 1_000_000
N_GT = 1_000_000
ITERS_PER_FRAME = 3
METRIC = "fwd+bwd mapping iters/s @1200x680, 1M Gaussians"
WORKLOAD = ("room map 1M Gaussians, 1200x680 f=600, seeded trajectory; per frame: render + Fourier seeding (<=50k) "
            "+ 3 mapping iterations + pruning (opacity < 0.005 or scale > 0.5 m)")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--tile", default="16x16")
    p.add_argument("--batch", type=int, default=128)
    p.add_argument("--mapping-only", action="store_true", help="steps of mapping iterations without seeding")
    p.add_argument("--no-window", action="store_true", help="skip the keyframe-window measurement")
    p.add_argument("--no-convergence", action="store_true", help="skip the iterations-to-PSNR comparison")
    p.add_argument("--no-tracking", action="store_true", help="skip the GICP tracking / keyframe measurement")
    p.add_argument("--no-ablation", action="store_true", help="skip the densification ablation")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------------------------

def build_workload(seed_offset: int, n_frames: int, tile, batch, device):
    import torch

    from paper_2503_01109_gb300 import fgs, synthetic as syn
    from paper_2503_01109_gb300.frames import FramePipeline

    cams = syn.trajectory(n_frames, seed=100 + seed_offset, width=W, height=H, f=F)
    scene = syn.room_scene(N_MAP, seed=seed_offset, kind="map")
    gt = syn.room_scene(N_GT, seed=1000 + seed_offset, kind="gt")
    pipe = FramePipeline(scene, cams, gt, capacity=N_MAP + (n_frames + 1) * 50_000, tile=tile, batch=batch,
                         iters_per_frame=ITERS_PER_FRAME, device=device, extra_views=window_views(seed_offset))
    return pipe


def window_views(seed_offset: int):
    """The keyframe window: 4 views at 640x480 (f = 525) and 4 at 1200x680 (f = 600)
    taken along the trajectory."""
    from paper_2503_01109_gb300 import synthetic as syn
    a = syn.trajectory(16, seed=100 + seed_offset, width=640, height=480, f=525.0)
    b = syn.trajectory(16, seed=100 + seed_offset, width=W, height=H, f=F)
    return [a[0], a[4], a[8], a[12], b[2], b[6], b[10], b[14]]


def window_measure(pipe, steps: int, warmup: int):
    """The keyframe window on the map the frames built: autotune the tiling,
    capture one iteration in a CUDA graph, time `steps` replays."""
    import torch
    from paper_2503_01109_gb300 import fgs
    from paper_2503_01109_gb300.window import Window, autotune

    cams = window_views(0)
    color, depth = pipe.extra
    best, table = autotune(pipe.g, cams, color, depth, reps=3)
    trial = pipe.g.zeros_like()
    trial.buf.copy_(pipe.g.buf)
    win = Window(trial, cams, best)
    win.set_target(color, depth)
    win.capture(warmup=max(warmup, 3))
    for _ in range(warmup):
        win.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = fgs.launch_count()
    e0.record(stream)
    for _ in range(steps):
        win.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    win.check_status()
    ms = e0.elapsed_time(e1) / steps
    return {"views": "4x640x480 f=525 + 4x1200x680 f=600", "pixels": int(sum(c["width"] * c["height"] for c in cams)),
            "gaussians": pipe.live_count(), "iters_per_s": 1e3 / ms, "ms_per_iter": ms,
            "tiling": f"{best.tile_w}x{best.tile_h}/{best.batch_depth}", "cuda_graph": True,
            "persistent_launch": True,
            "autotune_ms": {f"{t[0]}x{t[1]}/{b}": round(v, 3) for (t, b), v in sorted(table.items())}}


def convergence_measure(seed_offset: int = 0, target_pairs: int = 2_000_000):
    """Iterations and wall time to 30 dB from an empty map: the plain per-view
    Fourier-prior loop vs the learned prior vs the batched 8-view keyframe window
    (co-visible + random keyframes) without and with the learned prior, on a test
    trajectory of a 1200x680 room scene.  The prior is trained on about 2M
    (patch, converged Gaussian) pairs from plain mapping runs of the RGB-D-sequence
    size (640x480, 300k-Gaussian ground truth) and of the benchmark size (1200x680,
    1M-Gaussian ground truth), each a seeded trajectory from an empty map."""
    from paper_2503_01109_gb300 import synthetic as syn
    from paper_2503_01109_gb300.convergence import compare
    from paper_2503_01109_gb300.frames import render_targets

    def runs():
        # eight ground-truth scenes (four of each size), each seen along many short
        # trajectories: a run's first frame seeds most of its pairs
        scenes = []
        for r in range(8):
            if r % 2 == 0:       # RGB-D-sequence size
                scenes.append((syn.room_scene(300_000, seed=7000 + seed_offset + r, kind="gt"), 640, 480, 525.0))
            else:                # benchmark size
                scenes.append((syn.room_scene(N_GT, seed=7000 + seed_offset + r, kind="gt"), W, H, F))
        for t in range(1000):
            gt, w, h, f = scenes[t % len(scenes)]
            cams = syn.trajectory(4, seed=10_000 + seed_offset + t, width=w, height=h, f=f)
            c, d = render_targets(gt, cams)
            yield c, d, cams

    gt = syn.room_scene(N_GT, seed=2000 + seed_offset, kind="gt")
    te = syn.trajectory(10, seed=500 + seed_offset, width=W, height=H, f=F)
    tec, ted = render_targets(gt, te)
    out = compare(runs(), tec, ted, te, capacity=4_000_000, target_psnr=30.0, target_pairs=target_pairs)
    out["setup"] = ("prior trained on pairs from plain mapping runs (4-frame seeded trajectories, 40 iterations per "
                    "frame, from an empty map) over four 640x480 / 300k-Gaussian and four 1200x680 / 1M-Gaussian room "
                    f"scenes in turn until {target_pairs} pairs or 120 s; compared on 10 frames of another 1200x680 "
                    "room scene from an empty map; cap 100 iterations per frame; window = current frame + up to 7 "
                    "co-visible/random keyframes")
    return out


def tracking_measure(frames: int = 20, warmup: int = 3):
    """GICP tracking (Sec. III-B) of 1200x680 frames: exact depth of the room box
    seen by cameras facing a corner, source = every 4th pixel, sparse map of 3 cm
    voxels grown by keyframes, at most 30 Gauss-Newton iterations per frame.  Times the
    per-frame tracking (observed points, their grid and covariances, GICP) with
    CUDA events, reports the ATE against the true poses, and times the keyframe
    co-visibility of the frame against 100 keyframes."""
    import torch
    from paper_2503_01109_gb300 import fgs, synthetic as syn
    from paper_2503_01109_gb300.tracking import SparseMap, Tracker, cam_pose_inverse

    n = frames + warmup + 1
    cams = syn.corner_trajectory(n, W, H, F)
    depths = [torch.as_tensor(syn.box_depth(c)).cuda() for c in cams]
    smap = SparseMap(fgs.grid((-2.5, -2.0, -2.0), 0.1, (50, 40, 40)), fgs.grid((-2.5, -2.0, -2.0), 0.03, (167, 134, 134)))
    tr = Tracker(cams[0], smap, fgs.grid((-6.0, -6.0, 0.0), 0.1, (120, 120, 80)), step=4, iterations=30)
    truth = [cam_pose_inverse(c["world_to_cam"]) for c in cams]
    tr.observe(depths[0])
    tr.add_keyframe(truth[0])
    est, ms, err, its, keyframes = truth[0], [], [], [], 1
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(1, n):
        torch.cuda.synchronize()
        e0.record()
        tr.observe(depths[k])
        est, stats = tr.track(est)          # reads the pose back: the frame's work is done
        e1.record()
        torch.cuda.synchronize()
        if k > warmup:
            ms.append(e0.elapsed_time(e1))
            err.append(float(np.linalg.norm(est[:, 3] - truth[k][:, 3])))
            its.append(float(stats[3]))
        if stats[2] < 0.9:
            tr.add_keyframe(est)
            keyframes += 1
    kf = (cams * (100 // len(cams) + 1))[:100]
    inside = torch.zeros(100, dtype=torch.int64, device="cuda")
    valid = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(3):
        fgs.fgs_covisibility(depths[-1], cams[-1], kf, 4, inside, valid)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(10):
        fgs.fgs_covisibility(depths[-1], cams[-1], kf, 4, inside, valid)
    e1.record()
    torch.cuda.synchronize()
    return {"frames": frames, "ms_per_frame": float(np.mean(ms)), "source_points": int(tr.n_src.item()),
            "map_points": smap.count(), "keyframes": keyframes, "max_iterations": 30,
            "iterations_run_mean": float(np.mean(its)),
            "ate_m": float(np.sqrt(np.mean(np.square(err)))),
            "covisibility_ms_100_keyframes": e0.elapsed_time(e1) / 10,
            "setup": "1200x680 f=600, exact room-box depth, cameras facing a corner; GICP against a 3 cm-voxel "
                     "sparse map; keyframe when under 90% of the source points overlap the map"}


def ablation_measure(seed_offset: int = 0):
    """The densification ablation (tab6's variants) on 8 frames of the 1200x680
    room trajectory from an empty map, 20 mapping iterations per frame."""
    from paper_2503_01109_gb300 import synthetic as syn
    from paper_2503_01109_gb300.ablation import densification_ablation
    from paper_2503_01109_gb300.frames import render_targets

    gt = syn.room_scene(N_GT, seed=3000 + seed_offset, kind="gt")
    cams = syn.trajectory(8, seed=600 + seed_offset, width=W, height=H, f=F)
    colors, depths = render_targets(gt, cams)
    return densification_ablation(colors, depths, cams, capacity=4_000_000)


def aggregate(ms_local: float, units_local: float, world: int, dist=None):
    """Whole-job throughput of N independent replicas: the slowest rank's time
    and the units all ranks processed (max / sum over ranks; no data exchange)."""
    if world <= 1 or dist is None:
        return ms_local, units_local / (ms_local / 1e3)
    import torch
    t = torch.tensor([ms_local, units_local], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    mx = t[:1].clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    tot = t[1:].clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    ms = float(mx.item())
    return ms, float(tot.item()) / (ms / 1e3)


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)
    from paper_2503_01109_gb300 import fgs

    tw, th = (int(x) for x in args.tile.split("x"))
    n_frames = args.warmup + args.steps
    pipe = build_workload(rank, n_frames, (tw, th), args.batch, device)
    step = pipe.mapping_step if args.mapping_only else pipe.frame_step
    iters_per_step = 1 if args.mapping_only else ITERS_PER_FRAME

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up frames
    for k in range(args.warmup):
        step(k)
    barrier()
    pipe.check()
    stream = torch.cuda.current_stream()
    # events around the adjoint only (the roofline's kernel: the dominant one, as
    # the breakdown pass shows); every other span would end the programmatic-launch
    # overlap at its boundaries, so the per-call breakdown comes from a separate
    # pass after the timed region
    pipe.kernel_timer.enable(("render_bwd",))
    with ClockSampler(local) as clk:
        barrier()
        l0 = fgs.launch_count()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(args.warmup, args.warmup + args.steps):
            step(k)
        t1.record(stream)
        barrier()
        launches = fgs.launch_count() - l0
        ms = t0.elapsed_time(t1)
    pipe.kernel_timer.disable()
    pipe.check()
    clocks = clk.summary()
    ms_max, value = aggregate(ms, iters_per_step * args.steps, world, dist if world > 1 else None)
    total_iters = iters_per_step * args.steps * world
    peaks = load_peaks()
    measured = fgs.measure_peaks()          # on-chip rates of this device, after the timed region
    roof = pipe.roofline(peaks, os.path.join(ROOT, "profiles"), total_ms=ms, measured=measured)
    pipe.mapper.nc_snap.clear()

    e2e = None
    if not args.no_e2e:
        e2e = pipe.e2e_measure(args.warmup, args.steps, step)
        _, e2e_value = aggregate(e2e["ms"], iters_per_step * args.steps, world, dist if world > 1 else None)
        e2e = {"value": e2e_value, "unit": "iters/s", "h2d_bytes_per_step": e2e["h2d"],
               "d2h_bytes_per_step": e2e["d2h"]}

    # per-call breakdown: a separate pass with events around every call
    bd_steps = min(args.steps, 10)
    pipe.kernel_timer.enable()
    for k in range(args.warmup + args.steps, args.warmup + args.steps + bd_steps):
        step(k)
    barrier()
    pipe.kernel_timer.disable()
    pipe.check()
    breakdown = pipe.kernel_timer.summary(bd_steps)
    pipe.mapper.nc_snap.clear()

    window = None
    if not args.no_window and pipe.extra is not None:
        window = window_measure(pipe, args.steps, args.warmup)
    conv = None
    if not args.no_convergence and rank == 0:
        try:
            conv = convergence_measure()
        except Exception as e:  # the comparison is reported, never fatal to the bench line
            conv = {"error": f"{type(e).__name__}: {e}"}

    tracking = None
    if not args.no_tracking and rank == 0:
        tracking = tracking_measure()
    ablation = None
    if not args.no_ablation and rank == 0:
        ablation = ablation_measure()

    out = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if not args.mapping_only else WORKLOAD + " (mapping iterations only)",
                   "width": W, "height": H, "gaussians": N_MAP, "gt_gaussians": N_GT,
                   "iters_per_step": iters_per_step, "tile": args.tile, "batch_depth": args.batch,
                   "l2": "inputs larger than L2 (map + optimiser state + pair lists >> 129 MB)",
                   "final_gaussians": pipe.live_count(), "pairs_last": pipe.last_pairs(),
                   "parallelism": f"replicas x{world}"},
        "clocks": clocks, "gpu_launches": int(launches), "e2e": e2e, "roofline": roof,
        "peaks_measured": {k: (round(v, 2) if isinstance(v, float) else v) for k, v in measured.items()},
        "kernels_ms_per_step": breakdown,
        "kernels_breakdown": f"separate pass of {bd_steps} steps after the timed region, events around every call",
        "window": window,
        "iters_to_psnr": conv,
        "tracking": tracking,
        "densification_ablation": ablation,
    }
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(pipe)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def oracle_iteration(scene_np: dict, cam: dict, color_gt: np.ndarray, depth_gt: np.ndarray, rows: int, y0: int):
    """One FP64 oracle mapping iteration (project, bin, blend, eq16 loss, adjoint,
    eq15, Adam) on a horizontal band of `rows` image rows starting at y0.  Returns
    the estimated seconds of a full-frame iteration: the per-Gaussian stages as
    timed plus the per-pixel stages scaled by H / rows."""
    from oracle import render as orr
    band = dict(cam)
    band["height"], band["cy"] = rows, cam["cy"] - y0
    cg = np.ascontiguousarray(color_gt[:, y0:y0 + rows], np.float64)
    dg = np.ascontiguousarray(depth_gt[y0:y0 + rows], np.float64)
    t0 = time.perf_counter()
    sa = orr.aos(scene_np)
    pr = orr.project(sa, band)
    t1 = time.perf_counter()
    _, ids, ranges = orr.bin_sort([band], 16, 16, pr["depth"][None].astype(np.float32), pr["radius"][None],
                                  pr["rect"][None])
    out = orr.render_fwd(pr, sa["rgb"], band, ids, ranges)
    _, dC, dD = orr.loss(out["color"], out["depth"], cg, dg, 0.9, 0.1, 0.1)
    g2, grgb = orr.render_bwd(pr, sa["rgb"], band, ids, ranges, dC, dD)
    t2 = time.perf_counter()
    grads = orr.project_bwd(sa, band, g2)
    grads["rgb"] = grgb
    _, greg = orr.scale_reg(sa["log_scales"], 0.01)
    grads["log_scales"] += greg
    lrs = {"means": 1e-3, "log_scales": 5e-3, "quats": 1e-3, "logits": 5e-2, "rgb": 2.5e-3}
    for k, lr in lrs.items():
        p = sa[k].reshape(-1)
        orr.adam(p, np.ascontiguousarray(grads[k].reshape(-1)), np.zeros_like(p), np.zeros_like(p), lr, t=1)
    t3 = time.perf_counter()
    per_gauss = (t1 - t0) + (t3 - t2)
    per_pix = t2 - t1
    return per_gauss + per_pix * (cam["height"] / rows), (t3 - t0)


def cpu_baseline(pipe, budget_s: float = 12.0):
    """The FP64 oracle's mapping iteration on a bounded sample of the workload: the
    map as the GPU left it and the last frame; a band of rows first, then whole
    frames repeated while they fit in about budget_s seconds."""
    from oracle import render as orr
    k = (len(pipe.cams) - 1)
    cam = pipe.cams[k]
    scene = pipe.g.to_scene(pipe.live_count())
    color = pipe.colors[k].view(3, H, W).cpu().numpy()
    depth = pipe.depths[k].view(H, W).cpu().numpy()
    y0 = (H // 2 // 16) * 16
    est, wall = oracle_iteration(scene, cam, color, depth, 32, y0)
    if est * 1.2 < budget_s:
        runs, t0 = [], time.perf_counter()
        while not runs or (time.perf_counter() - t0) + est < budget_s:
            e, _ = oracle_iteration(scene, cam, color, depth, H, 0)
            runs.append(e)
        est = float(np.mean(runs))
        sample = (f"{len(runs)} full-frame mapping iteration(s) (1200x680, {pipe.live_count()} Gaussians), "
                  f"{time.perf_counter() - t0:.1f} s wall")
    else:
        sample = (f"one mapping iteration on rows {y0}-{y0 + 32} of 680 ({pipe.live_count()} Gaussians); "
                  f"{wall:.1f} s wall, per-pixel stages scaled by {H / 32:.1f}")
    cores = orr.num_threads()
    # the same iteration on one core: a band of 32 rows, per-pixel stages scaled to the frame
    prev = orr.set_num_threads(1)
    try:
        est1, wall1 = oracle_iteration(scene, cam, color, depth, 32, y0)
    finally:
        orr.set_num_threads(prev)
    return {"value": 1.0 / est, "unit": "iters/s", "cores": cores, "kind": "oracle", "sample": sample,
            "one_core": {"value": 1.0 / est1, "unit": "iters/s", "cores": 1,
                         "sample": f"one mapping iteration on rows {y0}-{y0 + 32} of 680, per-pixel stages scaled "
                                   f"by {H / 32:.1f}; {wall1:.1f} s wall"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import render as orr
    from paper_2503_01109_gb300 import synthetic as syn

    n_frames = args.warmup + args.steps
    cams = syn.trajectory(n_frames, seed=100, width=W, height=H, f=F)
    scene = syn.room_scene(N_MAP, seed=0, kind="map")
    gt = syn.room_scene(N_GT, seed=1000, kind="gt")

    def target(cam, rows, y0):
        band = dict(cam)
        band["height"], band["cy"] = rows, cam["cy"] - y0
        ref = orr.render_views(gt, [band])["out"][0]          # target (untimed set-up)
        color = np.zeros((3, H, W)); depth = np.zeros((H, W))
        color[:, y0:y0 + rows] = ref["color"]
        depth[y0:y0 + rows] = np.where(ref["alpha"] > 0.5, ref["depth"] / np.maximum(ref["alpha"], 1e-6), 0.0)
        return color, depth

    # size each step: whole frames when the run fits in ~150 s, else a band of rows
    y0 = (H // 2 // 16) * 16
    c, d = target(cams[0], 32, y0)
    probe, _ = oracle_iteration(scene, cams[0], c, d, 32, y0)
    rows, y0 = (H, 0) if probe * n_frames < 150.0 else (32, y0)
    est = []
    for k in range(n_frames):
        c, d = target(cams[k], rows, y0)
        e, _ = oracle_iteration(scene, cams[k], c, d, rows, y0)
        if k >= args.warmup:
            est.append(e)
    ms = 1e3 * float(np.mean(est))
    value = 1e3 / ms
    desc = (f"FP64 C oracle, one mapping iteration per step on rows {y0}-{y0 + rows} of 680 with the full 1M map"
            + ("" if rows == H else f"; per-pixel stages scaled by {H / rows:.1f}"))
    out = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "width": W, "height": H, "gaussians": N_MAP},
           "cpu_baseline": {"value": value, "unit": "iters/s", "cores": orr.num_threads(), "kind": "oracle",
                            "sample": desc},
           "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
