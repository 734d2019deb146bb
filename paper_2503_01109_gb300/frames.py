"""Per-frame mapping pipeline over a camera trajectory (the benchmark workload).

For every frame: render the map at the frame's pose (eq1's colour, depth and
opacity readings), seed new Gaussians with the Fourier analysis of Sec. III-A
(eq2-eq11, plus the learned prior when one is given), then run a few mapping
iterations (Sec. III-D).  The live Gaussian count stays on the device, so a
frame needs no host synchronisation.

Ground-truth frames are renders of a separate seeded scene made with the same
library (colour, and depth normalised by the rendered opacity where it exceeds
0.5, else 0 = invalid), standing in for an RGB-D sensor.
"""
from __future__ import annotations

import hashlib
import os
import re

import numpy as np
import torch

from . import fgs
from .mapping import Mapper, PAPER_LOSS, PAPER_REG


class KernelTimer:
    """CUDA events around selected library calls on the current stream.

    An event between two launches ends the overlap of programmatic dependent
    launch there, so a measurement of whole steps times only the spans it needs
    (`enable(names)`) and leaves the others to a separate breakdown pass."""

    def __init__(self):
        self.on = False
        self.only = None
        self.events = {}

    def enable(self, names=None):
        self.on = True
        self.only = None if names is None else set(names)
        self.events = {}

    def disable(self):
        self.on = False

    def active(self, name) -> bool:
        return self.on and (self.only is None or name in self.only)

    def span(self, name):
        timer = self

        class _Span:
            def __enter__(self_):
                self_.live = timer.active(name)
                if self_.live:
                    self_.e0 = torch.cuda.Event(enable_timing=True)
                    self_.e0.record(torch.cuda.current_stream())

            def __exit__(self_, *a):
                if self_.live:
                    e1 = torch.cuda.Event(enable_timing=True)
                    e1.record(torch.cuda.current_stream())
                    timer.events.setdefault(name, []).append((self_.e0, e1))
        return _Span()

    def durations(self, name):
        return [a.elapsed_time(b) for a, b in self.events.get(name, [])]

    def summary(self, steps):
        return {k: round(sum(self.durations(k)) / max(steps, 1), 4) for k in self.events}


class TimedMapper(Mapper):
    """Mapper whose render and adjoint calls are bracketed by timer spans and whose
    per-launch work (sum of per-pixel contributor counts) is snapshotted."""

    def __init__(self, *a, timer: KernelTimer | None = None, **kw):
        super().__init__(*a, **kw)
        self.timer = timer or KernelTimer()
        self.nc_snap = []          # (render belongs to an iteration, n_contrib copy)
        self._in_iteration = False

    def render(self, sample_stride: int = 1):
        with self.timer.span("project"):
            fgs.fgs_project(self.g, self.cams, self.til, self.proj, self.status, self.use_dc)
        n = self.g.capacity if self.use_dc else self.g.n
        with self.timer.span("bin_sort"):
            fgs.fgs_bin_sort(self.proj, n, self.cams, self.til, self.ws_bin, self.tile_keys, self.ids, self.ranges,
                             self.num_pairs, self.status, d_n=self.g.d_n if self.use_dc else None)
        with self.timer.span("render_fwd" if sample_stride == 1 else "render_fwd_sampled"):
            self._blend(sample_stride)
        with self.timer.span("tile_order"):
            self._order()
        if self.timer.on and sample_stride == 1:  # the roofline covers the full-frame renders
            snap = torch.empty_like(self.frame.n_contrib)
            fgs.fgs_memcpy_async(snap, self.frame.n_contrib)   # copy engine; summed after timing
            self.nc_snap.append((self._in_iteration, snap))

    def backward(self, dC, dD, dA=None):
        fgs.fgs_memset_async(self.grads.buf)
        fgs.fgs_memset_async(self.grad2d)
        with self.timer.span("render_bwd"):
            fgs.fgs_render_bwd_splats(self.g, self.proj, self.cams, self.til, self.ids, self.ranges, self.frame, dC,
                                      dD, dA, self.grad2d, self.grads, self.status, self.use_dc,
                                      tile_order=self.tile_order)
        with self.timer.span("project_bwd"):
            fgs.fgs_project_bwd(self.g, self.proj, self.cams, self.grad2d, self.grads, self.use_dc)
        self._clean = False

    def iteration(self):
        self._in_iteration = True
        self.render()
        self._in_iteration = False
        fgs.fgs_memset_async(self.loss_acc)
        with self.timer.span("loss"):
            fgs.fgs_loss(self.cams, self.frame.color, self.frame.depth, self.color_gt, self.depth_gt, *self.loss_w,
                         self.dC, self.dD, self.loss_acc, self.ws_loss)
        if self.fused_tail:
            self.ensure_clean()
            with self.timer.span("render_bwd"):
                fgs.fgs_render_bwd_splats(self.g, self.proj, self.cams, self.til, self.ids, self.ranges, self.frame,
                                          self.dC, self.dD, None, self.grad2d, self.grads, self.status, self.use_dc,
                                          tile_order=self.tile_order)
            with self.timer.span("project_bwd_adam"):
                self.fused_tail_step()
            return
        self.backward(self.dC, self.dD)
        if self.reg_w != 0.0:
            fgs.fgs_scale_reg(self.g, self.reg_w, self.grads, self.loss_acc, self.ws_reg, self.use_dc)
        self.host_step += 1
        with self.timer.span("adam"):
            fgs.fgs_adam(self.g, self.grads, self.m, self.v, self.lr, step=self.host_step,
                         d_step=self.d_step if self.use_dc else None, use_device_count=self.use_dc)


def render_targets(gt_scene: dict, cams: list, tile=(16, 16), batch=128, device="cuda"):
    """Colour and normalised depth of the ground-truth scene at every pose."""
    g = fgs.GaussianMap.from_scene(gt_scene, device=device)
    m = Mapper(g, cams[:1], fgs.tiling(*tile, batch), use_device_count=False)
    colors, depths = [], []
    for cam in cams:
        m.set_cameras([cam])
        m.render()
        A = m.frame.alpha
        D = torch.where(A > 0.5, m.frame.depth / A.clamp_min(1e-6), torch.zeros_like(A))
        colors.append(m.frame.color.clone())
        depths.append(D)
    torch.cuda.synchronize()
    m.check_status()
    del m, g
    return colors, depths


def render_targets_views(gt_scene: dict, cams: list, tile=(16, 16), batch=128, device="cuda"):
    """Targets of a view set of possibly different resolutions, concatenated as the
    library's multi-view images: (colour [3 sum HW], depth [sum HW])."""
    colors, depths = [], []
    for cam in cams:
        c, d = render_targets(gt_scene, [cam], tile, batch, device)
        colors.append(c[0])
        depths.append(d[0])
    return torch.cat(colors), torch.cat(depths)


class FramePipeline:
    def __init__(self, scene: dict, cams: list, gt_scene: dict, capacity: int, tile=(16, 16), batch=128,
                 iters_per_frame: int = 3, device="cuda", loss_w=PAPER_LOSS, reg_w=PAPER_REG, seed_params=None,
                 prior=None, extra_views: list | None = None, prune: fgs.PruneParams | None = None,
                 overlap_seeding: bool = True):
        self.cams = cams
        # Gaussian pruning after each frame's iterations (Sec. III-A): opacity below
        # 0.005 or a scale above 0.5 m (a tenth of the 4 x 3 x 3 m room's extent)
        self.prune = prune if prune is not None else fgs.prune_params(0.005, 0.5)
        self.iters = iters_per_frame
        self.kernel_timer = KernelTimer()
        self.colors, self.depths = render_targets(gt_scene, cams, tile, batch, device)
        # targets of other view sets (e.g. a keyframe window of mixed resolutions)
        self.extra = None
        if extra_views:
            self.extra = render_targets_views(gt_scene, extra_views, tile, batch, device)
        self.g = fgs.GaussianMap.from_scene(scene, capacity, device)
        self.mapper = TimedMapper(self.g, cams[:1], fgs.tiling(*tile, batch), loss_w=loss_w, reg_w=reg_w,
                                  use_device_count=True, timer=self.kernel_timer, keep_tile_keys=False)
        from .seeding import Seeder
        self.seeder = Seeder(self.mapper, seed_params, prior)
        self.side = torch.cuda.Stream(device=device) if overlap_seeding else None
        self.loss_host = torch.zeros(1, dtype=torch.float32).pin_memory()
        self.stage_c = torch.zeros_like(self.colors[0])
        self.stage_d = torch.zeros_like(self.depths[0])

    # ------------------------------------------------------------------------------
    def _use_frame(self, k: int, from_host=None):
        self.mapper.set_cameras([self.cams[k]])
        if from_host is None:       # frames already resident in HBM: point at them
            self.mapper.color_gt = self.colors[k]
            self.mapper.depth_gt = self.depths[k]
        else:                       # end-to-end: copy this frame from pinned host memory (C ABI)
            c, d = from_host
            fgs.fgs_memcpy_async(self.stage_c, c)
            fgs.fgs_memcpy_async(self.stage_d, d)
            self.mapper.color_gt, self.mapper.depth_gt = self.stage_c, self.stage_d

    def mapping_step(self, k: int, from_host=None):
        self._use_frame(k % len(self.cams), from_host)
        self.mapper.iteration()

    def frame_step(self, k: int, from_host=None):
        self._use_frame(k % len(self.cams), from_host)
        cam = self.cams[k % len(self.cams)]
        # The seeding's frame-only half (the FFTs, E and its threshold) runs on a
        # second stream beside the render at the frame's pose, whose projection and
        # binning kernels leave SMs idle; the seeds wait for both.
        if self.side is not None:
            self.side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(self.side):
                self.seeder.compute_energy(self.mapper.color_gt, cam)
        with self.kernel_timer.span("seed"):
            self.seeder.seed_frame(self.mapper.color_gt, self.mapper.depth_gt, cam, energy_stream=self.side)
        for _ in range(self.iters):
            self.mapper.iteration()
        with self.kernel_timer.span("prune"):
            self.mapper.prune(self.prune)

    # ------------------------------------------------------------------------------
    def check(self):
        torch.cuda.synchronize()
        self.mapper.check_status()

    def live_count(self) -> int:
        return int(self.g.d_n.item())

    def last_pairs(self) -> int:
        return int(self.mapper.num_pairs.item())

    def e2e_measure(self, warmup: int, steps: int, step_fn):
        """The same steps with each frame's colour + depth copied from pinned host
        memory and the loss read back to the host inside the timed region, both
        through the library's fgs_memcpy_async with host pointers."""
        hosts = [(c.cpu().pin_memory(), d.cpu().pin_memory()) for c, d in zip(self.colors, self.depths)]
        h2d = hosts[0][0].numel() * 4 + hosts[0][1].numel() * 4
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(warmup, warmup + steps):
            step_fn(k, from_host=hosts[k % len(hosts)])
            fgs.fgs_memcpy_async(self.loss_host, self.mapper.loss_acc)     # device -> pinned host
        e1.record(stream)
        torch.cuda.synchronize()
        return {"ms": e0.elapsed_time(e1), "h2d": h2d, "d2h": 4}

    # ------------------------------------------------------------------------------
    # roofline of the dominant kernel
    # FP32 operations per blended (pixel, splat) pair, counted from the kernels'
    # arithmetic: forward = power 8, exp 2, alpha 2, compare 1, T update 2, five
    # accumulations 10, misc 2; adjoint = recompute 12, T recovery 2, dalpha 20,
    # suffix sums 10, ten gradient terms 24.
    FLOP_FWD_PAIR = 27
    FLOP_BWD_PAIR = 68

    def contributor_work(self, iterations_only: bool = False):
        """Sum over pixels of contributor counts, one entry per timed render."""
        return [int(s.sum().item()) for it, s in self.mapper.nc_snap if it or not iterations_only]

    @staticmethod
    def kernel_source_hash(kernel: str) -> str:
        """sha256 of the code a kernel is built from, comments and blank space
        removed (a code change invalidates its ncu figures, a comment does not)."""
        here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
        files = {"render_bwd": ["common.cuh", "render_tile.cuh", "render.cu"],
                 "render_fwd": ["common.cuh", "render_tile.cuh", "render.cu"]}[kernel]
        h = hashlib.sha256()
        for f in files:
            text = open(os.path.join(here, f)).read()
            text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
            text = re.sub(r"//[^\n]*", " ", text)
            h.update(" ".join(text.split()).encode())
        return h.hexdigest()[:16]

    @staticmethod
    def profiled_traffic(kernel: str, profiles_dir: str):
        """DRAM bytes per launch from the committed ncu summary of `kernel`, if its
        source hash matches the current sources; else None."""
        path = os.path.join(profiles_dir, f"{kernel}_room1M_1200x680.md")
        try:
            text = open(path).read()
        except OSError:
            return None
        m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+);\s*source_sha256:\s*([0-9a-f]+)", text)
        if not m or m.group(2) != FramePipeline.kernel_source_hash(kernel):
            return None
        return float(m.group(1))

    # MUFU evaluations per pair: the forward's ex2; the adjoint's ex2 and 1 / (1 - alpha)
    MUFU_FWD_PAIR = 1
    MUFU_BWD_PAIR = 2

    def roofline(self, peaks: dict, profiles_dir: str | None = None, total_ms: float | None = None,
                 measured: dict | None = None):
        """The dominant render kernel against the FP32 FMA rate, from the launches
        timed since the timer was enabled; share_of_step relative to total_ms (the
        timed region) when given, else to the sum of the timed spans.  `measured`
        holds the on-chip rates fgs.measure_peaks() measured on this device (FP32
        FMA, MUFU ex2); without it the FP32 peak is derived from the SM count the
        library reports, 128 FP32 lanes, 2 FLOP per FMA and the maximum SM clock."""
        t = self.kernel_timer
        totals = {k: sum(t.durations(k)) for k in t.events}
        if not totals:
            return None
        fwd = t.durations("render_fwd")
        bwd = t.durations("render_bwd")
        name = max(("render_fwd", "render_bwd"), key=lambda k: totals.get(k, 0.0))
        durs = fwd if name == "render_fwd" else bwd
        per_pair = self.FLOP_FWD_PAIR if name == "render_fwd" else self.FLOP_BWD_PAIR
        mufu_pair = self.MUFU_FWD_PAIR if name == "render_fwd" else self.MUFU_BWD_PAIR
        # the bwd of iteration i walks the lists rendered by the fwd of iteration i;
        # the seeding render of a frame has no backward
        w = self.contributor_work(iterations_only=(name == "render_bwd"))
        n = min(len(w), len(durs))
        if n == 0:
            return None
        pairs = np.array(w[-n:], np.float64)
        secs = np.array(durs[-n:], np.float64) / 1e3
        achieved = float(np.mean(pairs * per_pair / secs)) / 1e12
        if measured and measured.get("fp32_fma_tflops"):
            peak = float(measured["fp32_fma_tflops"])
            source = (f"measured: fgs_peak_probe FP32 FMA on this device ({measured.get('sms')} SMs), "
                      "best of 3 launches of ~20 ms")
        else:
            sm_max = float(peaks.get("sm_max_mhz", 2070.0))
            peak = fgs.fgs_num_sms() * 128 * 2 * sm_max * 1e6 / 1e12
            source = "derived: SMs (library) x 128 FP32 lanes x 2 x max SM clock (MEASURED_PEAKS sm_max_mhz)"
        traffic = self.profiled_traffic(name, profiles_dir) if profiles_dir else None
        out = {"kernel": name, "bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2),
               "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": traffic,
               "traffic_unit": "bytes per launch (DRAM read + write, ncu)", "peak_source": source,
               "flop_per_pair": per_pair, "pairs_per_launch": float(np.mean(pairs)),
               "share_of_step": round(totals[name] / (total_ms or sum(totals.values())), 3),
               "avg_launch_ms": round(float(np.mean(durs)), 4)}
        if measured and measured.get("mufu_ex2_gops"):
            mufu = float(np.mean(pairs * mufu_pair / secs)) / 1e9
            out["mufu"] = {"achieved_gops": round(mufu, 1), "peak_gops": round(float(measured["mufu_ex2_gops"]), 1),
                           "frac": round(mufu / float(measured["mufu_ex2_gops"]), 4), "per_pair": mufu_pair}
        return out
