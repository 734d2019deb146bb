"""Iterations and wall time to a fixed PSNR: the plain per-view Fourier-prior
loop against the batched keyframe window with the learned prior.

Both loops start from an empty map and process a trajectory frame by frame, as
the paper's mapping does (Sec. III-A, III-D): seed the frame (eq2-eq11, with
the eq11 radius or the learned prior), then run mapping iterations until the
render of the frame reaches the target PSNR (or an iteration cap).  The plain
loop optimises the current view only; the batched loop optimises the current
view together with the previous keyframes in one persistent window launch.

The learned prior is trained on pairs the plain loop itself produces: the
features of every seed pixel at seeding time and the seed's parameters after the
whole training trajectory has been mapped (log-scales sorted in decreasing order,
opacity logit).

PSNR here is a measurement (10 log10(1 / MSE) of colour in [0, 1]), computed
with torch outside the mapping step.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import fgs
from .mapping import Mapper
from .prior import PriorMLP, features as prior_features
from .seeding import Seeder
from .window import KeyframeSelector, Window


def psnr(color: torch.Tensor, target: torch.Tensor) -> float:
    mse = torch.mean((color.clamp(0, 1) - target) ** 2).item()
    return 10.0 * math.log10(1.0 / max(mse, 1e-12))


class SlamLoop:
    """Frame-by-frame mapping from an empty map."""

    def __init__(self, colors, depths, cams, capacity: int, prior: PriorMLP | None = None, window: int = 1,
                 tiling: fgs.Tiling | None = None, target_psnr: float = 30.0, max_iters: int = 60,
                 seed_params: fgs.SeedParams | None = None, record_seeds: bool = False,
                 selector: KeyframeSelector | None = None, track_map: bool = False):
        """window > 1: optimise the current frame with earlier keyframes -- the
        window - 1 previous frames, or, with `selector`, the co-visible and random
        keyframes it picks among all earlier frames (at most window - 1)."""
        self.colors, self.depths, self.cams = colors, depths, cams
        self.target, self.max_iters, self.window = target_psnr, max_iters, window
        self.selector = selector
        self.g = fgs.GaussianMap(capacity, "cuda", 0)
        self.til = tiling or fgs.tiling(16, 16, 128)
        self.mapper = Mapper(self.g, [cams[0]], self.til, use_device_count=True)
        self.seeder = Seeder(self.mapper, seed_params, prior)
        self.win = None
        self.record = record_seeds
        self.track_map = track_map
        self.seed_log = []   # (first index, count, features [n][272])
        self.frames = []     # per frame: iterations, seconds, final psnr

    def _window_for(self, k: int, picked: list | None = None):
        ks = sorted(picked) + [k] if picked is not None else list(range(max(0, k - self.window + 1), k + 1))
        cams = [self.cams[j] for j in ks]
        if self.win is None or len(self.win.cams) != len(cams):
            self.win = None   # release the previous window's buffers first
            self.win = Window(self.g, cams, self.til, pair_capacity=32_000_000 * len(cams))
        else:
            self.win.set_cameras(cams)
        self.win.color_gt = torch.cat([self.colors[j] for j in ks])
        self.win.depth_gt = torch.cat([self.depths[j] for j in ks])
        return self.win

    def run_frame(self, k: int):
        cam = self.cams[k]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        base = int(self.g.d_n.item()) if self.record else 0
        self.seeder.seed_frame(self.colors[k], self.depths[k], cam, first_frame=(k == 0))
        if self.record:
            n_new = int(self.seeder.num_new.item())
            xy = self.seeder.seed_xy[:n_new].clone()
            W, H = cam["width"], cam["height"]
            hi = (self.seeder.mask[(xy[:, 1] * W + xy[:, 0]).long()] & 1).bool()   # M_h at the seed pixel
            self.seed_log.append((base, n_new, prior_features(self.colors[k], self.depths[k], W, H, xy), hi))
        it, p = 0, 0.0
        use_window = self.window > 1 and k > 0
        picked = None
        if use_window and self.selector is not None:
            self.selector.max_k = self.window - 1
            picked = self.selector.select(self.depths[k].reshape(cam["height"], cam["width"]), cam, self.cams[:k])
            use_window = len(picked) > 0
        while it < self.max_iters:
            if use_window:
                w = self._window_for(k, picked)
                w.iteration()
                f = w.frame.view(len(w.cams) - 1)["color"].reshape(-1)
            else:
                self.mapper.set_cameras([cam])
                self.mapper.color_gt, self.mapper.depth_gt = self.colors[k], self.depths[k]
                self.mapper.iteration()
                f = self.mapper.frame.color
            it += 1
            if math.isfinite(self.target):
                p = psnr(f, self.colors[k])      # the render this iteration optimised
                if p >= self.target:
                    break
        torch.cuda.synchronize()
        self.frames.append({"iters": it, "seconds": time.perf_counter() - t0, "psnr": p,
                            "gaussians": int(self.g.d_n.item())})
        if self.track_map:   # the map's quality over every frame seen so far (not timed)
            self.frames[-1]["map_psnr_seen"] = self.evaluate_all(k + 1)

    def run(self, n_frames: int | None = None):
        for k in range(n_frames or len(self.cams)):
            self.run_frame(k)
        self.mapper.check_status()
        return self.frames

    def evaluate_all(self, n_frames: int | None = None) -> float:
        """Mean PSNR of the map over the first n_frames frames (all by default)."""
        vals = []
        for k, cam in enumerate(self.cams[:n_frames]):
            self.mapper.set_cameras([cam])
            self.mapper.render()
            vals.append(psnr(self.mapper.frame.color, self.colors[k]))
        return float(np.mean(vals))

    def training_pairs(self, high_only: bool = True):
        """(features [n][272] int16, targets [n][4] float32) of the recorded seeds
        (high-frequency ones only by default), targets from the map's current
        parameters: log-scales sorted in decreasing order, opacity logit."""
        feats, targs = [], []
        ls = self.g.plane("log_scales")
        lg = self.g.plane("logits")[0]
        for base, n, f, hi in self.seed_log:
            if n == 0:
                continue
            s = ls[:, base:base + n].t()
            s_sorted = torch.sort(s, dim=1, descending=True).values
            t = torch.cat([s_sorted, lg[base:base + n, None]], 1)
            sel = hi if high_only else torch.ones_like(hi)
            targs.append(t[sel])
            feats.append(f[sel])
        return torch.cat(feats).contiguous(), torch.cat(targs).contiguous()


def opacity_weighted(feats: torch.Tensor, targets: torch.Tensor, seed: int = 0):
    """Resamples the pairs with probability proportional to the converged opacity,
    so that seeds the optimiser faded out (redundant, about to be pruned) weigh
    little and the opaque ones that make the image dominate the regression."""
    w = torch.sigmoid(targets[:, 3]).double()
    g = torch.Generator(device=feats.device).manual_seed(seed)
    idx = torch.multinomial(w, feats.shape[0], replacement=True, generator=g)
    return feats[idx].contiguous(), targets[idx].contiguous()


def train_prior(feats: torch.Tensor, targets: torch.Tensor, epochs: int = 4, batch: int = 8192, lr: float = 1e-3,
                seed: int = 0, prior: PriorMLP | None = None):
    """Mini-batch Adam on the pairs; returns the prior and the per-epoch mean losses."""
    prior = prior or PriorMLP()
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = feats.shape[0]
    history = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).to(feats.device)
        losses = []
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            losses.append(prior.train_step(feats[idx].contiguous(), targets[idx].contiguous(), lr=lr).clone())
        history.append(float(torch.stack(losses).mean().item()) if losses else float("nan"))
    return prior, history


def summarise(frames: list, target: float | None = None) -> dict:
    it = [f["iters"] for f in frames]
    out = {"frames": len(frames), "iters_total": int(sum(it)), "iters_per_frame": float(np.mean(it)),
           "seconds_total": float(sum(f["seconds"] for f in frames)),
           "psnr_at_stop_mean": float(np.mean([f["psnr"] for f in frames])),
           "gaussians": frames[-1]["gaussians"] if frames else 0}
    if target is not None:
        out["frames_reaching_target"] = int(sum(1 for f in frames if f["psnr"] >= target))
    if frames and "map_psnr_seen" in frames[0]:
        out["map_psnr_seen_mean"] = float(np.mean([f["map_psnr_seen"] for f in frames]))
    return out


def init_error(prior: PriorMLP, feats: torch.Tensor, targets: torch.Tensor, depth: torch.Tensor, f: float,
               alpha_h: float = 1.0, init_logit: float = 0.0) -> dict:
    """Mean squared distance to the converged parameters of (a) the learned
    prior's initial values and (b) eq11's (log-scale log(alpha_h d / f) on every
    axis, logit init_logit), for high-frequency seeds with depth d."""
    pred = prior.infer(feats)
    ls = torch.log(alpha_h * depth / f)[:, None].expand(-1, 3)
    eq11 = torch.cat([ls, torch.full_like(depth[:, None], init_logit)], 1)
    return {"learned": float(((pred - targets) ** 2).mean().item()),
            "eq11": float(((eq11 - targets) ** 2).mean().item()),
            "learned_scale": float(((pred[:, :3] - targets[:, :3]) ** 2).mean().item()),
            "eq11_scale": float(((eq11[:, :3] - targets[:, :3]) ** 2).mean().item()),
            "learned_logit": float(((pred[:, 3] - targets[:, 3]) ** 2).mean().item()),
            "eq11_logit": float(((eq11[:, 3] - targets[:, 3]) ** 2).mean().item())}


def collect_pairs(runs, capacity: int, train_iters: int, target_pairs: int, time_budget_s: float = 120.0):
    """Training pairs of the learned prior from plain mapping runs: each run maps
    its trajectory from an empty map (eq11 seeding, `train_iters` iterations per
    frame) and yields the features of its high-frequency seeds and their
    parameters at the end of the run.  Runs are taken in order until
    `target_pairs` pairs or the time budget is reached.  Returns (features,
    targets, per-run pair counts)."""
    feats, targs, counts = [], [], []
    total, t0 = 0, time.perf_counter()
    for colors, depths, cams in runs:
        rec = SlamLoop(colors, depths, cams, capacity, target_psnr=math.inf, max_iters=train_iters,
                       record_seeds=True)
        rec.run()
        f, t = rec.training_pairs(high_only=True)
        feats.append(f)
        targs.append(t)
        counts.append(int(f.shape[0]))
        total += int(f.shape[0])
        del rec
        if total >= target_pairs or time.perf_counter() - t0 > time_budget_s:
            break
    return torch.cat(feats), torch.cat(targs), counts


def compare(train_runs, gt_colors_test, gt_depths_test, cams_test, capacity: int, target_psnr: float = 30.0,
            train_iters: int = 40, max_iters: int = 100, epochs: int = 8, window: int = 8,
            target_pairs: int = 2_000_000, batch: int = 8192) -> dict:
    """The whole experiment: pairs from plain mapping runs (configuration-2/3-like
    trajectories, `train_runs` = [(colours, depths, cameras)]), prior training on
    the GPU, then on a test trajectory of another scene four loops from an empty
    map -- the plain per-view loop, the per-view loop with the learned prior, the
    batched window of the current frame and up to window - 1 co-visible and
    random keyframes (Sec. III-C) without and with the learned prior -- each run
    until the current frame reaches target_psnr (at most max_iters iterations per
    frame; a window iteration renders all its views).  Reported per loop: the
    iterations and wall time to the target, and the map's PSNR over all frames
    seen so far after each frame (its mean) and over the whole trajectory at the
    end."""
    t0 = time.perf_counter()
    feats, targs, counts = collect_pairs(train_runs, capacity, train_iters, target_pairs)
    t_pairs = time.perf_counter() - t0
    t1 = time.perf_counter()
    fw, tw = opacity_weighted(feats, targs)
    n_train = int(0.95 * fw.shape[0])
    prior, hist = train_prior(fw[:n_train], tw[:n_train], epochs=epochs, batch=batch)
    held_f, held_t = fw[n_train:], tw[n_train:]
    d = held_f[:, 256].to(torch.int32).bitwise_left_shift(16).view(torch.float32)
    cam = cams_test[0]
    err = init_error(prior, held_f, held_t, d, 0.5 * (cam["fx"] + cam["fy"]))
    t_train = time.perf_counter() - t1  # weighting, training and the held-out error
    out = {"target_psnr": target_psnr, "pairs": int(feats.shape[0]), "pairs_per_run": counts,
           "pairs_seconds": t_pairs, "train_loss": hist, "init_mse_held_out": err, "train_seconds": t_train}
    del feats, targs
    variants = (("plain", None, 1), ("learned_prior", prior, 1), ("window", None, window),
                ("learned_prior_window", prior, window))
    for name, pr, win in variants:
        sel = KeyframeSelector(seed=0, max_keyframes=window - 1) if win > 1 else None
        L = SlamLoop(gt_colors_test, gt_depths_test, cams_test, capacity, prior=pr, window=win,
                     target_psnr=target_psnr, max_iters=max_iters, selector=sel, track_map=True)
        L.run()
        res = summarise(L.frames, target_psnr)
        res["psnr_all_frames_end"] = L.evaluate_all()
        out[name] = res
        del L
    p, lp, w, lw = (out[k] for k in ("plain", "learned_prior", "window", "learned_prior_window"))
    out["verdict"] = {
        "learned_vs_plain_iters": lp["iters_total"] / max(p["iters_total"], 1),
        "learned_vs_plain_seconds": lp["seconds_total"] / max(p["seconds_total"], 1e-9),
        "learned_window_vs_plain_iters": lw["iters_total"] / max(p["iters_total"], 1),
        "learned_window_vs_plain_seconds": lw["seconds_total"] / max(p["seconds_total"], 1e-9),
        "learned_window_vs_plain_map_psnr_db": lw["psnr_all_frames_end"] - p["psnr_all_frames_end"],
        "window_vs_plain_map_psnr_db": w["psnr_all_frames_end"] - p["psnr_all_frames_end"]}
    return out
